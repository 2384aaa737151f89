"""Tuning knobs on the GPU: every quadrature-node block shape and tile shape
of fdx_tuning gives the oracle's pattern within the parity gates, the same
in-support term counts (the set of terms does not depend on the shapes, only
the order of the node sums does), the adjoint within 1e-4 of the oracle
adjoint, and the batched step stays bitwise equal to the per-model entry
points under a non-default setting."""
import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import L2_REL, MAX_REL, api_precision, oracle_hkl, parity

pytestmark = pytest.mark.gpu

ADJ_TOL = 1e-4


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


@pytest.fixture
def tuned(gpu):
    """Set a tuning for one test and restore the defaults afterwards."""
    def apply(**knobs):
        gpu.fdx_set_tuning(gpu.Tuning.of(**knobs))
    yield apply
    gpu.fdx_set_tuning(None)


def _forward(gpu, p, hkl, M):
    import torch
    hk = torch.as_tensor(np.ascontiguousarray(hkl, np.int32), device="cuda").reshape(-1, 3)
    Mt = torch.as_tensor(np.ascontiguousarray(M, np.float32), device="cuda")
    prob = gpu.make_problem(p.cell, p.br, p.geom, hk, Mt)
    img = torch.empty((p.geom.n_y, p.geom.n_x), dtype=torch.float32, device="cuda")
    gpu.fdx_pattern([prob], [img])
    cnt = torch.empty((p.geom.n_y, p.geom.n_x), dtype=torch.int32, device="cuda")
    gpu.fdx_pattern_evals(prob, cnt)
    torch.cuda.synchronize()
    return img.cpu().numpy().reshape(-1), cnt.cpu().numpy().reshape(-1)


def _fine_helix():
    """The reduced helix with 0.2 mm pixels: its 8 x 8 patches span less than
    half a lattice period, so the kernels take two pixels per lane (the other
    reduced workloads take one)."""
    from dataclasses import replace
    p = W.small_helix()
    return replace(p, geom=replace(p.geom, pixel=0.2))


@pytest.mark.parametrize("make", [W.small_helix, W.small_triclinic, W.small_tilted, W.small_sinc, _fine_helix])
def test_node_block_shapes_forward(gpu, orc, tuned, make):
    p = api_precision(make())
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl).astype(np.float32)
    I, E = orc.pattern(p, hkl, M.astype(np.float64))
    counts = None
    for ppl in (2, 1):
        for nb in range(4):
            tuned(node_block=nb, ppl_max=ppl)
            img, cnt = _forward(gpu, p, hkl, M)
            mr, l2 = parity(img, I)
            assert mr <= MAX_REL and l2 <= L2_REL, (ppl, nb, mr, l2)
            assert np.all(cnt >= E[:, 1]) and np.all(cnt <= E[:, 2]), (ppl, nb)
            if counts is None:
                counts = cnt
            assert np.array_equal(cnt, counts), (ppl, nb)


def _close(got, ref, what):
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= ADJ_TOL and l2 <= ADJ_TOL, (what, err, l2)


@pytest.mark.parametrize("make", [W.small_helix, _fine_helix])
@pytest.mark.parametrize("nb", [0, 2, 3])
def test_node_block_shapes_adjoint(gpu, orc, tuned, nb, make):
    """The adjoint of the helix model for a seeded upstream gradient (the
    model's own loss gradient against a perturbed target, so the sums are
    not dominated by cancellation) under each non-default block shape."""
    import torch
    p = api_precision(make())
    tuned(node_block=nb)
    sim = gpu.Simulation(p)
    img = sim.forward()
    rng = np.random.default_rng(23)
    target = img.cpu().numpy() * (1.0 + 0.2 * rng.uniform(-1, 1, img.shape))
    gI = torch.empty_like(img)
    It = torch.as_tensor(target.astype(np.float32), device="cuda")
    gpu.fdx_loss(img, It, None, dL_dI=gI)
    na, n = p.atoms.n, sim.hkl.shape[0]
    dfrac = torch.empty((na, 3), dtype=torch.float64, device="cuda")
    dB = torch.empty(na, dtype=torch.float64, device="cuda")
    dg = torch.empty(8, dtype=torch.float64, device="cuda")
    dM = torch.empty(n, dtype=torch.float32, device="cuda")
    gpu.fdx_pattern_backward(sim.prob, sim.atoms, sim.F, gI, dfrac, dB, dg, dM)
    torch.cuda.synchronize()
    hkl = oracle_hkl(orc, p, sim.hkl_host)
    gIo = gI.cpu().numpy().astype(np.float64).reshape(-1)
    F = orc.structure_factors(p.cell, p.atoms, hkl)
    _, P, DW = orc.refl_scalars(p, hkl)
    G, dbeta, dsig, dgam = orc.pattern_adjoint(p, hkl, np.abs(F) ** 2 * P * DW, gIo)
    dL, dgo = orc.chain_globals(p, hkl, np.abs(F) ** 2, G, dbeta)
    dfo, dBo = orc.sf_adjoint(p.cell, p.atoms, hkl, F, G * P * DW)
    _close(dM.cpu().numpy(), G, "dM")
    _close(dfrac.cpu().numpy(), dfo, "dfrac")
    _close(dB.cpu().numpy(), dBo, "dB")
    glob = dg.cpu().numpy()
    ref = np.concatenate([dL, dgo, [dsig, dgam]])
    for k in range(8):
        if ref[k] == 0.0:
            assert abs(glob[k]) <= 1e-6 * np.max(np.abs(ref)), k
        else:
            assert glob[k] == pytest.approx(ref[k], rel=ADJ_TOL), k


def test_batch_bitwise_under_tuning(gpu, tuned):
    """fdx_batch_refine against the per-model entry points with a
    non-default block shape, tile shape and launch shape."""
    import torch
    tuned(node_block=3, ppl_max=1, fwd_ctas_per_sm=3, adj_ctas_per_sm=2, adj_bands=32)
    models = [api_precision(p) for p in W.small_batch(3)]
    sims = [gpu.Simulation(p) for p in models]
    tims = [gpu.Simulation(api_precision(W.config4_target(p, m))).forward().clone() for m, p in enumerate(models)]
    ref = []
    for s, It in zip(sims, tims):
        s.forward()
        gI = torch.empty_like(s.image)
        loss, _ = gpu.fdx_loss(s.image, It, None, dL_dI=gI)
        na = s.atoms.frac.shape[0]
        dfrac = torch.empty((na, 3), dtype=torch.float64, device="cuda")
        dB = torch.empty(na, dtype=torch.float64, device="cuda")
        dg = torch.empty(8, dtype=torch.float64, device="cuda")
        gpu.fdx_pattern_backward(s.prob, s.atoms, s.F, gI, dfrac, dB, dg, None)
        ref.append((s.image.clone(), loss.clone(), dfrac, dB, dg))
    step = gpu.BatchStep([s.prob for s in sims], [s.atoms for s in sims], targets=tims)
    step()
    torch.cuda.synchronize()
    for m, (img, loss, dfrac, dB, dg) in enumerate(ref):
        assert torch.equal(step.images[m], img), m
        assert step.losses[m].item() == loss.item(), m
        assert torch.equal(step.dfrac[m], dfrac), m
        assert torch.equal(step.dB[m], dB), m
        assert torch.equal(step.dglobal[m], dg), m


def test_tuning_validation(gpu):
    with pytest.raises(RuntimeError):
        gpu.fdx_set_tuning(gpu.Tuning.of(node_block=4))
    with pytest.raises(RuntimeError):
        gpu.fdx_set_tuning(gpu.Tuning.of(node_block=-1))
    gpu.fdx_set_tuning(gpu.Tuning.of(node_block=2))
    assert gpu.fdx_get_tuning().as_dict()["node_block"] == 2
    gpu.fdx_set_tuning(None)
    assert gpu.fdx_get_tuning().as_dict() == gpu.Tuning.DEFAULTS
