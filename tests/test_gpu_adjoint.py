"""GPU refinement path against the FP64 oracle: the loss, the hand-written
adjoint (dL/dM, coordinates, B, sizes, g, sigma, gamma) for a common upstream
gradient, the end-to-end refinement gradient of the perturbed helix (config 3
recipe) on a pixel subset, and the autograd wrapper.  Gate: relative error
<= 1e-4 against the oracle adjoint (which is itself pinned to FP64 central
differences in test_oracle_pattern.py)."""
import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import api_precision, oracle_hkl

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


def _close(got, ref, tol=ADJ_TOL, what=""):
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    scale = np.max(np.abs(ref))
    assert scale > 0, what
    err = np.max(np.abs(got - ref)) / scale
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= tol and l2 <= tol, (what, err, l2)


def _oracle_grads(orc, p, hkl, gI, pix=None):
    F = orc.structure_factors(p.cell, p.atoms, hkl)
    _, P, DW = orc.refl_scalars(p, hkl)
    M = np.abs(F) ** 2 * P * DW
    G, dbeta, dsig, dgam = orc.pattern_adjoint(p, hkl, M, gI, pix)
    dL, dg = orc.chain_globals(p, hkl, np.abs(F) ** 2, G, dbeta)
    dfrac, dB = orc.sf_adjoint(p.cell, p.atoms, hkl, F, G * P * DW)
    return {"dM": G, "dfrac": dfrac, "dB": dB, "dL": dL, "dg": dg, "dsigma": dsig, "dgamma": dgam}


def _gpu_grads(gpu, p, gI):
    import torch
    sim = gpu.Simulation(p)
    sim.forward()
    n, na = sim.hkl.shape[0], p.atoms.n
    dfrac = torch.empty((na, 3), dtype=torch.float64, device="cuda")
    dB = torch.empty((na,), dtype=torch.float64, device="cuda")
    dglob = torch.empty(8, dtype=torch.float64, device="cuda")
    dM = torch.empty((n,), dtype=torch.float32, device="cuda")
    gIt = torch.as_tensor(np.ascontiguousarray(gI, np.float32).reshape(p.geom.n_y, p.geom.n_x), device="cuda")
    gpu.fdx_pattern_backward(sim.prob, sim.atoms, sim.F, gIt, dfrac, dB, dglob, dM)
    torch.cuda.synchronize()
    g = dglob.cpu().numpy()
    return sim, {"dM": dM.cpu().numpy(), "dfrac": dfrac.cpu().numpy(), "dB": dB.cpu().numpy(), "dL": g[0:3],
                 "dg": g[3:6], "dsigma": g[6], "dgamma": g[7]}


def test_loss_kernel(gpu):
    import torch
    rng = np.random.default_rng(3)
    I = rng.uniform(0, 3, 10007).astype(np.float32)
    It = rng.uniform(0, 3, 10007).astype(np.float32)
    m = (rng.uniform(size=10007) < 0.7).astype(np.float32)
    gI = torch.empty(10007, dtype=torch.float32, device="cuda")
    loss, _ = gpu.fdx_loss(torch.as_tensor(I, device="cuda"), torch.as_tensor(It, device="cuda"),
                           torch.as_tensor(m, device="cuda"), dL_dI=gI)
    torch.cuda.synchronize()
    w = m.astype(np.float64) / (It.astype(np.float64) + 1)
    d = I.astype(np.float64) - It
    assert loss.item() == pytest.approx(np.sum(w * d * d), rel=1e-12)
    assert np.allclose(gI.cpu().numpy(), 2 * w * d, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("make", [W.small_helix, W.small_lorentz, W.small_triclinic, W.small_tilted, W.small_sinc,
                                  W.small_gauss])
def test_backward_matches_oracle_adjoint(gpu, orc, make):
    """Common seeded upstream gradient dL/dI into both adjoints."""
    p = api_precision(make())
    rng = np.random.default_rng(17)
    gI = rng.uniform(-1.0, 1.0, p.geom.n_x * p.geom.n_y).astype(np.float32)
    sim, g = _gpu_grads(gpu, p, gI)
    o = _oracle_grads(orc, p, oracle_hkl(orc, p, sim.hkl_host), gI.astype(np.float64))
    _close(g["dM"], o["dM"], what="dM")
    _close(g["dfrac"], o["dfrac"], what="dfrac")
    _close(g["dB"], o["dB"], what="dB")
    glob_g = np.concatenate([g["dL"], g["dg"], [g["dsigma"], g["dgamma"]]])
    glob_o = np.concatenate([o["dL"], o["dg"], [o["dsigma"], o["dgamma"]]])
    for k, name in enumerate(["dL_a", "dL_b", "dL_c", "dg_a", "dg_b", "dg_c", "dsigma", "dgamma"]):
        if glob_o[k] == 0.0:
            assert abs(glob_g[k]) <= 1e-6 * np.max(np.abs(glob_o)), name
        else:
            assert glob_g[k] == pytest.approx(glob_o[k], rel=ADJ_TOL), name


def test_backward_deterministic(gpu):
    p = api_precision(W.small_helix())
    gI = np.random.default_rng(5).uniform(-1, 1, p.geom.n_x * p.geom.n_y).astype(np.float32)
    _, a = _gpu_grads(gpu, p, gI)
    _, b = _gpu_grads(gpu, p, gI)
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_refinement_gradient_helix_subset(gpu, orc):
    """Config-3 recipe at full size (2,000 atoms, 5,062 reflections, 1024^2
    detector): loss over a seeded 48-pixel subset of the central region, each
    side with its own forward of model and target; gradients w.r.t. all
    coordinates, B, sizes, g, sigma and gamma."""
    import torch
    from paper_2608_23245_b300.autograd import RefineModel, fiber_pattern, refinement_loss
    model, target = W.config3()
    model, target = api_precision(model), api_precision(target)
    rng = np.random.default_rng(31)
    n = model.geom.n_x
    ii = rng.integers(3 * n // 8, 5 * n // 8, 48)
    jj = rng.integers(3 * n // 8, 5 * n // 8, 48)
    mask = np.zeros((n, n), np.float32)
    mask[jj, ii] = 1.0
    pix = np.stack([ii, jj], 1).astype(np.int32)
    # GPU
    tsim = gpu.Simulation(target)
    It_g = tsim.forward().clone()
    rm = RefineModel(model)
    frac, B, L, g, sig, gam = rm.initial()
    for t in (frac, B, L, g, sig, gam):
        t.requires_grad_(True)
    img = fiber_pattern(frac, B, L, g, sig, gam, rm)
    loss = refinement_loss(img, It_g, torch.as_tensor(mask, device="cuda"))
    loss.backward()
    torch.cuda.synchronize()
    # oracle
    hkl = oracle_hkl(orc, model, rm.hkl_host)
    Mt = orc.intensities_M(target, hkl)
    It_o, _ = orc.pattern(target, hkl, Mt, pix)
    loss_o, go, _ = orc.full_gradient(model, hkl, It_o, pix)
    assert loss.item() == pytest.approx(loss_o, rel=1e-5)
    _close(frac.grad.cpu().numpy(), go["frac"], what="frac")
    _close(B.grad.cpu().numpy(), go["B"], what="B")
    _close(L.grad.numpy(), go["L"], what="L")
    _close(g.grad.numpy()[:2], go["g"][:2], what="g")
    assert sig.grad.item() == pytest.approx(go["sigma"], rel=ADJ_TOL)
    assert gam.grad.item() == pytest.approx(go["gamma"], rel=ADJ_TOL)


def test_batch_refine_rejects_other_lineshapes(gpu):
    """The batched refinement runs the Hosemann adjoint only; a model with the
    sinc lineshape is refused on the host (the single-model backward takes
    every lineshape)."""
    import torch
    p = api_precision(W.small_sinc())
    sim = gpu.Simulation(p)
    It = torch.zeros((p.geom.n_y, p.geom.n_x), dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.FdxError):
        gpu.BatchStep([sim.prob], [sim.atoms], targets=[It])()
