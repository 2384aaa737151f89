"""Ring-integrated cylindrical average on the GPU (fdx_ring) against the FP64
oracle, full images of reduced detectors, every lineshape and a tilted fiber.
Gate: the pattern tolerances; in-support term counts within 1e-4 (a node at
the edge of the support is a floating-point decision)."""
from dataclasses import replace

import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import L2_REL, MAX_REL, api_precision, oracle_hkl, parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


def _small(make):
    p = make()
    return replace(p, geom=replace(p.geom, n_x=30, n_y=24, pixel=p.geom.pixel * p.geom.n_x / 30),
                   br=replace(p.br, n_nodes=16))


@pytest.mark.parametrize("make", [W.small_helix, W.small_gauss, W.small_tilted, W.small_sinc, W.small_lorentz])
def test_ring_matches_oracle(gpu, orc, make):
    import torch
    p = api_precision(_small(make))
    sim = gpu.Simulation(p)
    sim.structure_factors()
    img = sim.ring().cpu().numpy().reshape(-1)
    cnt = sim.ring_evals().cpu().numpy().reshape(-1)
    torch.cuda.synchronize()
    hkl = oracle_hkl(orc, p, sim.hkl_host)
    I, E = orc.ring(p, hkl, orc.intensities_M(p, hkl))
    assert I.max() > 0
    mr, l2 = parity(img, I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    assert abs(int(cnt.sum()) - int(E.sum())) <= 1e-4 * E.sum()


def test_ring_mirror_symmetry_gpu(gpu):
    import torch
    p = api_precision(_small(W.small_helix))
    sim = gpu.Simulation(p)
    sim.structure_factors()
    img = sim.ring().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(img - img[:, ::-1])) <= MAX_REL * img.max()


def test_ring_unsplit_large_detector(gpu, orc):
    """A detector of 1024 x 1024 pixels has enough 8 x 8 patches to fill the
    GPU with one warp each, so every reflection's azimuth points stay in one
    warp (the reduced detectors above deal them to several): sampled pixels
    against the oracle, and the in-support count of those pixels."""
    import torch
    p = W.small_helix()
    p = replace(p, geom=replace(p.geom, n_x=1024, n_y=1024, pixel=p.geom.pixel * p.geom.n_x / 1024),
                br=replace(p.br, n_nodes=8))
    p = api_precision(p)
    sim = gpu.Simulation(p)
    sim.structure_factors()
    img = sim.ring().cpu().numpy()
    cnt = sim.ring_evals().cpu().numpy()
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    pix = np.stack([rng.integers(0, 1024, 32), rng.integers(0, 1024, 32)], 1)
    hkl = oracle_hkl(orc, p, sim.hkl_host)
    I, E = orc.ring(p, hkl, orc.intensities_M(p, hkl), pix=pix)
    got = img[pix[:, 1], pix[:, 0]].astype(np.float64)
    assert I.max() > 0
    mr, l2 = parity(got, I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    n = int(cnt[pix[:, 1], pix[:, 0]].astype(np.int64).sum())
    assert abs(n - int(E.sum())) <= 1e-4 * E.sum()


def test_ring_edge_cases(gpu, orc):
    """Empty reflection list (zero image), 1 x 1 and ragged detectors."""
    import torch
    p = api_precision(_small(W.small_triclinic))
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    for nx, ny, n in ((30, 24, 0), (1, 1, len(hkl)), (17, 9, len(hkl)), (33, 5, len(hkl))):
        q = replace(p, geom=replace(p.geom, n_x=nx, n_y=ny, pixel=p.geom.pixel * 30 / nx))
        hk = torch.as_tensor(np.ascontiguousarray(hkl[:n], np.int32), device="cuda").reshape(-1, 3)
        Mt = torch.as_tensor(np.ascontiguousarray(M[:n], np.float32), device="cuda")
        prob = gpu.make_problem(q.cell, q.br, q.geom, hk, Mt)
        img = torch.full((ny, nx), float("nan"), dtype=torch.float32, device="cuda")
        gpu.fdx_ring(prob, img)
        torch.cuda.synchronize()
        img = img.cpu().numpy().reshape(-1)
        if n == 0:
            assert np.all(img == 0.0)
            continue
        I, _ = orc.ring(q, hkl[:n], M[:n].astype(np.float32).astype(np.float64))
        mr, l2 = parity(img, I)
        assert mr <= MAX_REL and l2 <= L2_REL, (nx, ny, mr, l2)


def test_ring_helix_central_region(gpu, orc):
    """The ring average as the benchmark runs it: the helix model's central
    128 x 128 pixels (0.1 mm), all 5,062 reflections, 64^2 nodes, so that
    each reflection's azimuth points are dealt to 128 warps per patch and
    summed by the reduce kernel; seeded pixels against the oracle (both sides
    fed the oracle's reflections and intensities), and their in-support
    counts."""
    import torch
    p = W.config1()
    p = api_precision(replace(p, geom=replace(p.geom, n_x=128, n_y=128)))
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl).astype(np.float32)
    hk = torch.as_tensor(np.ascontiguousarray(hkl, np.int32), device="cuda").reshape(-1, 3)
    Mt = torch.as_tensor(M, device="cuda")
    prob = gpu.make_problem(p.cell, p.br, p.geom, hk, Mt)
    img = torch.full((128, 128), float("nan"), dtype=torch.float32, device="cuda")
    cnt = torch.zeros((128, 128), dtype=torch.int32, device="cuda")
    gpu.fdx_ring(prob, img)
    gpu.fdx_ring_evals(prob, cnt)
    torch.cuda.synchronize()
    img, cnt = img.cpu().numpy(), cnt.cpu().numpy()
    rng = np.random.default_rng(11)
    pix = np.stack([rng.integers(0, 128, 12), rng.integers(0, 128, 12)], 1)
    I, E = orc.ring(p, hkl, M.astype(np.float64), pix=pix)
    got = img[pix[:, 1], pix[:, 0]].astype(np.float64)
    assert I.max() > 0
    mr, l2 = parity(got, I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    n = int(cnt[pix[:, 1], pix[:, 0]].astype(np.int64).sum())
    assert abs(n - int(E.sum())) <= 1e-4 * E.sum()
