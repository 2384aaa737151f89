"""Scatter form on the GPU (fdx_scatter) against the FP64 oracle on the same
seeded samples.  Two floating-point decisions are integer-valued: the pixel
a hit falls in, and whether a node sits inside a sample's support (|t_i| <=
t_max).  Hits within 1e-4 pixel of a pixel edge, and samples with a node
within 1e-6 of the edge of the support (both found from the oracle's own
values), may go either way, so the pixels they touch are left out of the
element-wise comparison; every other pixel must match within the pattern
tolerances, and the totals must agree."""
import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import L2_REL, MAX_REL, api_precision, parity

pytestmark = pytest.mark.gpu

EDGE = 1e-4
SUPPORT_EDGE = 1e-6


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


def _edge_mask(p, samp):
    """Pixels on either side of a pixel edge that a hit lies within EDGE of,
    and pixels hit by samples with a node at the edge of their support."""
    nx, ny = p.geom.n_x, p.geom.n_y
    bad = np.zeros((ny, nx), bool)
    for b in (0, 1):
        x = samp[..., 3 + 2 * b].reshape(-1)
        y = samp[..., 4 + 2 * b].reshape(-1)
        amb = samp[..., 7].reshape(-1) < SUPPORT_EDGE
        ok = ~np.isnan(x)
        xa, ya = x[ok & amb], y[ok & amb]
        inside = (xa >= 0) & (xa < nx) & (ya >= 0) & (ya < ny)
        bad[np.floor(ya[inside]).astype(int), np.floor(xa[inside]).astype(int)] = True
        x, y = x[ok], y[ok]
        for dx in (-EDGE, 0.0, EDGE):
            for dy in (-EDGE, 0.0, EDGE):
                xi, yi = np.floor(x + dx).astype(int), np.floor(y + dy).astype(int)
                moved = (xi != np.floor(x)) | (yi != np.floor(y))
                for a, c in ((np.floor(x[moved]).astype(int), np.floor(y[moved]).astype(int)), (xi[moved], yi[moved])):
                    inside = (a >= 0) & (a < nx) & (c >= 0) & (c < ny)
                    bad[c[inside], a[inside]] = True
    return bad


@pytest.mark.parametrize("make", [W.small_helix, W.small_gauss, W.small_tilted, W.small_sinc, W.small_triclinic])
def test_scatter_matches_oracle(gpu, orc, make):
    import torch
    p = api_precision(make())
    xs = W.scatter_samples(4, 8, 8)
    sim = gpu.Simulation(p)
    sim.structure_factors()
    smp = torch.as_tensor(xs, device="cuda")
    img = sim.scatter(smp).cpu().numpy().astype(np.float64)
    E = int(sim.scatter_evals(smp).item())
    torch.cuda.synchronize()
    hkl = sim.hkl_host
    ref, E_ref, samp = orc.scatter(p, hkl, orc.intensities_M(p, hkl), xs.astype(np.float64), with_samples=True)
    assert ref.max() > 0
    bad = _edge_mask(p, samp)
    assert bad.mean() < 0.25, bad.mean()
    mr, l2 = parity(np.where(bad, 0.0, img).reshape(-1), np.where(bad, 0.0, ref).reshape(-1))
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    assert img.sum() == pytest.approx(ref.sum(), rel=1e-5)
    assert abs(E - E_ref) <= 1e-4 * E_ref, (E, E_ref)


@pytest.mark.parametrize("n", [1, 31, 77])
def test_scatter_ragged_sample_counts(gpu, orc, n):
    """Sample counts that leave the last warp of samples partly empty."""
    import torch
    p = api_precision(W.small_helix())
    xs = W.scatter_samples(4, 8, 8)[:n]
    sim = gpu.Simulation(p)
    sim.structure_factors()
    smp = torch.as_tensor(np.ascontiguousarray(xs), device="cuda")
    img = sim.scatter(smp).cpu().numpy().astype(np.float64)
    E = int(sim.scatter_evals(smp).item())
    torch.cuda.synchronize()
    hkl = sim.hkl_host
    ref, E_ref, samp = orc.scatter(p, hkl, orc.intensities_M(p, hkl), xs.astype(np.float64), with_samples=True)
    assert ref.max() > 0
    bad = _edge_mask(p, samp)
    mr, l2 = parity(np.where(bad, 0.0, img).reshape(-1), np.where(bad, 0.0, ref).reshape(-1))
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    assert abs(E - E_ref) <= 1e-4 * E_ref + 2, (E, E_ref)


def test_scatter_mirror_symmetry_gpu(gpu):
    """The two Ewald solutions are mirror images: the GPU image is symmetric
    about the meridian except where a hit sits at a pixel edge."""
    import torch
    p = api_precision(W.small_helix())
    sim = gpu.Simulation(p)
    sim.structure_factors()
    img = sim.scatter(torch.as_tensor(W.scatter_samples(4, 8, 8), device="cuda")).cpu().numpy().astype(np.float64)
    d = np.abs(img - img[:, ::-1])
    assert np.median(d) <= 1e-6 * img.max()
    assert np.sum(d > 1e-5 * img.max()) <= 0.02 * img.size


def test_scatter_rejects_bad_samples(gpu):
    import torch
    p = api_precision(W.small_helix())
    sim = gpu.Simulation(p)
    out = torch.empty_like(sim.image)
    xs = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.FdxError):
        gpu.fdx_scatter(sim.prob, xs, out, workspace=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
