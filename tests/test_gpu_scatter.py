"""Scatter form on the GPU (fdx_scatter) against the FP64 oracle on the same
seeded samples.  Two floating-point decisions are integer-valued: the pixel
a hit falls in, and whether a node sits inside a sample's support (|t_i| <=
t_max).  Hits within 1e-4 pixel of a pixel edge, and samples with a node
within 1e-6 of the edge of the support (both found from the oracle's own
values), may go either way, so the pixels they touch are left out of the
element-wise comparison; every other pixel must match within the pattern
tolerances, and the totals must agree."""
import math

import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import L2_REL, MAX_REL, api_precision, oracle_hkl, parity

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


def _dilate(mask, h):
    """Pixels within h of a marked pixel (a hit's spot covers (2h+1)^2 pixels)."""
    if h == 0:
        return mask
    out = mask.copy()
    ny, nx = mask.shape
    for dj in range(-h, h + 1):
        for di in range(-h, h + 1):
            out[max(dj, 0):ny + min(dj, 0), max(di, 0):nx + min(di, 0)] |= \
                mask[max(-dj, 0):ny + min(-dj, 0), max(-di, 0):nx + min(-di, 0)]
    return out


def _ambiguous_value(samp):
    """Summed magnitude dV L I of the hits whose pixel or whose node set is
    decided within rounding (hits within EDGE of a pixel edge, samples with a
    node within SUPPORT_EDGE of the support's edge): the most the excluded
    pixels can differ by, counted on both pixels a hit can move between."""
    v = np.abs(samp[..., 0] * samp[..., 1] * samp[..., 2])
    amb_s = samp[..., 7] < SUPPORT_EDGE
    tot = 0.0
    for b in (0, 1):
        x, y = samp[..., 3 + 2 * b], samp[..., 4 + 2 * b]
        ok = ~np.isnan(x)
        fx, fy = np.where(ok, x - np.floor(x), 0.5), np.where(ok, y - np.floor(y), 0.5)
        near = ok & ((np.minimum(fx, 1 - fx) < EDGE) | (np.minimum(fy, 1 - fy) < EDGE))
        tot += np.sum(v[(near | (amb_s & ok))])
    return 2.0 * tot


def _edge_mask(p, samp, spot=1):
    """Pixels on either side of a pixel edge that a hit lies within EDGE of,
    and pixels hit by samples with a node at the edge of their support; with
    a detector spot, every pixel of those hits' spots."""
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
    return _dilate(bad, (spot - 1) // 2)


def _cauchy_samples(p):
    """Heavy-tailed samples (half-width tan(gamma)/T, reaching 1.6 T)."""
    return W.scatter_samples_cauchy(4, 8, 8, math.tan(max(p.br.gamma, math.radians(1.0))) / p.br.T, 1.6)


CASES = [(W.small_helix, "stratified", 1), (W.small_gauss, "stratified", 1), (W.small_tilted, "stratified", 1),
         (W.small_sinc, "stratified", 1), (W.small_triclinic, "stratified", 1), (W.small_lorentz, "cauchy", 1),
         (W.small_helix, "cauchy", 1), (W.small_helix, "stratified", 3), (W.small_tilted, "cauchy", 3)]


@pytest.mark.parametrize("make,kind,spot", CASES)
def test_scatter_matches_oracle(gpu, orc, make, kind, spot):
    """Element-wise parity outside the excluded pixels; the excluded pixels
    differ in all by no more than the ambiguous hits carry; equal totals."""
    import torch
    p = api_precision(make())
    xs = W.scatter_samples(4, 8, 8) if kind == "stratified" else _cauchy_samples(p)
    sim = gpu.Simulation(p)
    sim.structure_factors()
    smp = torch.as_tensor(xs, device="cuda")
    img = sim.scatter(smp, spot_size=spot).cpu().numpy().astype(np.float64)
    E = int(sim.scatter_evals(smp).item())
    torch.cuda.synchronize()
    hkl = oracle_hkl(orc, p, sim.hkl_host)
    ref, E_ref, samp = orc.scatter(p, hkl, orc.intensities_M(p, hkl), xs.astype(np.float64), with_samples=True,
                                   spot=spot)
    assert ref.max() > 0
    bad = _edge_mask(p, samp, spot)
    assert bad.mean() < 0.5, bad.mean()
    mr, l2 = parity(np.where(bad, 0.0, img).reshape(-1), np.where(bad, 0.0, ref).reshape(-1))
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    diff_bad = float(np.sum(np.abs(img - ref)[bad]))
    assert diff_bad <= _ambiguous_value(samp) + MAX_REL * ref.max() * bad.sum(), (diff_bad, _ambiguous_value(samp))
    assert img.sum() == pytest.approx(ref.sum(), rel=1e-5)
    assert abs(E - E_ref) <= 1e-4 * E_ref, (E, E_ref)


@pytest.mark.parametrize("n", [1, 31, 50, 77, 100])
def test_scatter_ragged_sample_counts(gpu, orc, n):
    """Sample counts that leave the last warp of samples partly empty (a warp
    takes 64, two per lane: 31 leaves every lane's second sample out, 50 and
    100 part of them)."""
    import torch
    p = api_precision(W.small_helix())
    xs = W.scatter_samples(4, 8, 8)[:n]
    sim = gpu.Simulation(p)
    sim.structure_factors()
    smp = torch.as_tensor(np.ascontiguousarray(xs), device="cuda")
    img = sim.scatter(smp).cpu().numpy().astype(np.float64)
    E = int(sim.scatter_evals(smp).item())
    torch.cuda.synchronize()
    hkl = oracle_hkl(orc, p, sim.hkl_host)
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


@pytest.mark.parametrize("spot", [3, 5])
def test_scatter_spot_box_filter_gpu(gpu, spot):
    """On the GPU alone: away from the detector's edges the spot image is the
    one-pixel image filtered by a spot x spot box of weight 1/spot^2 (each hit
    is spread evenly over the block around its pixel); heavy-tailed samples
    on a tilted fiber."""
    import torch
    p = api_precision(W.small_tilted())
    sim = gpu.Simulation(p)
    sim.structure_factors()
    smp = torch.as_tensor(_cauchy_samples(p), device="cuda")
    img1 = sim.scatter(smp).cpu().numpy().astype(np.float64)
    imgs = sim.scatter(smp, spot_size=spot).cpu().numpy().astype(np.float64)
    h = (spot - 1) // 2
    ny, nx = img1.shape
    box = np.zeros((ny - 2 * h, nx - 2 * h))
    for dj in range(-h, h + 1):
        for di in range(-h, h + 1):
            box += img1[h + dj:ny - h + dj, h + di:nx - h + di]
    box /= spot * spot
    assert imgs.max() > 0
    assert np.max(np.abs(imgs[h:ny - h, h:nx - h] - box)) <= 1e-6 * imgs.max()


def test_scatter_helix_full_geometry(gpu, orc):
    """The scatter form in the benchmark's geometry: the helix model's 1024 x
    1024 detector, 64^2 nodes and 16^3 stratified samples per reflection
    (bricks, two samples per lane), on 12 seeded reflections of the oracle's
    list with the oracle's intensities (the oracle's cost grows with samples
    x nodes per reflection): element-wise parity outside the excluded pixels,
    the excluded pixels bounded by their ambiguous hits, equal totals and
    term counts."""
    import torch
    p = api_precision(W.config1())
    hkl_all = orc.reflections(p.cell, p.d_min)
    pick = np.sort(np.random.default_rng(13).choice(len(hkl_all), 12, replace=False))
    hkl = np.ascontiguousarray(hkl_all[pick], np.int32)
    M = orc.intensities_M(p, hkl).astype(np.float32)
    hk = torch.as_tensor(hkl, device="cuda").reshape(-1, 3)
    Mt = torch.as_tensor(M, device="cuda")
    prob = gpu.make_problem(p.cell, p.br, p.geom, hk, Mt)
    xs = W.scatter_samples(16, 16, 16)
    smp = torch.as_tensor(xs, device="cuda")
    img = torch.zeros((p.geom.n_y, p.geom.n_x), dtype=torch.float32, device="cuda")
    gpu.fdx_scatter(prob, smp, img)
    count = torch.zeros((), dtype=torch.int64, device="cuda")
    gpu.fdx_scatter_evals(prob, smp, count)
    torch.cuda.synchronize()
    img = img.cpu().numpy().astype(np.float64)
    E = int(count.item())
    ref, E_ref, samp = orc.scatter(p, hkl, M.astype(np.float64), xs.astype(np.float64), with_samples=True)
    assert ref.max() > 0
    bad = _edge_mask(p, samp)
    mr, l2 = parity(np.where(bad, 0.0, img).reshape(-1), np.where(bad, 0.0, ref).reshape(-1))
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)
    diff_bad = float(np.sum(np.abs(img - ref)[bad]))
    assert diff_bad <= _ambiguous_value(samp) + MAX_REL * ref.max() * bad.sum(), (diff_bad, _ambiguous_value(samp))
    assert img.sum() == pytest.approx(ref.sum(), rel=1e-5)
    assert abs(E - E_ref) <= 1e-4 * E_ref, (E, E_ref)
