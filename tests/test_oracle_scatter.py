"""Pins of the oracle's scatter form (the paper's own sampling + Ewald
projection pipeline), each against something other than the oracle's own
formulae: the closed-form volume integral of the reflection profile, the
mirror symmetry of the two Ewald solutions, and the independent pixel ->
scattering-vector map of the detector."""
import math
from dataclasses import replace

import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W


def _broad_gauss_problem():
    """small_helix with a Gaussian orientation spread whose node patch reaches
    6 sigma (edge weight e^-18), so that the sampled box holds the whole
    profile; no paracrystal term."""
    p = W.small_helix()
    sig = math.radians(3.0)
    br = replace(p.br, sigma=sig, gamma=0.0, T=math.tan(6 * sig), n_nodes=48, L=(60.0, 60.0, 80.0),
                 g=(0.0, 0.0, 0.0))
    return replace(p, br=br)


def test_scatter_profile_integral(orc):
    """Sum over samples of dV I / (M r0^2) is a quadrature of the volume
    integral of sum_k w_k prod_i K_i(a_i . (S - s_k)) over S, which is
    sum_k w_k / V_cell (each Hosemann factor integrates to one over its
    period and d^3 t = V_cell d^3 S).  Stratified 16 x 64 x 64 samples reach it
    within the sampling error (~1e-3)."""
    p = _broad_gauss_problem()
    hkl = orc.reflections(p.cell, p.d_min)
    A, As = orc.basis(p.cell)
    Vc = abs(np.linalg.det(np.asarray(A).reshape(3, 3)))
    w = orc.nodes(p)[2]
    r0s = np.linalg.norm(hkl @ np.asarray(As).reshape(3, 3), axis=1)
    xs = W.scatter_samples(16, 64, 64)
    for idx in (int(np.argmax(r0s)), int(np.argsort(r0s)[len(r0s) // 2])):
        _, _, samp = orc.scatter(p, hkl[idx:idx + 1], np.ones(1), xs, with_samples=True)
        tot = np.sum(samp[0, :, 0] * samp[0, :, 1]) / r0s[idx] ** 2
        assert tot == pytest.approx(np.sum(w) / Vc, rel=2e-3), hkl[idx]


@pytest.mark.parametrize("make", [W.small_helix, W.small_tilted])
def test_scatter_mirror_and_branches(orc, make):
    """The two solutions of Eq. solutions are mirror images about the plane of
    beam and fiber axis: their hits have x0 + x1 = n_x and y0 = y1, and the
    accumulated image is mirror symmetric (u -> -u)."""
    p = make()
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    img, E, samp = orc.scatter(p, hkl, M, W.scatter_samples(4, 8, 8), with_samples=True)
    assert E > 0 and img.max() > 0
    both = ~np.isnan(samp[..., 3]) & ~np.isnan(samp[..., 5])
    assert both.sum() > 0.5 * both.size
    assert np.max(np.abs(samp[..., 3][both] + samp[..., 5][both] - p.geom.n_x)) < 1e-9
    assert np.max(np.abs(samp[..., 4][both] - samp[..., 6][both])) < 1e-9
    assert np.max(np.abs(img - img[:, ::-1])) <= 1e-12 * img.max()


def test_scatter_hits_match_pixel_geometry(orc):
    """A hit in pixel (i, j) must have the (R, Z) of that pixel's scattering
    vector (the detector map of Eq. laue) to within the pixel's extent in
    reciprocal space: the closed-form rotation lands where the pixel map
    says it should."""
    p = W.small_tilted()
    hkl = orc.reflections(p.cell, p.d_min)[::7]
    xs = W.scatter_samples(2, 4, 4)
    _, _, samp = orc.scatter(p, hkl, np.ones(len(hkl)), xs, with_samples=True)
    ext = 1.5 * p.geom.pixel / (p.geom.wavelength * p.geom.distance)
    checked = 0
    for r in range(len(hkl)):
        for m in range(len(xs)):
            row = samp[r, m]
            for b in (0, 1):
                xp, yp = row[3 + 2 * b], row[4 + 2 * b]
                if np.isnan(xp) or not (0 <= xp < p.geom.n_x and 0 <= yp < p.geom.n_y):
                    continue
                # the sample's ring radius R from its Lorentz factor L = delta/(R + delta)
                R_s = p.geom.delta_L / row[2] - p.geom.delta_L
                _, R_px, _ = orc.pixel_S(p, int(math.floor(xp)), int(math.floor(yp)))
                assert abs(R_px - R_s) <= ext * (1 + 1e-6), (r, m, R_px, R_s)
                checked += 1
    assert checked > 100


def _lorentz_problem():
    """small_helix with a Lorentzian orientation spread (gamma = 3 deg, node
    patch T = tan(3 gamma)) and no paracrystal term."""
    p = W.small_helix()
    gam = math.radians(3.0)
    br = replace(p.br, sigma=0.0, gamma=gam, T=W.patch_extent(0.0, gam), n_nodes=48, L=(60.0, 60.0, 80.0),
                 g=(0.0, 0.0, 0.0))
    return replace(p, br=br)


def test_scatter_cauchy_sampling_covers_the_tails(orc):
    """Heavy-tailed sampling (Sect. "Angular peak shapes": Cauchy sampling of
    the shell when a Lorentzian is present).  With a Lorentzian spread the
    profile reaches past the node patch by the kernel's support: samples
    confined to the patch ([-1, 1] in x_1, x_2) miss that part (several %),
    while Cauchy samples of half-width tan(gamma)/T over an extended range
    recover the closed-form volume integral sum_k w_k / V_cell (each lattice
    factor integrates to one per period) to 1e-3."""
    p = _lorentz_problem()
    hkl = orc.reflections(p.cell, p.d_min)
    A, As = orc.basis(p.cell)
    As = np.asarray(As).reshape(3, 3)
    Vc = abs(np.linalg.det(np.asarray(A).reshape(3, 3)))
    ref = np.sum(orc.nodes(p)[2]) / Vc
    r0s = np.linalg.norm(hkl @ As, axis=1)
    idx = int(np.argsort(r0s)[len(r0s) // 2])
    r0 = r0s[idx]
    beta, _, _ = orc.refl_scalars(p, hkl[idx:idx + 1])
    tm = [orc.support(p.br.lineshape, beta[0, i], p.br.K_z) for i in range(3)]
    rho = max(np.linalg.norm(tm[0] * As[0] + sb * tm[1] * As[1] + sc * tm[2] * As[2])
              for sb in (1, -1) for sc in (1, -1))
    extent = 1.0 + 1.5 * rho / (r0 * p.br.T)
    xs_c = W.scatter_samples_cauchy(16, 64, 64, math.tan(p.br.gamma) / p.br.T, extent)
    assert np.abs(xs_c[:, 1:3]).max() > 1.0
    tots = []
    for xs in (W.scatter_samples(16, 64, 64), xs_c):
        _, _, samp = orc.scatter(p, hkl[idx:idx + 1], np.ones(1), xs, with_samples=True)
        tots.append(np.sum(samp[0, :, 0] * samp[0, :, 1]) / r0 ** 2)
    assert tots[0] < (1.0 - 0.03) * ref, tots[0] / ref
    assert tots[1] == pytest.approx(ref, rel=1e-3), tots[1] / ref


@pytest.mark.parametrize("spot", [3, 5])
def test_scatter_spot_is_a_box_filter_of_the_single_pixel_image(orc, spot):
    """The detector spot (the paper's simulate() spot size) spreads each hit
    evenly over the spot x spot block around its pixel.  So away from the
    detector's edges, the spot image is exactly the one-pixel image filtered
    by a spot x spot box of weight 1/spot^2."""
    p = W.small_helix()
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    xs = W.scatter_samples(2, 8, 8)
    img1, _ = orc.scatter(p, hkl, M, xs)
    imgs, _ = orc.scatter(p, hkl, M, xs, spot=spot)
    h = (spot - 1) // 2
    ny, nx = img1.shape
    box = np.zeros((ny - 2 * h, nx - 2 * h))
    for dj in range(-h, h + 1):
        for di in range(-h, h + 1):
            box += img1[h + dj:ny - h + dj, h + di:nx - h + di]
    box /= spot * spot
    assert imgs.max() > 0
    assert np.max(np.abs(imgs[h:ny - h, h:nx - h] - box)) <= 1e-12 * imgs.max()
    with pytest.raises(ValueError):
        orc.scatter(p, hkl, M, xs, spot=2)
