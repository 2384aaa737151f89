"""Pins of the oracle's ring-integrated cylindrical average (Eq. cyl-average)
against an independent integration: the average of the reciprocal-space
intensity (evaluated at arbitrary points) over the whole ring, by composite
Gauss-Legendre in a laboratory-frame azimuth that knows nothing of the
per-reflection windows, step rule or frames of the oracle's quadrature."""
import math
from dataclasses import replace

import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W


def _small(make):
    p = make()
    return replace(p, geom=replace(p.geom, n_x=30, n_y=24, pixel=p.geom.pixel * p.geom.n_x / 30),
                   br=replace(p.br, n_nodes=16))


def _ring_gl(orc, p, hkl, M, i, j, panels=2048, order=4):
    n = np.asarray(p.geom.fiber_axis, float)
    n /= np.linalg.norm(n)
    u = np.cross(n, np.asarray(p.geom.beam_axis, float))
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    S, R, Z = orc.pixel_S(p, i, j)
    _, As = orc.basis(p.cell)
    r0 = np.linalg.norm(hkl @ np.asarray(As).reshape(3, 3), axis=1)
    near = np.abs(r0 - math.hypot(R, Z)) < 0.05  # the others cannot reach this ring
    xg, wg = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(-math.pi, math.pi, panels + 1)
    mid, half = 0.5 * (edges[1:] + edges[:-1]), 0.5 * (edges[1:] - edges[:-1])
    psi = (mid[:, None] + half[:, None] * xg[None, :]).reshape(-1)
    wts = (half[:, None] * wg[None, :]).reshape(-1)
    pts = Z * n[None, :] + R * (np.cos(psi)[:, None] * u[None, :] + np.sin(psi)[:, None] * v[None, :])
    return float(np.sum(orc.point(p, hkl[near], M[near], pts) * wts) / (2 * math.pi))


@pytest.mark.parametrize("make", [W.small_gauss, lambda: W.tilted(W.small_gauss(), 20.0)])
def test_ring_matches_full_circle_quadrature(orc, make):
    """Gaussian lineshape (smooth integrand): the per-reflection midpoint rule
    over the window equals the full-circle integral to rounding."""
    p = _small(make)
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    for (i, j) in ((6, 16), (10, 5)):
        I, E = orc.ring(p, hkl, M, pix=[[i, j]])
        ref = _ring_gl(orc, p, hkl, M, i, j)
        assert ref > 0 and E[0] > 0
        assert I[0] == pytest.approx(ref, rel=1e-9)


def test_ring_hosemann_rule_converges(orc):
    """Hosemann lineshape (the support edge is a jump): the definition's rule
    is within 1e-3 of the refined rule and of the full-circle integral."""
    p = _small(W.small_helix)
    hkl = orc.reflections(p.cell, p.d_min)
    M = orc.intensities_M(p, hkl)
    i, j = 6, 16
    I1 = orc.ring(p, hkl, M, pix=[[i, j]])[0][0]
    I8 = orc.ring(p, hkl, M, pix=[[i, j]], refine=8)[0][0]
    ref = _ring_gl(orc, p, hkl, M, i, j, panels=8192)
    assert I1 == pytest.approx(I8, rel=1e-3)
    assert I8 == pytest.approx(ref, rel=3e-4)


def test_ring_mirror_symmetry(orc):
    """A pixel and its mirror about the meridian have the same ring."""
    p = _small(W.small_helix)
    hkl = orc.reflections(p.cell, p.d_min)
    nx = p.geom.n_x
    pix = np.array([[i, j] for j in (5, 16) for i in range(nx)])
    I, _ = orc.ring(p, hkl, orc.intensities_M(p, hkl), pix=pix)
    rows = I.reshape(2, nx)
    assert rows.max() > 0
    assert np.max(np.abs(rows - rows[:, ::-1])) <= 1e-12 * rows.max()
