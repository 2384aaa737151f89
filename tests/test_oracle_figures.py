"""The model of the paper's figures with |F| = 1 (Figs. GvL and equator) on
the oracle: the unit atom gives F = 1 exactly, and the reciprocal-space
intensity around a reflection follows the closed forms of the two
orientation distributions of Fig. GvL along the azimuth (Gaussian
exp(-D^2 / 2 sigma^2), Lorentzian 1 / (1 + D^2 / gamma^2), each smoothed a
little by the crystallite-size kernel)."""
import math

import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W


def test_unit_model_has_unit_structure_factors(orc):
    p = W.gvl("gauss", n_px=95)
    hkl = orc.reflections(p.cell, p.d_min)
    assert len(hkl) > 100
    F = orc.structure_factors(p.cell, p.atoms, hkl)
    assert np.all(F == 1.0)


def _azimuth_profile(orc, p, h, degs):
    """Mean intensity at angular distance D from the reflection's centre on
    its shell |S| = r0, over four directions and a 0.3 deg spread."""
    _, As = orc.basis(p.cell)
    D = np.asarray(h, float) @ np.asarray(As).reshape(3, 3)
    r0 = np.linalg.norm(D)
    s = D / r0
    n = np.asarray(p.geom.fiber_axis, float)
    e1 = np.cross(n, s)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(s, e1)
    out = []
    for deg in degs:
        pts = [r0 * (math.cos(math.radians(deg + j)) * s + math.sin(math.radians(deg + j)) * e)
               for e in (e1, e2, -e1, -e2) for j in np.linspace(-0.15, 0.15, 5)]
        out.append(np.mean(orc.point(p, np.array([h]), np.ones(1), np.array(pts))))
    return np.array(out) / out[0]


@pytest.mark.parametrize("h", [(3, 0, 0), (2, 2, 0)])
def test_gvl_azimuthal_tails(orc, h):
    g = _azimuth_profile(orc, W.gvl("gauss", n_px=95), h, (0.0, 4.5, 7.5))
    lz = _azimuth_profile(orc, W.gvl("lorentz", n_px=95), h, (0.0, 4.5, 7.5))
    ga = [math.exp(-0.5 * (d / 3.0) ** 2) for d in (4.5, 7.5)]
    la = [1.0 / (1.0 + (d / 3.0) ** 2) for d in (4.5, 7.5)]
    for got, ref in ((g[1:], ga), (lz[1:], la)):
        assert np.all(np.abs(np.asarray(got) / ref - 1.0) < 0.35), (got, ref)
    assert lz[2] > 2.0 * g[2]  # the Lorentzian's heavy tail


def test_pgm_writer(tmp_path):
    """The figure writer's log-scaled 8-bit view: header, size, orientation
    (last image row first) and the decade clamp."""
    from paper_2608_23245_b300 import figures
    img = np.array([[1e-6, 1e-2], [1.0, 0.0]])
    path = tmp_path / "x.pgm"
    figures.write_pgm(str(path), img, decades=4.0)
    raw = path.read_bytes()
    head = b"P5\n2 2\n255\n"
    assert raw.startswith(head)
    px = np.frombuffer(raw[len(head):], np.uint8).reshape(2, 2)
    assert px[0, 0] == 255 and px[0, 1] == 0          # image row 1 (1.0, 0.0) on top
    assert px[1, 0] == 0 and px[1, 1] == 128          # 1e-6 clamps to 1e-4; 1e-2 is half-way
