"""The paper's model figures with |F| = 1 through the GPU path
(``figures.py``): full reduced images against the oracle, and the features
the figures show: the equatorial peaks stay in place as disorder grows, the
high orders lose height with the paracrystal g, and the axis Debye-Waller B
damps the high orders more than the low ones."""
import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import L2_REL, MAX_REL, api_precision, parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, figures
    _build.build()
    return figures


@pytest.mark.parametrize("p", [W.gvl("gauss", n_px=95, n_nodes=32), W.gvl("lorentz", n_px=95, n_nodes=32),
                               W.equator(0.0, 0.0, n_x=255, n_y=9, n_nodes=32),
                               W.equator(0.03, 10.0, n_x=255, n_y=9, n_nodes=32)], ids=lambda p: p.name)
def test_figure_images_match_oracle(gpu, orc, p):
    p = api_precision(p)
    img = gpu.simulate(p)
    hkl = orc.reflections(p.cell, p.d_min)
    I, _ = orc.pattern(p, hkl, orc.intensities_M(p, hkl))
    assert I.max() > 0
    mr, l2 = parity(img.reshape(-1), I)
    assert mr <= MAX_REL and l2 <= L2_REL, (mr, l2)


def _peaks(row, n=6):
    """The first n local maxima of the half-profile beyond the beam centre."""
    half = row[len(row) // 2:]
    idx = [i for i in range(1, len(half) - 1) if half[i] > half[i - 1] and half[i] >= half[i + 1]
           and half[i] > 1e-3 * half.max()]
    return np.asarray(idx[:n])


def test_equator_profiles(gpu):
    params = ((0.0, 0.0), (0.01, 0.0), (0.03, 0.0), (0.05, 0.0), (0.03, 10.0))
    _, prof = gpu.equator_profiles(params, n_x=511, n_y=15, n_nodes=32)
    pk = {k: _peaks(v) for k, v in prof.items()}
    ref = pk[(0.0, 0.0)]
    assert len(ref) == 6
    for k in params:
        assert np.array_equal(pk[k], ref), (k, pk[k], ref)
    half = {k: v[len(v) // 2:] for k, v in prof.items()}
    # high order (6th peak) against the 2nd: falls as g grows
    ratio = [half[(g, 0.0)][ref[5]] / half[(g, 0.0)][ref[1]] for g in (0.0, 0.01, 0.03, 0.05)]
    assert all(a > b for a, b in zip(ratio, ratio[1:])), ratio
    # the axis B damps every peak, the higher orders more
    damp = half[(0.03, 10.0)][ref] / half[(0.03, 0.0)][ref]
    assert np.all(damp < 1.0) and np.all(np.diff(damp) < 0), damp
