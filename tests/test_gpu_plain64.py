"""The plain FP64 GPU form of the method (the refinement-throughput metric's
comparison path) against the FP64 oracle: same definition, both in FP64, so
they agree to rounding (relative 1e-9)."""
import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import api_precision, oracle_hkl

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


def _rel(got, ref):
    got, ref = np.asarray(got, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("make", [W.small_helix, W.small_lorentz, W.small_triclinic])
def test_plain64_forward_and_gradient(gpu, orc, make):
    import torch
    p = api_precision(make())
    sim = gpu.Simulation(p)
    n = (p.geom.n_y, p.geom.n_x)
    rng = np.random.default_rng(9)
    It = rng.uniform(0, 2e-4, n)
    img = torch.empty(n, dtype=torch.float64, device="cuda")
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    dfrac = torch.empty((p.atoms.n, 3), dtype=torch.float64, device="cuda")
    dB = torch.empty((p.atoms.n,), dtype=torch.float64, device="cuda")
    dglob = torch.empty(8, dtype=torch.float64, device="cuda")
    gpu.fdx_plain64_refine(sim.prob, sim.atoms, img, torch.as_tensor(It, device="cuda"), None, loss, dfrac, dB, dglob)
    torch.cuda.synchronize()
    hkl = oracle_hkl(orc, p, sim.hkl_host)
    Mo = orc.intensities_M(p, hkl)
    I, _ = orc.pattern(p, hkl, Mo)
    assert _rel(img.cpu().numpy(), I) <= TOL64
    loss_o, go, _ = orc.full_gradient(p, hkl, It.reshape(-1))
    assert loss.item() == pytest.approx(loss_o, rel=TOL64)
    assert _rel(dfrac.cpu().numpy(), go["frac"]) <= 1e-8
    assert _rel(dB.cpu().numpy(), go["B"]) <= 1e-8
    g = dglob.cpu().numpy()
    ref = np.concatenate([go["L"], go["g"], [go["sigma"], go["gamma"]]])
    for k in range(8):
        if ref[k] == 0.0:
            assert abs(g[k]) <= 1e-12 * np.max(np.abs(ref))
        else:
            assert g[k] == pytest.approx(ref[k], rel=1e-8)
