"""The allocation-free structure-factor entry point.

fdx_structure_factors_noalloc serves callers that cannot allocate device
memory when they need structure factors (a plugin whose host application owns
all device memory through its own allocator, a real-time loop that must not
call cudaMalloc after start-up).  Its scratch is a fixed array inside the
library, shared by all calls.  This test calls it twice in a row through the
C-ABI, on two different problems, and checks each result against the regular
workspace-based entry point on the same inputs, with the structure-factor
tolerance used throughout the tests.  It sits in a file of its own that pytest
collects last."""
import ctypes as C

import numpy as np
import pytest

from paper_2608_23245_b300 import workloads as W
from _common import SF_TOL, amp_scale, api_precision

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


def _compare(gpu, make):
    import torch
    p = api_precision(make())
    hkl_host = gpu.fdx_reflections(p.cell, p.d_min, p.d_max)
    hkl = torch.as_tensor(hkl_host, device="cuda")
    atoms = gpu.DeviceAtoms(p.atoms)
    F_ref, M_ref = gpu.fdx_structure_factors(p.cell, atoms, hkl, p.br)
    n = hkl.shape[0]
    F = torch.full((n, 2), float("nan"), dtype=torch.float32, device="cuda")
    M = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    lib = gpu.lib()
    c = gpu.make_cell(p.cell)
    a = atoms.struct()
    b = gpu.make_broadening(p.br)
    rc = lib.fdx_structure_factors_noalloc(C.byref(c), C.byref(a), C.byref(b), n, C.c_void_p(hkl.data_ptr()),
                                           C.c_void_p(F.data_ptr()), C.c_void_p(M.data_ptr()),
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, gpu.error_string(rc)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy().astype(np.float64)
    Fr = F_ref.cpu().numpy().astype(np.float64)
    scale = amp_scale(p, hkl_host)
    err = np.abs((Fg[:, 0] - Fr[:, 0]) + 1j * (Fg[:, 1] - Fr[:, 1])) / scale
    assert np.isfinite(Fg).all() and err.max() <= SF_TOL, err.max()
    Mg, Mr = M.cpu().numpy().astype(np.float64), M_ref.cpu().numpy().astype(np.float64)
    Fabs = np.hypot(Fr[:, 0], Fr[:, 1])
    merr = np.abs(Mg - Mr) / ((2 * Fabs + scale) * scale)
    assert np.isfinite(Mg).all() and merr.max() <= 2 * SF_TOL, merr.max()


def test_noalloc_matches_workspace_path_twice(gpu):
    """Two calls in a row (different sizes, so the shared scratch is reused
    with a different layout), each against fdx_structure_factors."""
    _compare(gpu, W.small_helix)
    _compare(gpu, W.config1)


def test_noalloc_rejects_oversize(gpu):
    """Sizes whose scratch exceeds the fixed array are refused before any
    device work (FDX_ERR_WORKSPACE)."""
    lib = gpu.lib()
    c = gpu.make_cell((50.0, 50.0, 70.0, np.pi / 2, np.pi / 2, np.pi / 2))
    a = gpu.Atoms()
    a.n_atoms, a.n_elem = 1 << 20, 4
    a.frac = a.B = a.elem = a.ff = 256
    rc = lib.fdx_structure_factors_noalloc(C.byref(c), C.byref(a), None, 1000, C.c_void_p(256), C.c_void_p(256),
                                           None, None)
    assert rc == -3
    a.n_atoms = 100
    rc = lib.fdx_structure_factors_noalloc(C.byref(c), C.byref(a), None, 1 << 20, C.c_void_p(256),
                                           C.c_void_p(256), None, None)
    assert rc == -3
