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


def _compare(gpu, make, n_refl=None):
    import torch
    p = api_precision(make())
    hkl_host = gpu.fdx_reflections(p.cell, p.d_min, p.d_max)
    if n_refl is not None:
        hkl_host = np.ascontiguousarray(hkl_host[:n_refl])
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


def _two_pass_tight():
    """400 atoms over 48 element types (two element passes) in the 50 x 50 x
    70 A cell, d >= 1.5 A; the first 200,000 reflections of that list are
    used.  The fixed scratch then holds exactly two rows of partial sums (one
    per element pass) and not three."""
    import math
    rng = np.random.default_rng(48200)
    n, n_elem = 400, 48
    ff = np.concatenate([rng.uniform(0.5, 3.0, (n_elem, 4)), rng.uniform(0.5, 40.0, (n_elem, 4)),
                         rng.uniform(0.0, 1.0, (n_elem, 1))], axis=1)
    atoms = W.Atoms(frac=rng.uniform(0.0, 1.0, (n, 3)), B=rng.uniform(10.0, 30.0, n), occ=np.ones(n),
                    elem=rng.integers(0, n_elem, n).astype(np.uint8), ff=ff)
    br = W.Broadening(L=(300.0, 300.0, 300.0), g=(0.01, 0.01, 0.01), B_axis=(2.0, 3.0, 1.0), gamma=math.radians(4),
                      T=W.patch_extent(0.0, math.radians(4)), n_nodes=16)
    geom = W.Geometry(wavelength=1.0, distance=200.0, pixel=0.075, n_x=16, n_y=16)
    return W.Problem("two_pass_tight", (50.0, 50.0, 70.0, math.pi / 2, math.pi / 2, math.pi / 2), atoms, 1.5, 0.0,
                     br, geom)


def test_noalloc_two_passes_tight_fit(gpu):
    """Two element passes when only two rows of partials fit: the call uses one
    atom split per pass (two rows in all) and matches the workspace path.
    Sizes: 24 B per atom + 4 B per reflection + 16 B per reflection and row."""
    n_refl = 200_000
    assert 24 * 400 + 4 * n_refl + 2 * 16 * n_refl < 8 << 20 < 24 * 400 + 4 * n_refl + 3 * 16 * n_refl
    _compare(gpu, _two_pass_tight, n_refl=n_refl)
