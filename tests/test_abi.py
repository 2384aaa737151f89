"""CPU-side checks of the C-ABI library: it loads, exports every entry point
declared in include/fdx.h, and rejects bad arguments on the host before any
device work (these calls return before touching a GPU)."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fdx():
    from paper_2608_23245_b300 import _build, fdx
    _build.build()
    return fdx


def _declared():
    src = open(os.path.join(ROOT, "include", "fdx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdx_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(fdx):
    names = _declared()
    assert {"fdx_reflections", "fdx_structure_factors", "fdx_pattern", "fdx_workspace_size"} <= set(names)
    lib = fdx.lib()
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_errors(fdx):
    assert fdx.fdx_version() >= 100
    for code in (0, -1, -2, -3, -4, -5):
        assert fdx.error_string(code)
    assert fdx.error_string(1234) == "unknown error"


def _problem(fdx, **geo):
    from paper_2608_23245_b300 import workloads as W
    p = W.small_helix()
    g = p.geom
    for k, v in geo.items():
        g = type(g)(**{**g.__dict__, k: v})
    prob = fdx.Problem()
    prob.cell = fdx.make_cell(p.cell)
    prob.br = fdx.make_broadening(p.br)
    prob.geom = fdx.make_geometry(g)
    prob.n_refl = 3
    prob.hkl = 16   # never dereferenced: validation fails first
    prob.M = 16
    return prob


def test_pattern_geometry_tilt_and_parallel_axes(fdx):
    """A fiber axis tilted towards the beam is accepted (fiber tilt, Sect.
    Experimental geometry); a fiber axis parallel to the beam has no detector
    frame and is rejected with FDX_ERR_GEOMETRY before any work is queued."""
    lib = fdx.lib()
    prob = _problem(fdx, beam_axis=(1.0, 0.0, 0.5))
    assert lib.fdx_workspace_size(1, fdx._problem_array([prob])) > 0
    prob = _problem(fdx, beam_axis=(0.0, 0.0, 1.0))
    arr = fdx._problem_array([prob])
    ims = (C.c_void_p * 1)(16)
    assert lib.fdx_pattern(1, arr, ims, C.c_void_p(256), 1 << 30, None) == -2
    prob = _problem(fdx, beam_axis=(1e-7, 0.0, -1.0))
    assert lib.fdx_pattern(1, fdx._problem_array([prob]), ims, C.c_void_p(256), 1 << 30, None) == -2


def test_pattern_rejects_bad_arguments(fdx):
    lib = fdx.lib()
    ims = (C.c_void_p * 1)(16)
    for kw in ({"n_x": 0}, {"pixel": -1.0}, {"wavelength": float("nan")}, {"delta_L": 0.0}):
        prob = _problem(fdx, **kw)
        assert lib.fdx_pattern(1, fdx._problem_array([prob]), ims, C.c_void_p(256), 1 << 30, None) == -1
    prob = _problem(fdx)
    prob.br.n_nodes = 0
    assert lib.fdx_pattern(1, fdx._problem_array([prob]), ims, C.c_void_p(256), 1 << 30, None) == -1
    prob = _problem(fdx)
    prob.br.lineshape = 7
    assert lib.fdx_pattern(1, fdx._problem_array([prob]), ims, C.c_void_p(256), 1 << 30, None) == -1
    prob = _problem(fdx)
    assert lib.fdx_pattern(0, fdx._problem_array([prob]), ims, C.c_void_p(256), 1 << 30, None) == -1
    # workspace too small / misaligned
    need = lib.fdx_workspace_size(1, fdx._problem_array([prob]))
    assert lib.fdx_pattern(1, fdx._problem_array([prob]), ims, C.c_void_p(256), need - 1, None) == -3
    assert lib.fdx_pattern(1, fdx._problem_array([prob]), ims, C.c_void_p(260), need, None) == -3


def test_reflections_count_mode_and_capacity(fdx):
    """Count/fill protocol on a host buffer (integer enumeration only)."""
    lib = fdx.lib()
    cell = fdx.make_cell((9.0, 9.0, 15.0, math.pi / 2, math.pi / 2, math.pi / 2))
    n = C.c_int32(-1)
    assert lib.fdx_reflections(C.byref(cell), 2.5, 0.0, 0, None, C.byref(n)) == 0
    assert n.value == 304
    buf = (C.c_int32 * 30)()
    assert lib.fdx_reflections(C.byref(cell), 2.5, 0.0, 10, buf, C.byref(n)) == -5
    assert lib.fdx_reflections(C.byref(cell), 0.0, 0.0, 0, None, C.byref(n)) == -2
    bad = fdx.make_cell((9.0, 9.0, 15.0, math.pi / 2, math.pi / 2, 3 * math.pi / 2))
    assert lib.fdx_reflections(C.byref(bad), 2.5, 0.0, 0, None, C.byref(n)) == -2


def test_structure_factor_argument_checks(fdx):
    lib = fdx.lib()
    cell = fdx.make_cell((9.0, 9.0, 15.0, math.pi / 2, math.pi / 2, math.pi / 2))
    a = fdx.Atoms()
    a.n_atoms, a.n_elem = 0, 1
    assert lib.fdx_structure_factors(C.byref(cell), C.byref(a), None, 5, C.c_void_p(16), C.c_void_p(16), None,
                                     C.c_void_p(256), 1 << 20, None) == -1
    a.n_atoms, a.n_elem = 10, 65
    a.frac = a.B = a.elem = a.ff = 16
    assert lib.fdx_structure_factors(C.byref(cell), C.byref(a), None, 5, C.c_void_p(16), C.c_void_p(16), None,
                                     C.c_void_p(256), 1 << 20, None) == -1
    a.n_elem = 4
    need = lib.fdx_sf_workspace_size(10, 5)
    assert need > 0
    assert lib.fdx_structure_factors(C.byref(cell), C.byref(a), None, 5, C.c_void_p(16), C.c_void_p(16), None,
                                     C.c_void_p(256), need - 1, None) == -3


def test_ring_and_scatter_argument_checks(fdx):
    """Host-side rejections of the ring average and the scatter form (before
    any device work): bad geometry, parallel axes, missing outputs or samples,
    misaligned samples, short or misaligned workspace."""
    lib = fdx.lib()
    img = C.c_void_p(16)
    for kw, code in (({"n_x": 0}, -1), ({"beam_axis": (0.0, 0.0, 1.0)}, -2)):
        prob = _problem(fdx, **kw)
        assert lib.fdx_ring(C.byref(prob), img, C.c_void_p(256), 1 << 30, None) == code
        assert lib.fdx_scatter(C.byref(prob), 16, C.c_void_p(16), 1, img, C.c_void_p(256), 1 << 30, None) == code
    prob = _problem(fdx)
    need = lib.fdx_ring_workspace_size(C.byref(prob))
    assert need >= lib.fdx_workspace_size(1, fdx._problem_array([prob]))
    assert lib.fdx_ring(C.byref(prob), None, C.c_void_p(256), need, None) == -1
    assert lib.fdx_ring(C.byref(prob), img, C.c_void_p(256), need - 1, None) == -3
    assert lib.fdx_ring(C.byref(prob), img, C.c_void_p(264), need, None) == -3
    need_s = lib.fdx_scatter_workspace_size(C.byref(prob), 64)
    assert need_s > lib.fdx_scatter_workspace_size(C.byref(prob), 32) > 0
    assert lib.fdx_scatter(C.byref(prob), 0, C.c_void_p(16), 1, img, C.c_void_p(256), need_s, None) == -1
    assert lib.fdx_scatter(C.byref(prob), 64, None, 1, img, C.c_void_p(256), need_s, None) == -1
    assert lib.fdx_scatter(C.byref(prob), 64, C.c_void_p(24), 1, img, C.c_void_p(256), need_s, None) == -1
    assert lib.fdx_scatter(C.byref(prob), 64, C.c_void_p(16), 1, img, C.c_void_p(256), need_s - 1, None) == -3
    for spot in (0, 2, -1, 17):     # the detector spot is an odd block of 1..15 pixels
        assert lib.fdx_scatter(C.byref(prob), 64, C.c_void_p(16), spot, img, C.c_void_p(256), need_s, None) == -1


def test_ring_workspace_holds_the_split_partials(fdx):
    """A small detector deals each reflection's azimuth points to several warps
    per patch and needs room for their partial images; a detector of 1024 x
    1024 pixels keeps one warp per patch and needs none."""
    lib = fdx.lib()
    small = _problem(fdx, n_x=30, n_y=24)
    assert lib.fdx_ring_workspace_size(C.byref(small)) >= lib.fdx_workspace_size(1, fdx._problem_array([small])) \
        + 8 * 30 * 24 * 2
    big = _problem(fdx, n_x=1024, n_y=1024)
    extra = lib.fdx_ring_workspace_size(C.byref(big)) - lib.fdx_workspace_size(1, fdx._problem_array([big]))
    assert 0 < extra < 16 * 64 * 4 + 4096  # the ring records only


def test_backward_and_loss_argument_checks(fdx):
    """An unknown lineshape, missing inputs and short workspaces are rejected
    on the host (the adjoint covers the three lineshapes)."""
    lib = fdx._bind_refine(fdx.lib())
    prob = _problem(fdx)
    a = fdx.Atoms()
    a.n_atoms, a.n_elem = 10, 4
    a.frac = a.B = a.elem = a.ff = 16
    g = fdx.Grads()
    prob.br.lineshape = 3  # no such lineshape
    assert lib.fdx_pattern_backward(C.byref(prob), C.byref(a), C.c_void_p(16), C.c_void_p(16), C.byref(g),
                                    C.c_void_p(256), 1 << 30, None) == -1
    prob.br.lineshape = 1
    assert lib.fdx_pattern_backward(C.byref(prob), C.byref(a), C.c_void_p(16), None, C.byref(g),
                                    C.c_void_p(256), 1 << 30, None) == -1
    need = lib.fdx_backward_workspace_size(C.byref(prob), 10, 4)
    assert need > 0
    assert lib.fdx_pattern_backward(C.byref(prob), C.byref(a), C.c_void_p(16), C.c_void_p(16), C.byref(g),
                                    C.c_void_p(256), need - 1, None) == -3
    loss = C.c_double(0.0)
    assert lib.fdx_loss(0, C.c_void_p(16), C.c_void_p(16), None, C.byref(loss), None, C.c_void_p(256), 1 << 20,
                        None) == -1
    assert lib.fdx_loss(100, C.c_void_p(16), C.c_void_p(16), None, C.byref(loss), None, C.c_void_p(256),
                        lib.fdx_loss_workspace_size(100) - 1, None) == -3


def _noalloc_call(fdx, cell, n_atoms, n_elem, n_refl, br=None):
    """fdx_structure_factors_noalloc with dummy device pointers: only calls
    that fail validation or sizing may be made this way (nothing is read)."""
    lib = fdx.lib()
    c = fdx.make_cell(cell)
    a = fdx.Atoms()
    a.n_atoms, a.n_elem = n_atoms, n_elem
    a.frac = a.B = a.elem = a.ff = 256
    return lib.fdx_structure_factors_noalloc(C.byref(c), C.byref(a), C.byref(br) if br is not None else None,
                                             n_refl, C.c_void_p(256), C.c_void_p(256), None, None)


def test_noalloc_rejects_two_pass_problem_with_one_row_of_room(fdx):
    """With more than 40 element types the structure factors take two element
    passes, each writing its own row of partial sums.  2,000 atoms and 250,000
    reflections leave room in the fixed 8 MiB scratch for one row of partials
    (24 B per atom + 4 B per reflection + 16 B per reflection and row) but not
    two: with 48 types the call must refuse (FDX_ERR_WORKSPACE) instead of
    writing a second row past the scratch."""
    orth = (50.0, 50.0, 70.0, math.pi / 2, math.pi / 2, math.pi / 2)
    per_row = 16 * 250_000
    assert 24 * 2000 + 4 * 250_000 + 2 * per_row > 8 << 20 > 24 * 2000 + 4 * 250_000 + per_row
    assert _noalloc_call(fdx, orth, 2000, 48, 250_000) == -3


def test_noalloc_validates_like_workspace_path(fdx):
    """The allocation-free entry point refuses the same cells and broadening
    parameters as fdx_structure_factors, with the same codes: a cell with an
    angle outside (0, pi) or no volume is a geometry error, a broadening
    record with a bad size, lineshape or node count an argument error."""
    lib = fdx.lib()
    from paper_2608_23245_b300 import workloads as W
    p = W.small_helix()
    a = fdx.Atoms()
    a.n_atoms, a.n_elem = 100, 4
    a.frac = a.B = a.elem = a.ff = 256
    bad_cells = [(10.0, 10.0, 10.0, 0.0, math.pi / 2, math.pi / 2),
                 (10.0, 10.0, 10.0, math.pi, math.pi / 2, math.pi / 2),
                 (10.0, 10.0, 10.0, 2.0, 2.0, 2.3)]          # angles with no positive volume
    for cell in bad_cells:
        c = fdx.make_cell(cell)
        ws = lib.fdx_structure_factors(C.byref(c), C.byref(a), None, 10, C.c_void_p(256), C.c_void_p(256), None,
                                       C.c_void_p(256), 1 << 30, None)
        na = _noalloc_call(fdx, cell, 100, 4, 10)
        assert ws == na == -2, (cell, ws, na)
    for field, value in (("L", (0.0, 1.0, 1.0)), ("lineshape", 7), ("n_nodes", 0), ("T", 0.0), ("K_z", -1.0)):
        br = fdx.make_broadening(p.br)
        setattr(br, field, type(getattr(br, field))(*value) if isinstance(value, tuple) else value)
        c = fdx.make_cell(p.cell)
        ws = lib.fdx_structure_factors(C.byref(c), C.byref(a), C.byref(br), 10, C.c_void_p(256), C.c_void_p(256),
                                       None, C.c_void_p(256), 1 << 30, None)
        na = _noalloc_call(fdx, p.cell, 100, 4, 10, br)
        assert ws == na == -1, (field, ws, na)


def test_status_reports_cuda_failure_without_device(fdx):
    """fdx_status waits for a stream and reports how its work ended; on a
    machine without a usable CUDA device the wait itself fails, which must
    come back as FDX_ERR_CUDA with the nonzero CUDA code (never FDX_OK)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: the GPU tests cover fdx_status")
    lib = fdx.lib()
    lib.fdx_status.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    code = C.c_int(0)
    assert lib.fdx_status(None, C.byref(code)) == -4
    assert code.value != 0
    assert lib.fdx_status(None, None) == -4


def test_debug_status_of_a_normal_build(fdx):
    """The product library has no bounds checks compiled in: fdx_debug_status
    reports so without touching the device."""
    assert fdx.fdx_debug_status() == (False, 0, -1)
    assert fdx.fdx_debug_probe() is False
