"""Thin ctypes binding of libfdx (include/fdx.h).

Argument marshalling only: every step of the path runs in the CUDA library.
PyTorch supplies device memory (tensors) and the stream; the structs below
mirror the C structs field by field.  The functions carry the C entry points'
names.  There is no CPU fallback: if libfdx.so is missing or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdx.so")
_lock = threading.Lock()
_lib = None

FDX_OK = 0
LINESHAPE_SINC, LINESHAPE_HOSEMANN = 0, 1
INTENSITY_NONE, INTENSITY_HOSEMANN = 0, 1


class FdxError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s failed: %s (%d)" % (where, error_string(code), code))
        self.code = code


class Cell(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("c", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double)]


class Atoms(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("n_elem", C.c_int32), ("frac", C.c_void_p), ("B", C.c_void_p),
                ("occ", C.c_void_p), ("elem", C.c_void_p), ("ff", C.c_void_p)]


class Broadening(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("g", C.c_double * 3), ("B_axis", C.c_double * 3),
                ("lineshape", C.c_int32), ("intensity_model", C.c_int32),
                ("sigma", C.c_double), ("gamma", C.c_double), ("sigma_r", C.c_double), ("T", C.c_double),
                ("n_nodes", C.c_int32), ("reserved", C.c_int32), ("K_z", C.c_double)]


class Geometry(C.Structure):
    _fields_ = [("wavelength", C.c_double), ("distance", C.c_double), ("pixel", C.c_double),
                ("n_x", C.c_int32), ("n_y", C.c_int32), ("fiber_axis", C.c_double * 3),
                ("beam_axis", C.c_double * 3), ("delta_L", C.c_double)]


class Problem(C.Structure):
    _fields_ = [("cell", Cell), ("br", Broadening), ("geom", Geometry), ("n_refl", C.c_int32),
                ("reserved", C.c_int32), ("hkl", C.c_void_p), ("M", C.c_void_p)]


def lib():
    """Load libfdx.so (built in-tree by _build.py); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libfdx.so is not built (run `python -m paper_2608_23245_b300._build`)")
            L = C.CDLL(LIB_PATH)
            L.fdx_version.restype = C.c_int
            L.fdx_error_string.restype = C.c_char_p
            L.fdx_error_string.argtypes = [C.c_int]
            L.fdx_reflections.argtypes = [C.POINTER(Cell), C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                          C.POINTER(C.c_int32)]
            L.fdx_sf_workspace_size.restype = C.c_size_t
            L.fdx_sf_workspace_size.argtypes = [C.c_int32, C.c_int32]
            L.fdx_structure_factors.argtypes = [C.POINTER(Cell), C.POINTER(Atoms), C.POINTER(Broadening), C.c_int32,
                                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                                C.c_void_p]
            L.fdx_structure_factors_noalloc.argtypes = [C.POINTER(Cell), C.POINTER(Atoms), C.POINTER(Broadening),
                                                        C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.fdx_workspace_size.restype = C.c_size_t
            L.fdx_workspace_size.argtypes = [C.c_int32, C.POINTER(C.POINTER(Problem))]
            L.fdx_pattern.argtypes = [C.c_int32, C.POINTER(C.POINTER(Problem)), C.POINTER(C.c_void_p), C.c_void_p,
                                      C.c_size_t, C.c_void_p]
            L.fdx_pattern_evals.argtypes = [C.POINTER(Problem), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
            L.fdx_ring_workspace_size.restype = C.c_size_t
            L.fdx_ring_workspace_size.argtypes = [C.POINTER(Problem)]
            L.fdx_ring.argtypes = [C.POINTER(Problem), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
            L.fdx_ring_evals.argtypes = [C.POINTER(Problem), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
            L.fdx_scatter_workspace_size.restype = C.c_size_t
            L.fdx_scatter_workspace_size.argtypes = [C.POINTER(Problem), C.c_int32]
            L.fdx_scatter.argtypes = [C.POINTER(Problem), C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                      C.c_size_t, C.c_void_p]
            L.fdx_scatter_evals.argtypes = [C.POINTER(Problem), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_size_t, C.c_void_p]
            _lib = L
    return _lib


def error_string(code: int) -> str:
    return lib().fdx_error_string(int(code)).decode()


def _check(rc: int, where: str):
    if rc != FDX_OK:
        raise FdxError(rc, where)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# struct builders (from plain values or a workloads.Problem)
# ---------------------------------------------------------------------------

def make_cell(cell) -> Cell:
    return Cell(*[float(x) for x in cell])


def make_broadening(br) -> Broadening:
    b = Broadening()
    b.L[:] = [float(x) for x in br.L]
    b.g[:] = [float(x) for x in br.g]
    b.B_axis[:] = [float(x) for x in br.B_axis]
    b.lineshape = int(br.lineshape)
    b.intensity_model = int(br.intensity_model)
    b.sigma, b.gamma, b.sigma_r, b.T = float(br.sigma), float(br.gamma), float(br.sigma_r), float(br.T)
    b.n_nodes = int(br.n_nodes)
    b.K_z = float(br.K_z)
    return b


def make_geometry(ge) -> Geometry:
    g = Geometry()
    g.wavelength, g.distance, g.pixel = float(ge.wavelength), float(ge.distance), float(ge.pixel)
    g.n_x, g.n_y = int(ge.n_x), int(ge.n_y)
    g.fiber_axis[:] = [float(x) for x in ge.fiber_axis]
    g.beam_axis[:] = [float(x) for x in ge.beam_axis]
    g.delta_L = float(ge.delta_L)
    return g


def make_problem(cell, br, geom, hkl, M) -> Problem:
    """hkl: int32 [n, 3] and M: float32 [n] CUDA tensors (kept alive by the caller)."""
    p = Problem()
    p.cell = make_cell(cell)
    p.br = make_broadening(br)
    p.geom = make_geometry(geom)
    p.n_refl = int(hkl.shape[0])
    p.hkl = hkl.data_ptr() if p.n_refl else None
    p.M = M.data_ptr() if p.n_refl else None
    return p


class DeviceAtoms:
    """Device copies of an atom set in the C-ABI's dtypes (frac f64, B/occ/ff f32, elem u8)."""

    def __init__(self, atoms, device="cuda"):
        import torch
        self.frac = torch.as_tensor(np.ascontiguousarray(atoms.frac, np.float64), device=device)
        self.B = torch.as_tensor(np.ascontiguousarray(atoms.B, np.float32), device=device)
        self.occ = torch.as_tensor(np.ascontiguousarray(atoms.occ, np.float32), device=device)
        self.elem = torch.as_tensor(np.ascontiguousarray(atoms.elem, np.uint8), device=device)
        self.ff = torch.as_tensor(np.ascontiguousarray(atoms.ff, np.float32).reshape(-1, 9), device=device)

    def struct(self) -> Atoms:
        a = Atoms()
        a.n_atoms = int(self.frac.shape[0])
        a.n_elem = int(self.ff.shape[0])
        a.frac, a.B, a.occ = self.frac.data_ptr(), self.B.data_ptr(), self.occ.data_ptr()
        a.elem, a.ff = self.elem.data_ptr(), self.ff.data_ptr()
        return a


# ---------------------------------------------------------------------------
# entry points (names of include/fdx.h)
# ---------------------------------------------------------------------------

def fdx_version() -> int:
    return int(lib().fdx_version())


def fdx_status(stream=None) -> int:
    """Wait for the stream's queued work; returns its CUDA error code (0 =
    success) and raises FdxError when that work failed."""
    L = lib()
    L.fdx_status.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    code = C.c_int(0)
    rc = L.fdx_status(_stream(stream), C.byref(code))
    if rc != 0:
        raise FdxError(rc, "fdx_status: CUDA error %d on the stream" % code.value)
    return code.value


def fdx_debug_status():
    """Bounds checks of a debugging build (libfdx_debug.so): returns
    (checks_compiled_in, failed_check_bits, last_bad_index) and clears the
    record; a normal build returns (False, 0, -1)."""
    L = lib()
    L.fdx_debug_status.argtypes = [C.POINTER(C.c_ulonglong), C.POINTER(C.c_longlong)]
    flags, idx = C.c_ulonglong(0), C.c_longlong(0)
    rc = L.fdx_debug_status(C.byref(flags), C.byref(idx))
    if rc < 0:
        raise FdxError(rc, "fdx_debug_status")
    return bool(rc == 1), int(flags.value), int(idx.value)


def fdx_debug_probe(stream=None) -> bool:
    """Queue one deliberately failing bounds check in a debugging build
    (True); a normal build does nothing (False)."""
    L = lib()
    L.fdx_debug_probe.argtypes = [C.c_void_p]
    rc = L.fdx_debug_probe(_stream(stream) if stream is not None else None)
    if rc < 0:
        raise FdxError(rc, "fdx_debug_probe")
    return rc == 1


def fdx_reflections(cell, d_min, d_max=0.0) -> np.ndarray:
    """Reflection list as a host int32 [n, 3] array (count, then fill)."""
    c = make_cell(cell)
    n = C.c_int32(0)
    _check(lib().fdx_reflections(C.byref(c), float(d_min), float(d_max), 0, None, C.byref(n)), "fdx_reflections")
    out = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    _check(lib().fdx_reflections(C.byref(c), float(d_min), float(d_max), n.value, out.ctypes.data_as(C.c_void_p),
                                 C.byref(n)), "fdx_reflections")
    return out[:n.value]


def fdx_sf_workspace_size(n_atoms: int, n_refl: int) -> int:
    return int(lib().fdx_sf_workspace_size(int(n_atoms), int(n_refl)))


def fdx_structure_factors(cell, datoms: DeviceAtoms, hkl, br=None, F_out=None, M_out=None, workspace=None,
                          stream=None):
    """F (float32 [n, 2]) and M (float32 [n]) for device hkl (int32 [n, 3])."""
    import torch
    n = int(hkl.shape[0])
    dev = hkl.device
    if F_out is None:
        F_out = torch.empty((n, 2), dtype=torch.float32, device=dev)
    if M_out is None:
        M_out = torch.empty((n,), dtype=torch.float32, device=dev)
    need = fdx_sf_workspace_size(int(datoms.frac.shape[0]), n)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    c = make_cell(cell)
    a = datoms.struct()
    b = make_broadening(br) if br is not None else None
    _check(lib().fdx_structure_factors(C.byref(c), C.byref(a), C.byref(b) if b is not None else None, n,
                                       _ptr(hkl), _ptr(F_out), _ptr(M_out), _ptr(workspace),
                                       int(workspace.numel()), _stream(stream)), "fdx_structure_factors")
    return F_out, M_out


def fdx_structure_factors_noalloc(cell, datoms: DeviceAtoms, hkl, br=None, F_out=None, M_out=None, stream=None):
    """fdx_structure_factors without a workspace: the library's fixed device
    scratch (FDX_NOALLOC_SF_SCRATCH_BYTES) is used instead, so nothing is
    allocated for scratch.  Calls sharing that scratch must not overlap on the
    GPU."""
    import torch
    n = int(hkl.shape[0])
    dev = hkl.device
    if F_out is None:
        F_out = torch.empty((n, 2), dtype=torch.float32, device=dev)
    if M_out is None:
        M_out = torch.empty((n,), dtype=torch.float32, device=dev)
    c = make_cell(cell)
    a = datoms.struct()
    b = make_broadening(br) if br is not None else None
    _check(lib().fdx_structure_factors_noalloc(C.byref(c), C.byref(a), C.byref(b) if b is not None else None, n,
                                               _ptr(hkl), _ptr(F_out), _ptr(M_out), _stream(stream)),
           "fdx_structure_factors_noalloc")
    return F_out, M_out


def _problem_array(problems):
    arr = (C.POINTER(Problem) * len(problems))(*[C.pointer(p) for p in problems])
    return arr


def fdx_workspace_size(problems) -> int:
    return int(lib().fdx_workspace_size(len(problems), _problem_array(problems)))


def fdx_pattern(problems, images, workspace=None, stream=None):
    """images: list of float32 [n_y, n_x] CUDA tensors, one per problem."""
    import torch
    arr = _problem_array(problems)
    need = fdx_workspace_size(problems)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=images[0].device)
    ims = (C.c_void_p * len(images))(*[im.data_ptr() for im in images])
    _check(lib().fdx_pattern(len(problems), arr, ims, _ptr(workspace), int(workspace.numel()), _stream(stream)),
           "fdx_pattern")
    return images


def fdx_pattern_evals(problem, counts, workspace=None, stream=None):
    import torch
    need = fdx_workspace_size([problem])
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=counts.device)
    _check(lib().fdx_pattern_evals(C.byref(problem), _ptr(counts), _ptr(workspace), int(workspace.numel()),
                                   _stream(stream)), "fdx_pattern_evals")
    return counts


def fdx_ring_workspace_size(problem) -> int:
    return int(lib().fdx_ring_workspace_size(C.byref(problem)))


def fdx_ring(problem, image, workspace=None, stream=None):
    """Ring-integrated cylindrical average into image [n_y, n_x] float32 (device)."""
    import torch
    if workspace is None:
        workspace = torch.empty(fdx_ring_workspace_size(problem), dtype=torch.uint8, device=image.device)
    _check(lib().fdx_ring(C.byref(problem), _ptr(image), _ptr(workspace), int(workspace.numel()), _stream(stream)),
           "fdx_ring")
    return image


def fdx_ring_evals(problem, counts, workspace=None, stream=None):
    import torch
    if workspace is None:
        workspace = torch.empty(fdx_ring_workspace_size(problem), dtype=torch.uint8, device=counts.device)
    _check(lib().fdx_ring_evals(C.byref(problem), _ptr(counts), _ptr(workspace), int(workspace.numel()),
                                _stream(stream)), "fdx_ring_evals")
    return counts


def fdx_scatter_workspace_size(problem, n_samples: int) -> int:
    return int(lib().fdx_scatter_workspace_size(C.byref(problem), int(n_samples)))


def fdx_scatter(problem, samples, image, workspace=None, stream=None, spot_size=1):
    """Scatter form: samples [n_s, 4] float32 (device), image [n_y, n_x]
    float32 (device); each hit rendered as a spot_size x spot_size spot."""
    import torch
    n_s = int(samples.shape[0])
    if workspace is None:
        workspace = torch.empty(fdx_scatter_workspace_size(problem, n_s), dtype=torch.uint8, device=image.device)
    _check(lib().fdx_scatter(C.byref(problem), n_s, _ptr(samples), int(spot_size), _ptr(image), _ptr(workspace),
                             int(workspace.numel()), _stream(stream)), "fdx_scatter")
    return image


def fdx_scatter_evals(problem, samples, count, workspace=None, stream=None):
    """In-support (sample, node) term count of the scatter form into count (int64 scalar, device)."""
    import torch
    n_s = int(samples.shape[0])
    if workspace is None:
        workspace = torch.empty(fdx_scatter_workspace_size(problem, n_s), dtype=torch.uint8, device=count.device)
    _check(lib().fdx_scatter_evals(C.byref(problem), n_s, _ptr(samples), _ptr(count), _ptr(workspace),
                                   int(workspace.numel()), _stream(stream)), "fdx_scatter_evals")
    return count


# ---------------------------------------------------------------------------
# convenience: the whole forward path for one workloads.Problem
# ---------------------------------------------------------------------------

class Simulation:
    """Device-resident state for one problem: reflections, atoms, workspaces."""

    def __init__(self, problem, device="cuda"):
        import torch
        self.problem = problem
        self.device = device
        self.hkl_host = fdx_reflections(problem.cell, problem.d_min, problem.d_max)
        self.hkl = torch.as_tensor(self.hkl_host, device=device).contiguous()
        self.atoms = DeviceAtoms(problem.atoms, device)
        n = self.hkl.shape[0]
        self.F = torch.empty((n, 2), dtype=torch.float32, device=device)
        self.M = torch.empty((n,), dtype=torch.float32, device=device)
        self.sf_ws = torch.empty(max(fdx_sf_workspace_size(problem.atoms.n, n), 256), dtype=torch.uint8,
                                 device=device)
        self.prob = make_problem(problem.cell, problem.br, problem.geom, self.hkl, self.M)
        self.image = torch.empty((problem.geom.n_y, problem.geom.n_x), dtype=torch.float32, device=device)
        self.ws = torch.empty(max(fdx_workspace_size([self.prob]), 256), dtype=torch.uint8, device=device)

    def structure_factors(self, stream=None):
        fdx_structure_factors(self.problem.cell, self.atoms, self.hkl, self.problem.br, self.F, self.M, self.sf_ws,
                              stream)
        return self.F, self.M

    def pattern(self, stream=None):
        fdx_pattern([self.prob], [self.image], self.ws, stream)
        return self.image

    def forward(self, stream=None):
        self.structure_factors(stream)
        return self.pattern(stream)

    def evals(self, stream=None):
        import torch
        counts = torch.empty_like(self.image, dtype=torch.int32)
        fdx_pattern_evals(self.prob, counts, self.ws, stream)
        return counts

    def ring(self, image=None, workspace=None, stream=None):
        """Structure factors (for M) must have been computed; ring-average image."""
        import torch
        if image is None:
            image = torch.empty_like(self.image)
        return fdx_ring(self.prob, image, workspace, stream)

    def ring_evals(self, workspace=None, stream=None):
        import torch
        counts = torch.empty_like(self.image, dtype=torch.int32)
        return fdx_ring_evals(self.prob, counts, workspace, stream)

    def scatter(self, samples, image=None, workspace=None, stream=None, spot_size=1):
        """Structure factors (for M) must have been computed; scatter-form image."""
        import torch
        if image is None:
            image = torch.empty_like(self.image)
        return fdx_scatter(self.prob, samples, image, workspace, stream, spot_size)

    def scatter_evals(self, samples, workspace=None, stream=None):
        import torch
        count = torch.zeros((), dtype=torch.int64, device=self.image.device)
        fdx_scatter_evals(self.prob, samples, count, workspace, stream)
        return count


# ---------------------------------------------------------------------------
# refinement path: loss and the hand-written adjoint
# ---------------------------------------------------------------------------

class Grads(C.Structure):
    _fields_ = [("dfrac", C.c_void_p), ("dB", C.c_void_p), ("dglobal", C.c_void_p), ("dM", C.c_void_p)]


def _bind_refine(L):
    if getattr(L, "_refine_bound", False):
        return L
    L.fdx_backward_workspace_size.restype = C.c_size_t
    L.fdx_backward_workspace_size.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32]
    L.fdx_pattern_backward.argtypes = [C.POINTER(Problem), C.POINTER(Atoms), C.c_void_p, C.c_void_p,
                                       C.POINTER(Grads), C.c_void_p, C.c_size_t, C.c_void_p]
    L.fdx_loss_workspace_size.restype = C.c_size_t
    L.fdx_loss_workspace_size.argtypes = [C.c_int64]
    L.fdx_loss.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_size_t, C.c_void_p]
    L._refine_bound = True
    return L


def fdx_backward_workspace_size(problem, n_atoms: int, n_elem: int) -> int:
    return int(_bind_refine(lib()).fdx_backward_workspace_size(C.byref(problem), int(n_atoms), int(n_elem)))


def fdx_pattern_backward(problem, datoms: DeviceAtoms, F, dL_dI, dfrac=None, dB=None, dglobal=None, dM=None,
                         workspace=None, stream=None):
    """Gradients of a loss w.r.t. fractional coordinates, B, sizes, g, sigma
    and gamma given dL/dI; tensors passed as None are not written."""
    import torch
    L = _bind_refine(lib())
    a = datoms.struct()
    need = fdx_backward_workspace_size(problem, a.n_atoms, a.n_elem)
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dL_dI.device)
    g = Grads(dfrac.data_ptr() if dfrac is not None else None, dB.data_ptr() if dB is not None else None,
              dglobal.data_ptr() if dglobal is not None else None, dM.data_ptr() if dM is not None else None)
    _check(L.fdx_pattern_backward(C.byref(problem), C.byref(a), _ptr(F), _ptr(dL_dI), C.byref(g), _ptr(workspace),
                                  int(workspace.numel()), _stream(stream)), "fdx_pattern_backward")
    return dfrac, dB, dglobal, dM


def fdx_loss_workspace_size(n_px: int) -> int:
    return int(_bind_refine(lib()).fdx_loss_workspace_size(int(n_px)))


def fdx_loss(I, I_target, mask=None, loss_out=None, dL_dI=None, workspace=None, stream=None):
    """L = sum m (I - I_t)^2 / (I_t + 1) (device float64 scalar) and dL/dI."""
    import torch
    L = _bind_refine(lib())
    n = I.numel()
    if loss_out is None:
        loss_out = torch.empty((), dtype=torch.float64, device=I.device)
    if workspace is None:
        workspace = torch.empty(fdx_loss_workspace_size(n), dtype=torch.uint8, device=I.device)
    _check(L.fdx_loss(n, _ptr(I), _ptr(I_target), _ptr(mask), _ptr(loss_out), _ptr(dL_dI), _ptr(workspace),
                      int(workspace.numel()), _stream(stream)), "fdx_loss")
    return loss_out, dL_dI


# ---------------------------------------------------------------------------
# plain FP64 form of the method (comparison path)
# ---------------------------------------------------------------------------

def _bind_plain64(L):
    if getattr(L, "_plain64_bound", False):
        return L
    L.fdx_plain64_workspace_size.restype = C.c_size_t
    L.fdx_plain64_workspace_size.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32]
    L.fdx_plain64_refine.argtypes = [C.POINTER(Problem), C.POINTER(Atoms), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.POINTER(Grads), C.c_void_p, C.c_size_t, C.c_void_p]
    L._plain64_bound = True
    return L


def fdx_plain64_workspace_size(problem, n_atoms: int, n_elem: int) -> int:
    return int(_bind_plain64(lib()).fdx_plain64_workspace_size(C.byref(problem), int(n_atoms), int(n_elem)))


def fdx_plain64_refine(problem, datoms, image, I_target=None, mask=None, loss=None, dfrac=None, dB=None,
                       dglobal=None, workspace=None, stream=None):
    """Plain FP64 forward (image, float64 [n_y, n_x]) and, with I_target,
    the FP64 loss and adjoint."""
    import torch
    L = _bind_plain64(lib())
    a = datoms.struct()
    need = fdx_plain64_workspace_size(problem, a.n_atoms, a.n_elem)
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=image.device)
    g = Grads(dfrac.data_ptr() if dfrac is not None else None, dB.data_ptr() if dB is not None else None,
              dglobal.data_ptr() if dglobal is not None else None, None)
    _check(L.fdx_plain64_refine(C.byref(problem), C.byref(a), _ptr(I_target), _ptr(mask), _ptr(image), _ptr(loss),
                                C.byref(g), _ptr(workspace), int(workspace.numel()), _stream(stream)),
           "fdx_plain64_refine")
    return image, loss


# ---------------------------------------------------------------------------
# batched refinement of many models
# ---------------------------------------------------------------------------

def _bind_batch(L):
    if getattr(L, "_batch_bound", False):
        return L
    P = C.POINTER(C.POINTER(Problem))
    A = C.POINTER(C.POINTER(Atoms))
    V = C.POINTER(C.c_void_p)
    L.fdx_batch_workspace_size.restype = C.c_size_t
    L.fdx_batch_workspace_size.argtypes = [C.c_int32, P, A]
    L.fdx_batch_refine.argtypes = [C.c_int32, P, A, V, V, V, V, V, C.c_void_p, C.POINTER(C.POINTER(Grads)),
                                   C.c_void_p, C.c_size_t, C.c_void_p]
    L._batch_bound = True
    return L


def _atoms_array(atoms_structs):
    return (C.POINTER(Atoms) * len(atoms_structs))(*[C.pointer(a) for a in atoms_structs])


def _vptrs(tensors):
    return (C.c_void_p * len(tensors))(*[(t.data_ptr() if t is not None else None) for t in tensors])


def fdx_batch_workspace_size(problems, atoms_structs) -> int:
    L = _bind_batch(lib())
    return int(L.fdx_batch_workspace_size(len(problems), _problem_array(problems), _atoms_array(atoms_structs)))


class BatchStep:
    """Device buffers and argument arrays for fdx_batch_refine over fixed
    problems; call() issues the whole step on the current stream (capturable
    in a CUDA graph: every argument is a device pointer fixed at construction)."""

    def __init__(self, problems, datoms, targets=None, masks=None, device="cuda"):
        import torch
        self.problems = problems
        self.datoms = datoms
        self.astructs = [d.struct() for d in datoms]
        n = len(problems)
        self.F = [torch.empty((p.n_refl, 2), dtype=torch.float32, device=device) for p in problems]
        self.M = [torch.empty((max(p.n_refl, 1),), dtype=torch.float32, device=device) for p in problems]
        self.images = [torch.empty((p.geom.n_y, p.geom.n_x), dtype=torch.float32, device=device) for p in problems]
        self.targets = targets
        self.masks = masks
        self.losses = torch.zeros(n, dtype=torch.float64, device=device)
        self.dfrac = [torch.empty((a.n_atoms, 3), dtype=torch.float64, device=device) for a in self.astructs]
        self.dB = [torch.empty((a.n_atoms,), dtype=torch.float64, device=device) for a in self.astructs]
        self.dglobal = [torch.empty(8, dtype=torch.float64, device=device) for _ in problems]
        self.dM = [torch.empty((max(p.n_refl, 1),), dtype=torch.float32, device=device) for p in problems]
        self.gstructs = [Grads(self.dfrac[m].data_ptr(), self.dB[m].data_ptr(), self.dglobal[m].data_ptr(),
                               self.dM[m].data_ptr()) for m in range(n)]
        self.ws = torch.empty(max(fdx_batch_workspace_size(problems, self.astructs), 256), dtype=torch.uint8,
                              device=device)
        self._args = (n, _problem_array(problems), _atoms_array(self.astructs), _vptrs(self.F), _vptrs(self.M),
                      _vptrs(self.images), _vptrs(targets) if targets is not None else None,
                      _vptrs(masks) if masks is not None else None,
                      C.c_void_p(self.losses.data_ptr()) if targets is not None else None,
                      (C.POINTER(Grads) * n)(*[C.pointer(g) for g in self.gstructs]) if targets is not None else None,
                      C.c_void_p(self.ws.data_ptr()), int(self.ws.numel()))

    def __call__(self, stream=None):
        L = _bind_batch(lib())
        _check(L.fdx_batch_refine(*self._args, _stream(stream)), "fdx_batch_refine")


class Tuning(C.Structure):
    _fields_ = [("ppl_max", C.c_int32), ("fwd_ctas_per_sm", C.c_int32), ("adj_ctas_per_sm", C.c_int32),
                ("adj_bands", C.c_int32), ("node_block", C.c_int32)]

    DEFAULTS = {"ppl_max": 2, "fwd_ctas_per_sm": 4, "adj_ctas_per_sm": 3, "adj_bands": 128, "node_block": 1}

    @classmethod
    def of(cls, **knobs):
        """A tuning with the library defaults, overridden by `knobs`."""
        v = dict(cls.DEFAULTS)
        v.update(knobs)
        return cls(**v)

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


def fdx_set_tuning(t=None):
    L = lib()
    L.fdx_set_tuning.argtypes = [C.POINTER(Tuning)]
    _check(L.fdx_set_tuning(C.byref(t) if t is not None else None), "fdx_set_tuning")


def fdx_get_tuning() -> Tuning:
    L = lib()
    L.fdx_get_tuning.argtypes = [C.POINTER(Tuning)]
    t = Tuning()
    _check(L.fdx_get_tuning(C.byref(t)), "fdx_get_tuning")
    return t
