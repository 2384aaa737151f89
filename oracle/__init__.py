"""FP64 CPU oracle for the fiber-diffraction hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The computation lives in
``fdx_oracle.c`` (plain C, FP64, OpenMP over pixels); this module compiles it
with gcc and marshals numpy arrays through ctypes.  It shares no code with the
GPU library and never imports it.

Loss helpers at the bottom follow the refinement loss of the scope:
L = sum_px w_px (I_sim - I_target)^2 with w_px = 1 / (I_target + 1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-Wno-unused-function", "-o", _LIB_PATH, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("cell", C.c_double * 6),
        ("L", C.c_double * 3),
        ("g", C.c_double * 3),
        ("B_axis", C.c_double * 3),
        ("lineshape", C.c_int32),
        ("intensity_model", C.c_int32),
        ("sigma", C.c_double),
        ("gamma", C.c_double),
        ("sigma_r", C.c_double),
        ("T", C.c_double),
        ("n_nodes", C.c_int32),
        ("pad0", C.c_int32),
        ("K_z", C.c_double),
        ("wavelength", C.c_double),
        ("distance", C.c_double),
        ("pixel", C.c_double),
        ("n_x", C.c_int32),
        ("n_y", C.c_int32),
        ("fiber", C.c_double * 3),
        ("beam", C.c_double * 3),
        ("delta_L", C.c_double),
    ]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            L.or_basis.argtypes = [_dp, _dp, _dp]
            L.or_reflections.argtypes = [_dp, C.c_double, C.c_double, C.c_int32, _ip]
            L.or_reflections.restype = C.c_int32
            L.or_structure_factors.argtypes = [_dp, C.c_int32, _dp, _dp, _dp, _ip, _dp, C.c_int32, _ip, _dp]
            L.or_refl_scalars.argtypes = [C.POINTER(Params), C.c_int32, _ip, _dp, _dp, _dp]
            L.or_lineshape.argtypes = [C.c_int32, C.c_double, C.c_double, C.POINTER(C.c_double)]
            L.or_lineshape.restype = C.c_double
            L.or_support.argtypes = [C.c_int32, C.c_double, C.c_double]
            L.or_support.restype = C.c_double
            L.or_angular.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_angular.restype = C.c_double
            L.or_nodes.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp]
            L.or_pixel_S.argtypes = [C.POINTER(Params), C.c_int32, C.c_int32, _dp,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_pattern.argtypes = [C.POINTER(Params), C.c_int32, _ip, _dp, C.c_int32, _ip, C.c_int32,
                                     C.c_double, _dp, _lp, C.c_void_p]
            L.or_pattern_adjoint.argtypes = [C.POINTER(Params), C.c_int32, _ip, _dp, C.c_int32, _ip, _dp,
                                             _dp, _dp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_chain_globals.argtypes = [C.POINTER(Params), C.c_int32, _ip, _dp, _dp, _dp, _dp, _dp]
            L.or_sf_adjoint.argtypes = [_dp, C.c_int32, _dp, _dp, _dp, _ip, _dp, C.c_int32, _ip, _dp, _dp,
                                        _dp, _dp]
            L.or_scatter.argtypes = [C.POINTER(Params), C.c_int32, _ip, _dp, C.c_int32, _dp, C.c_int32, _dp,
                                     C.c_void_p, C.POINTER(C.c_int64)]
            L.or_ring.argtypes = [C.POINTER(Params), C.c_int32, _ip, _dp, C.c_int32, _ip, C.c_int32, C.c_int32,
                                  _dp, _lp]
            L.or_point.argtypes = [C.POINTER(Params), C.c_int32, _ip, _dp, C.c_int32, _dp, _dp]
            L.or_ring_grid.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                                       C.POINTER(C.c_double), C.POINTER(C.c_int32)]
            L.or_num_threads.restype = C.c_int32
            L.or_set_threads.argtypes = [C.c_int32]
            _lib = L
    return _lib


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _i32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def params(problem, **over) -> Params:
    """Flatten a workloads.Problem (cell, broadening, geometry) into the C struct."""
    br, ge = problem.br, problem.geom
    P = Params()
    P.cell[:] = list(problem.cell)
    P.L[:] = list(br.L)
    P.g[:] = list(br.g)
    P.B_axis[:] = list(br.B_axis)
    P.lineshape = int(br.lineshape)
    P.intensity_model = int(br.intensity_model)
    P.sigma = float(br.sigma)
    P.gamma = float(br.gamma)
    P.sigma_r = float(br.sigma_r)
    P.T = float(br.T)
    P.n_nodes = int(br.n_nodes)
    P.K_z = float(br.K_z)
    P.wavelength = float(ge.wavelength)
    P.distance = float(ge.distance)
    P.pixel = float(ge.pixel)
    P.n_x = int(ge.n_x)
    P.n_y = int(ge.n_y)
    P.fiber[:] = list(ge.fiber_axis)
    P.beam[:] = list(ge.beam_axis)
    P.delta_L = float(ge.delta_L)
    for k, v in over.items():
        if isinstance(getattr(P, k), C.Array):
            getattr(P, k)[:] = list(v)
        else:
            setattr(P, k, v)
    return P


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------------------
# thin wrappers
# ---------------------------------------------------------------------------

def basis(cell):
    A = np.zeros(9)
    As = np.zeros(9)
    lib().or_basis(_f64(cell), A, As)
    return A.reshape(3, 3), As.reshape(3, 3)


def reflections(cell, d_min, d_max=0.0) -> np.ndarray:
    c = _f64(cell)
    dummy = np.zeros(3, dtype=np.int32)
    n = lib().or_reflections(c, float(d_min), float(d_max), 0, dummy)
    hkl = np.zeros((max(n, 1), 3), dtype=np.int32)
    lib().or_reflections(c, float(d_min), float(d_max), n, hkl)
    return hkl[:n].copy()


def structure_factors(cell, atoms, hkl) -> np.ndarray:
    """Complex F for each hkl (Eq. structure_factor)."""
    hkl = _i32(hkl).reshape(-1, 3)
    F = np.zeros(2 * max(len(hkl), 1))
    lib().or_structure_factors(_f64(cell), atoms.n, _f64(atoms.frac).reshape(-1), _f64(atoms.B), _f64(atoms.occ),
                               _i32(atoms.elem), _f64(atoms.ff).reshape(-1), len(hkl), hkl.reshape(-1), F)
    F = F[:2 * len(hkl)]
    return F[0::2] + 1j * F[1::2]


def refl_scalars(problem, hkl, **over):
    hkl = _i32(hkl).reshape(-1, 3)
    n = len(hkl)
    beta = np.zeros(3 * max(n, 1))
    P = np.zeros(max(n, 1))
    DW = np.zeros(max(n, 1))
    prm = params(problem, **over)
    lib().or_refl_scalars(C.byref(prm), n, hkl.reshape(-1), beta, P, DW)
    return beta[:3 * n].reshape(n, 3), P[:n], DW[:n]


def intensities_M(problem, hkl, F=None, **over):
    """M = |F|^2 P DW_axis per reflection."""
    if F is None:
        F = structure_factors(problem.cell, problem.atoms, hkl)
    _, P, DW = refl_scalars(problem, hkl, **over)
    return np.abs(F) ** 2 * P * DW


def lineshape(kind, t, beta, with_derivative=False):
    d = C.c_double(0.0)
    v = lib().or_lineshape(int(kind), float(t), float(beta), C.byref(d))
    return (v, d.value) if with_derivative else v


def support(kind, beta, K_z=3.0):
    return lib().or_support(int(kind), float(beta), float(K_z))


def angular(delta, sigma, gamma, with_derivatives=False):
    ds = C.c_double(0.0)
    dg = C.c_double(0.0)
    v = lib().or_angular(float(delta), float(sigma), float(gamma), C.byref(ds), C.byref(dg))
    return (v, ds.value, dg.value) if with_derivatives else v


def nodes(problem, **over):
    prm = params(problem, **over)
    n = prm.n_nodes
    out = [np.zeros(n * n) for _ in range(5)]
    lib().or_nodes(C.byref(prm), *out)
    return tuple(o.reshape(n, n) for o in out)


def pixel_S(problem, i, j, **over):
    prm = params(problem, **over)
    S = np.zeros(3)
    R = C.c_double(0.0)
    Z = C.c_double(0.0)
    lib().or_pixel_S(C.byref(prm), int(i), int(j), S, C.byref(R), C.byref(Z))
    return S, R.value, Z.value


def all_pixels(problem) -> np.ndarray:
    """(i, j) pairs of every pixel in row-major image order (row j, column i)."""
    nx, ny = problem.geom.n_x, problem.geom.n_y
    jj, ii = np.meshgrid(np.arange(ny, dtype=np.int32), np.arange(nx, dtype=np.int32), indexing="ij")
    return np.stack([ii.reshape(-1), jj.reshape(-1)], axis=1).astype(np.int32)


def pattern(problem, hkl, M, pix=None, cull=True, eta=1e-6, with_ambiguous=False, **over):
    """Pixel values I (Eq. direct_sum x Eq. lorentz) and in-support term counts.

    Returns (I[n_pix], E[n_pix, 3]) with E columns (exact, strict, loose);
    with_ambiguous adds A[n_pix], the summed magnitude of the terms whose
    inclusion is decided within eta of the support's edge."""
    if pix is None:
        pix = all_pixels(problem)
    pix = _i32(pix).reshape(-1, 2)
    hkl = _i32(hkl).reshape(-1, 3)
    prm = params(problem, **over)
    I = np.zeros(max(len(pix), 1))
    E = np.zeros(3 * max(len(pix), 1), dtype=np.int64)
    A = np.zeros(max(len(pix), 1)) if with_ambiguous else None
    lib().or_pattern(C.byref(prm), len(hkl), hkl.reshape(-1), _f64(M), len(pix), pix.reshape(-1),
                     int(bool(cull)), float(eta), I, E, A.ctypes.data_as(C.c_void_p) if A is not None else None)
    if with_ambiguous:
        return I[:len(pix)], E[:3 * len(pix)].reshape(-1, 3), A[:len(pix)]
    return I[:len(pix)], E[:3 * len(pix)].reshape(-1, 3)


RING_MAX_N = 1024  # cap on the azimuth points per reflection of the ring average


def ring(problem, hkl, M, pix=None, max_n=RING_MAX_N, refine=1, **over):
    """Ring-integrated cylindrical average (Eq. cyl-average) at the pixels;
    returns (I[n_pix], E[n_pix]) with E the in-support term counts.  refine > 1
    multiplies the azimuth points (convergence checks; 1 is the definition)."""
    if pix is None:
        pix = all_pixels(problem)
    pix = _i32(pix).reshape(-1, 2)
    hkl = _i32(hkl).reshape(-1, 3)
    prm = params(problem, **over)
    I = np.zeros(max(len(pix), 1))
    E = np.zeros(max(len(pix), 1), dtype=np.int64)
    lib().or_ring(C.byref(prm), len(hkl), hkl.reshape(-1), _f64(M), len(pix), pix.reshape(-1), int(max_n),
                  int(refine), I, E)
    return I[:len(pix)], E[:len(pix)]


def point(problem, hkl, M, pts, **over):
    """Reciprocal-space intensity sum_r M r0^2 sum_k w_k prod K at 3-D points [n, 3]."""
    hkl = _i32(hkl).reshape(-1, 3)
    pts = _f64(pts).reshape(-1, 3)
    prm = params(problem, **over)
    I = np.zeros(max(len(pts), 1))
    lib().or_point(C.byref(prm), len(hkl), hkl.reshape(-1), _f64(M), len(pts), pts.reshape(-1), I)
    return I[:len(pts)]


def ring_grid(r0, RD, rhoB, T, w_min, max_n=RING_MAX_N):
    """(Phi_r, N_r) of the ring average's azimuth rule for one reflection."""
    Phi, N = C.c_double(0.0), C.c_int32(0)
    lib().or_ring_grid(float(r0), float(RD), float(rhoB), float(T), float(w_min), int(max_n), C.byref(Phi),
                       C.byref(N))
    return Phi.value, N.value


def scatter(problem, hkl, M, samples, with_samples=False, spot=1, **over):
    """Scatter form: image [n_y, n_x] accumulated over all reflections and
    samples (samples [n_s, 4]: xi_r, xi_1, xi_2, q), each hit rendered as a
    spot x spot block (spot odd), the in-support count, and optionally per
    (reflection, sample) rows (I, dV, L, x0, y0, x1, y1, distance of the
    nearest node from the edge of the support)."""
    if spot < 1 or spot % 2 == 0:
        raise ValueError("spot size must be a positive odd number of pixels")
    hkl = _i32(hkl).reshape(-1, 3)
    xs = _f64(samples).reshape(-1, 4)
    prm = params(problem, **over)
    img = np.zeros(problem.geom.n_x * problem.geom.n_y)
    E = C.c_int64(0)
    samp = np.zeros(8 * max(1, len(hkl) * len(xs))) if with_samples else None
    lib().or_scatter(C.byref(prm), len(hkl), hkl.reshape(-1), _f64(M), len(xs), xs.reshape(-1), int(spot), img,
                     samp.ctypes.data_as(C.c_void_p) if samp is not None else None, C.byref(E))
    img = img.reshape(problem.geom.n_y, problem.geom.n_x)
    if with_samples:
        return img, E.value, samp[:8 * len(hkl) * len(xs)].reshape(len(hkl), len(xs), 8)
    return img, E.value


def pattern_adjoint(problem, hkl, M, gI, pix=None, **over):
    if pix is None:
        pix = all_pixels(problem)
    pix = _i32(pix).reshape(-1, 2)
    hkl = _i32(hkl).reshape(-1, 3)
    n = len(hkl)
    prm = params(problem, **over)
    G = np.zeros(max(n, 1))
    dbeta = np.zeros(3 * max(n, 1))
    ds = C.c_double(0.0)
    dg = C.c_double(0.0)
    lib().or_pattern_adjoint(C.byref(prm), n, hkl.reshape(-1), _f64(M), len(pix), pix.reshape(-1), _f64(gI),
                             G, dbeta, C.byref(ds), C.byref(dg))
    return G[:n], dbeta[:3 * n].reshape(n, 3), ds.value, dg.value


def chain_globals(problem, hkl, F2, G, dbeta, **over):
    hkl = _i32(hkl).reshape(-1, 3)
    prm = params(problem, **over)
    dL = np.zeros(3)
    dg = np.zeros(3)
    lib().or_chain_globals(C.byref(prm), len(hkl), hkl.reshape(-1), _f64(F2), _f64(G), _f64(dbeta).reshape(-1),
                           dL, dg)
    return dL, dg


def sf_adjoint(cell, atoms, hkl, F, Gw):
    hkl = _i32(hkl).reshape(-1, 3)
    Fri = np.zeros(2 * max(len(hkl), 1))
    Fri[0:2 * len(hkl):2] = np.real(F)
    Fri[1:2 * len(hkl):2] = np.imag(F)
    dfrac = np.zeros(3 * max(atoms.n, 1))
    dB = np.zeros(max(atoms.n, 1))
    lib().or_sf_adjoint(_f64(cell), atoms.n, _f64(atoms.frac).reshape(-1), _f64(atoms.B), _f64(atoms.occ),
                        _i32(atoms.elem), _f64(atoms.ff).reshape(-1), len(hkl), hkl.reshape(-1), Fri, _f64(Gw),
                        dfrac, dB)
    return dfrac[:3 * atoms.n].reshape(-1, 3), dB[:atoms.n]


# ---------------------------------------------------------------------------
# refinement loss (scope: L = sum w (I - I_t)^2, w = 1/(I_t + 1))
# ---------------------------------------------------------------------------

def loss_and_grad(I, I_target):
    I = np.asarray(I, dtype=np.float64)
    It = np.asarray(I_target, dtype=np.float64)
    w = 1.0 / (It + 1.0)
    r = I - It
    return float(np.sum(w * r * r)), 2.0 * w * r


def full_gradient(problem, hkl, I_target, pix=None):
    """Loss and its gradient w.r.t. fractional coordinates, B, sizes L, g,
    sigma and gamma, through the whole forward path."""
    F = structure_factors(problem.cell, problem.atoms, hkl)
    beta, P, DW = refl_scalars(problem, hkl)
    F2 = np.abs(F) ** 2
    M = F2 * P * DW
    I, _ = pattern(problem, hkl, M, pix)
    loss, gI = loss_and_grad(I, I_target)
    G, dbeta, dsig, dgam = pattern_adjoint(problem, hkl, M, gI, pix)
    dL, dg = chain_globals(problem, hkl, F2, G, dbeta)
    dfrac, dB = sf_adjoint(problem.cell, problem.atoms, hkl, F, G * P * DW)
    return loss, {"frac": dfrac, "B": dB, "L": dL, "g": dg, "sigma": dsig, "gamma": dgam}, I
