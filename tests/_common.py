"""Shared test helpers: input rounding to the C-ABI's dtypes and the parity
metrics of the scope (max |dI| <= 1e-5 max I, relative L2 <= 1e-6)."""
from dataclasses import replace

import numpy as np

# Accuracy gates for FP32 results against the FP64 oracle.
MAX_REL = 1e-5   # max |dI| / max |I_oracle|
L2_REL = 1e-6    # ||dI||_2 / ||I_oracle||_2


def api_precision(problem):
    """The problem with B, occupancy and form factors rounded to float32, the
    precision the C-ABI takes them in, so oracle and GPU see identical inputs."""
    a = problem.atoms
    atoms = replace(a, B=a.B.astype(np.float32).astype(np.float64),
                    occ=a.occ.astype(np.float32).astype(np.float64),
                    ff=a.ff.astype(np.float32).astype(np.float64))
    return replace(problem, atoms=atoms)


def parity(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    d = got - ref
    mx = float(np.max(np.abs(ref))) if ref.size else 0.0
    max_rel = float(np.max(np.abs(d)) / mx) if mx > 0 else float(np.max(np.abs(d)) if d.size else 0.0)
    nrm = float(np.linalg.norm(ref))
    l2 = float(np.linalg.norm(d) / nrm) if nrm > 0 else float(np.linalg.norm(d))
    return max_rel, l2


def amp_scale(p, hkl):
    """sqrt(sum_j amp_j^2) per reflection (amp_j = occ_j f_j(s) exp(-B_j s^2/4)):
    the natural scale of a direct sum's rounding error, used only to set the
    structure-factor tolerance |dF| <= SF_TOL * amp_scale."""
    a = p.atoms
    from oracle import basis
    _, As = basis(p.cell)
    s2_all = np.sum((np.asarray(hkl, np.float64) @ As) ** 2, axis=1)
    ff = a.ff[a.elem]
    out = np.empty(s2_all.shape[0])
    step = max(1, (1 << 22) // max(1, 4 * a.n))   # reflections per chunk: bounded temporaries
    for r0 in range(0, s2_all.shape[0], step):
        s2 = s2_all[r0:r0 + step]
        f = ff[:, 8][None, :] + np.sum(ff[None, :, 0:4] * np.exp(-ff[None, :, 4:8] * s2[:, None, None] / 4), axis=2)
        amp = a.occ[None, :] * f * np.exp(-a.B[None, :] * s2[:, None] / 4)
        out[r0:r0 + step] = np.sqrt(np.sum(amp * amp, axis=1))
    return out


SF_TOL = 2e-6   # |F_gpu - F_ref| <= SF_TOL * amp_scale per reflection


def oracle_hkl(orc, problem, lib_hkl):
    """The oracle's own reflection list for `problem`, after checking that the
    library's list (the order the GPU results are in) is the same, entry for
    entry (integer work: bit-exact).  Oracle calls take this list, never the
    library's."""
    h = np.asarray(orc.reflections(problem.cell, problem.d_min, problem.d_max), dtype=np.int32).reshape(-1, 3)
    lib = np.asarray(lib_hkl, dtype=np.int32).reshape(-1, 3)
    assert h.shape == lib.shape and np.array_equal(h, lib), "library and oracle reflection lists differ"
    return h
