"""Write the FP64 oracle's values of the large forward workload at sampled
pixels, for the full-size GPU parity test (tests/test_gpu_fullsize.py).

The workload is the 20,000-atom, 50 x 50 x 70 A cell (d >= 1.5 A: 217,252
reflections, Lorentzian 4 deg, L = 300 A, 128^2 nodes, 2048^2 detector of
0.075 mm pixels at 200 mm) with Hosemann g = 1 % and g = 4 %, inputs rounded
to the C-ABI's float32 where it takes float32.  The pixel set is 1,024 seeded
pixels over the whole detector, the full meridian column (i = n_x / 2) and
the full equator row (j = n_y / 2).  Per pixel the oracle gives I (Eq.
direct_sum x Eq. lorentz, structure factors by Eq. structure_factor), the
in-support term counts (exact, support shrunk by 1e-6, grown by 1e-6) and
the summed magnitude of the terms whose inclusion is decided within 1e-6 of
the support's edge (which the GPU, deciding in FP32, may take either way).

Only oracle/ computes here; the file also stores a fingerprint of the inputs
so that a change of the workload recipe makes the test fail instead of
comparing against stale values.  Run from the repository root:

    python tests/golden/make_config2_samples.py
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "config2_oracle_samples.npz")
G_VALUES = (0.01, 0.04)


def _rounded(problem):
    from dataclasses import replace
    a = problem.atoms
    atoms = replace(a, B=a.B.astype(np.float32).astype(np.float64),
                    occ=a.occ.astype(np.float32).astype(np.float64),
                    ff=a.ff.astype(np.float32).astype(np.float64))
    return replace(problem, atoms=atoms)


def problem(g):
    sys.path.insert(0, ROOT)
    from paper_2608_23245_b300 import workloads as W
    return _rounded(W.config2(g))


def pixels(p):
    """1,024 seeded pixels over the detector, then the meridian column and
    the equator row; (i, j) int32 pairs."""
    nx, ny = p.geom.n_x, p.geom.n_y
    rng = np.random.default_rng(2608202)
    rand = np.stack([rng.integers(0, nx, 1024), rng.integers(0, ny, 1024)], 1)
    mer = np.stack([np.full(ny, nx // 2), np.arange(ny)], 1)
    equ = np.stack([np.arange(nx), np.full(nx, ny // 2)], 1)
    return np.concatenate([rand, mer, equ]).astype(np.int32)


def fingerprint(p, hkl, pix) -> str:
    h = hashlib.sha256()
    a = p.atoms
    for arr in (a.frac, a.B, a.occ, a.elem, a.ff, np.asarray(hkl, np.int32), pix):
        h.update(np.ascontiguousarray(arr).tobytes())
    br, ge = p.br, p.geom
    h.update(repr((p.cell, p.d_min, p.d_max, br.L, br.g, br.B_axis, br.lineshape, br.intensity_model, br.sigma,
                   br.gamma, br.sigma_r, br.T, br.n_nodes, br.K_z, ge.wavelength, ge.distance, ge.pixel, ge.n_x,
                   ge.n_y, ge.fiber_axis, ge.beam_axis, ge.delta_L)).encode())
    return h.hexdigest()


def main():
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    out = {}
    p0 = problem(G_VALUES[0])
    hkl = oracle.reflections(p0.cell, p0.d_min, p0.d_max)
    pix = pixels(p0)
    t0 = time.time()
    F = oracle.structure_factors(p0.cell, p0.atoms, hkl)   # independent of g
    print("structure factors: %.1f s" % (time.time() - t0), flush=True)
    out["pix"] = pix
    for g in G_VALUES:
        p = problem(g)
        M = oracle.intensities_M(p, hkl, F)
        t0 = time.time()
        I, E, A = oracle.pattern(p, hkl, M, pix, with_ambiguous=True)
        print("g = %g: %d pixels in %.1f s" % (g, len(pix), time.time() - t0), flush=True)
        key = "g%d" % round(1000 * g)
        out[key + "_I"] = I
        out[key + "_E"] = E
        out[key + "_A"] = A
        out[key + "_fp"] = np.array(fingerprint(p, hkl, pix))
    np.savez_compressed(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
