"""Fit the polynomial coefficients used by the kernels (writes poly_coeffs.cuh).

Method: weighted least squares on Chebyshev nodes, refined by a few Lawson
iterations (iteratively reweighted least squares towards the minimax error),
in numpy float64.  Targets:
  sin(2 pi r) = r * S(r^2),      |r| <= 1/8 turn   (relative error)
  cos(2 pi r) = C(r^2),          |r| <= 1/8 turn   (absolute error)
  sin(2 pi r) = r * SH(r^2),     |r| <= 1/4 turn   (relative error; structure factors)
  cos(2 pi r) = CH(r^2),         |r| <= 1/4 turn   (absolute error; structure factors)
  sin^2(pi t) = t^2 * Q(t^2),    |t| <= 1/2        (relative error)
Run:  python paper_2608_23245_b300/csrc/fit_poly.py
"""
import os
import numpy as np


def lawson(f, x, deg, rel=True, iters=60):
    V = np.vander(x, deg + 1, increasing=True)
    y = f(x)
    w = np.ones_like(x)
    scale = np.abs(y) if rel else np.ones_like(y)
    for _ in range(iters):
        W = np.sqrt(w) / scale
        c, *_ = np.linalg.lstsq(V * W[:, None], y * W, rcond=None)
        err = np.abs(V @ c - y) / scale
        w = w * (err + 1e-300)
        w /= w.sum()
    return c, err.max()


def cheb(a, b, n=4000):
    k = np.arange(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / n)


def main():
    u = cheb(1e-12, (1 / 8) ** 2)
    S, eS = lawson(lambda u: np.sin(2 * np.pi * np.sqrt(u)) / np.sqrt(u), u, 3, rel=True)
    Cc, eC = lawson(lambda u: np.cos(2 * np.pi * np.sqrt(u)), u, 4, rel=False)
    uh = cheb(1e-12, (1 / 4) ** 2)
    SH, eSH = lawson(lambda u: np.sin(2 * np.pi * np.sqrt(u)) / np.sqrt(u), uh, 4, rel=True)
    CH, eCH = lawson(lambda u: np.cos(2 * np.pi * np.sqrt(u)), uh, 5, rel=False)
    v = cheb(1e-12, 0.25)
    Q, eQ = lawson(lambda v: np.sin(np.pi * np.sqrt(v)) ** 2 / v, v, 5, rel=True)
    out = ["/* Generated by fit_poly.py (weighted least squares + Lawson iterations). */",
           "#pragma once",
           "/* sin(2 pi r) = r * S(r^2), |r| <= 1/8; max rel err %.2e */" % eS,
           "#define FDX_SIN2PI_C {" + ", ".join("%.9ef" % c for c in S) + "}",
           "/* cos(2 pi r) = C(r^2), |r| <= 1/8; max abs err %.2e */" % eC,
           "#define FDX_COS2PI_C {" + ", ".join("%.9ef" % c for c in Cc) + "}",
           "/* sin(2 pi r) = r * SH(r^2), |r| <= 1/4; max rel err %.2e */" % eSH,
           "#define FDX_SIN2PI_H_C {" + ", ".join("%.9ef" % c for c in SH) + "}",
           "/* cos(2 pi r) = CH(r^2), |r| <= 1/4; max abs err %.2e */" % eCH,
           "#define FDX_COS2PI_H_C {" + ", ".join("%.9ef" % c for c in CH) + "}",
           "/* sin^2(pi t) = t^2 * Q(t^2), |t| <= 1/2; max rel err %.2e */" % eQ,
           "#define FDX_SINPI2_C {" + ", ".join("%.9ef" % c for c in Q) + "}",
           ""]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "poly_coeffs.cuh")
    open(path, "w").write("\n".join(out))
    print("\n".join(out))
    # float32 evaluation check (Horner, as the kernels do)
    def horner32(c, x):
        c = np.asarray(c, np.float32)
        x = np.asarray(x, np.float32)
        acc = np.full_like(x, c[-1])
        for k in range(len(c) - 2, -1, -1):
            acc = (acc * x + c[k]).astype(np.float32)
        return acc
    r = np.linspace(-1 / 8, 1 / 8, 200001).astype(np.float32)
    s32 = r * horner32(S, r * r)
    c32 = horner32(Cc, r * r)
    print("sin f32 max abs err", np.max(np.abs(s32 - np.sin(2 * np.pi * r.astype(np.float64)))))
    print("cos f32 max abs err", np.max(np.abs(c32 - np.cos(2 * np.pi * r.astype(np.float64)))))
    r = np.linspace(-1 / 4, 1 / 4, 200001).astype(np.float32)
    s32 = r * horner32(SH, r * r)
    c32 = horner32(CH, r * r)
    print("half-turn sin f32 max abs err", np.max(np.abs(s32 - np.sin(2 * np.pi * r.astype(np.float64)))))
    print("half-turn cos f32 max abs err", np.max(np.abs(c32 - np.cos(2 * np.pi * r.astype(np.float64)))))
    t = np.linspace(-0.5, 0.5, 200001).astype(np.float32)
    q32 = (t * t) * horner32(Q, t * t)
    ref = np.sin(np.pi * t.astype(np.float64)) ** 2
    m = ref > 1e-30
    print("sin^2 f32 max rel err", np.max(np.abs(q32[m] - ref[m]) / ref[m]))


if __name__ == "__main__":
    main()
