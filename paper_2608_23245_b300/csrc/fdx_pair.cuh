// One (pixel patch, reflection) pair of the shell quadrature, shared by the
// forward pattern kernel (pixel-major) and the adjoint kernel
// (reflection-major).  A warp owns an 8 x (4 PPL) pixel patch, PPL pixels per
// lane.
//
// For the pair the warp
//   1. bounds the node rows/columns that can be in any lane's support by the
//      gnomonic projection of the support-box corners around the patch's
//      reference point, widened by the patch's spread;
//   2. culls blocks of 32 nodes at their centres, then computes, one node per
//      lane, sigma_i(k) = a_i . (s_k - p_ref) relative to the reference point
//      (the patch's central pixel) with float-float differences, keeps the
//      nodes whose sigma lies within the warp's tau range widened by the
//      support half-width, and compacts them into the warp's shared buffer;
//   3. every lane walks the buffer: t_i = tau_i - sigma_i with
//      tau_i = a_i . (p - p_ref), support test, lineshape product, weight.
// Partial sums of 32 nodes are folded into float-float accumulators.
//
// For the Hosemann lineshape the node walk runs on packed FP32 pairs
// (__fadd2_rn/__fmul2_rn/__ffma2_rn: one instruction, two lanes of work):
// the staged nodes are stored pairwise (even node, odd node) and every
// arithmetic step of the walk handles two nodes of one pixel at once.
#pragma once

#include <type_traits>

#include "fdx_internal.cuh"

namespace fdx {

static constexpr int PAIR_WARPS = 4;     // warps per CTA in the pattern kernels
static constexpr int NODE_BUF = 512;     // staged nodes per warp

enum PairMode { MODE_FWD = 0, MODE_CNT = 1, MODE_ADJ = 2 };

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FDX_FULL_MASK, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FDX_FULL_MASK, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FDX_FULL_MASK, v, o);
    return v;
}

// Hosemann denominator den = beta^2 + (1 - beta^2) sin^2(pi t), sin^2(pi t) =
// x Q(x), x = t^2, folded into one degree-6 polynomial in x (coefficients c
// scaled per reflection).  K = beta / den.
__device__ __forceinline__ float hosemann_den(float t, const float (&c)[7]) {
    const float x = t * t;
    float d = c[6];
#pragma unroll
    for (int k = 5; k >= 0; --k) d = fmaf(d, x, c[k]);
    return d;
}

// Sinc lineshape product: with x = N t, y = x - rint(x),
// sinc^2(x) = Q(y^2) (y^2 / x^2) / pi^2 (the ratio is 1 when rint(x) = 0);
// returns prod_i Q(y_i^2) (y_i^2 / x_i^2), the factor prod N_i / pi^6 being in
// the pair factor.
__device__ __forceinline__ float sinc_term(float ta, float tb, float tc, const float *Nn) {
    const float Qc[6] = FDX_SINPI2_C;
    float num = 1.0f, den = 1.0f, q = 1.0f;
    const float tt[3] = {ta, tb, tc};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float x = Nn[i] * tt[i];
        const float k = rintf(x);
        const float y = x - k;
        const float y2 = y * y;
        q *= horner(Qc, y2);
        if (k != 0.0f) {
            num *= y2;
            den *= x * x;
        }
    }
    return q * __fdividef(num, den);
}

// Gaussian lineshape product: prod_i exp(-pi t_i^2 / beta_i^2) = 2^-(sum LA_i t_i^2)
// with LA_i = pi log2(e) / beta_i^2 (one SFU exp2); the factor prod 1/beta_i is
// in the pair factor.
__device__ __forceinline__ float gauss_term(float ta, float tb, float tc, const float *la) {
    const float x = fmaf(la[0] * ta, ta, fmaf(la[1] * tb, tb, la[2] * tc * tc));
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}

// Forward declaration (defined below).
__device__ __forceinline__ void sincospi_f(float x, float &s, float &c);

// Lineshape value K and its derivative dK/dbeta at fixed t for the adjoint of
// the non-Hosemann lineshapes (absolute values, unlike the forward's
// normalised products):
//   sinc (Eq. I_shape, N = 1/beta):  K = N sinc^2(N t),
//     dK/dbeta = -N^2 dK/dN = -N^2 sinc(x) (2 cos(pi x) - sinc(x)),  x = N t;
//   Gaussian of breadth beta:        K = 2^(-LA t^2) / beta, LA = pi log2(e) / beta^2,
//     dK/dbeta = (K / beta) (2 ln 2 LA t^2 - 1)   (= (K / beta)(2 pi t^2 / beta^2 - 1)).
__device__ __forceinline__ void sinc_k_dk(float t, float N, float &K, float &dK) {
    const float x = N * t;
    float sn, cs;
    sincospi_f(x, sn, cs);
    const float px = 3.14159265358979f * x;
    const float sc = fabsf(px) < 1e-3f ? fmaf(-px * px, 1.0f / 6.0f, 1.0f) : sn / px;
    K = N * sc * sc;
    dK = -N * N * sc * (2.0f * cs - sc);
}
__device__ __forceinline__ void gauss_k_dk(float t, float la, float beta, float &K, float &dK) {
    const float e = la * t * t;
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-e));
    const float ib = 1.0f / beta;
    K = y * ib;
    dK = K * ib * fmaf(2.0f * 0.69314718056f, e, -1.0f);
}

// sin(pi x), cos(pi x) for |x| < 2^20: x = q/2 + f with q = rint(2x), |f| <= 1/4,
// so pi x = q pi/2 + pi f; sin(pi f), cos(pi f) from the sin(2 pi r)/cos(2 pi r)
// polynomials at r = f/2, then a rotation by q quarter turns.
__device__ __forceinline__ void sincospi_f(float x, float &s, float &c) {
    const float q = rintf(2.0f * x);
    const float r = 0.5f * fmaf(-0.5f, q, x);
    const float Sc[4] = FDX_SIN2PI_C;
    const float Cc[5] = FDX_COS2PI_C;
    const float r2 = r * r;
    const float sn = r * horner(Sc, r2);
    const float cs = horner(Cc, r2);
    const int qi = (int)q;
    const float s1 = (qi & 1) ? cs : sn;
    const float c1 = (qi & 1) ? -sn : cs;
    s = (qi & 2) ? -s1 : s1;
    c = (qi & 2) ? -c1 : c1;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// sincospi_f for two arguments: the reduction and the polynomials on packed
// FP32x2 pairs, the quarter-turn rotation per element.
__device__ __forceinline__ void sincospi_f2(float2 x, float2 &s, float2 &c) {
    const float2 q = make_float2(rintf(2.0f * x.x), rintf(2.0f * x.y));
    const float2 r = __fmul2_rn(f2(0.5f), __ffma2_rn(f2(-0.5f), q, x));
    const float Sc[4] = FDX_SIN2PI_C;
    const float Cc[5] = FDX_COS2PI_C;
    const float2 r2 = __fmul2_rn(r, r);
    float2 S = f2(Sc[3]), C = f2(Cc[4]);
#pragma unroll
    for (int k = 2; k >= 0; --k) S = __ffma2_rn(S, r2, f2(Sc[k]));
#pragma unroll
    for (int k = 3; k >= 0; --k) C = __ffma2_rn(C, r2, f2(Cc[k]));
    S = __fmul2_rn(r, S);
    const int q0 = (int)q.x, q1 = (int)q.y;
    const float s0 = (q0 & 1) ? C.x : S.x, c0 = (q0 & 1) ? -S.x : C.x;
    const float s1 = (q1 & 1) ? C.y : S.y, c1 = (q1 & 1) ? -S.y : C.y;
    s = make_float2((q0 & 2) ? -s0 : s0, (q1 & 2) ? -s1 : s1);
    c = make_float2((q0 & 2) ? -c0 : c0, (q1 & 2) ? -c1 : c1);
}

// v if |a| <= ta and |b| <= tb and |c| <= tc, else o (one predicate chain).
__device__ __forceinline__ float support_sel(float a, float b, float c, float ta, float tb, float tc, float v, float o) {
    float r;
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.f32 p, %1, %4;\n\t"
        "setp.le.and.f32 p, %2, %5, p;\n\t"
        "setp.le.and.f32 p, %3, %6, p;\n\t"
        "selp.f32 %0, %7, %8, p;\n\t}"
        : "=f"(r)
        : "f"(fabsf(a)), "f"(fabsf(b)), "f"(fabsf(c)), "f"(ta), "f"(tb), "f"(tc), "f"(v), "f"(o));
    return r;
}

// A warp's pixels: PPL pixels per lane at (px0 + lane % 8, py0 + lane / 8 + 4 p),
// p < PPL, so the warp covers an 8 x 4 PPL patch.  The reference pixel is the
// patch's central pixel (column 4, row 2 PPL) when it lies on the detector,
// else the first pixel: offsets from it (tau) stay small, which is what keeps
// t = tau - sigma accurate in FP32.  (R, Z) as float-float.
template <int PPL>
struct PatchPix {
    float Rh[PPL], Rl[PPL], Zh[PPL], Zl[PPL];  // this lane's pixels
    float dRl[PPL], dZl[PPL];                  // (R, Z) - reference, small
    bool valid[PPL];
    float Rrh, Rrl, Zrh, Zrl;                  // reference
};

template <int PPL>
__device__ __forceinline__ PatchPix<PPL> load_patch(const float4 *pixgeo, int nx, int ny, int px0, int py0, int lane) {
    PatchPix<PPL> g;
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        const int px = px0 + (lane & 7), py = py0 + (lane >> 3) + 4 * p;
        g.valid[p] = (px < nx) && (py < ny);
        const size_t pidx = g.valid[p] ? (size_t)py * nx + px : (size_t)py0 * nx + px0;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (FDX_IN_BOUNDS(pidx, (long long)nx * ny, DBG_PIXGEO)) v = pixgeo[pidx];
        g.Rh[p] = v.x, g.Rl[p] = v.y, g.Zh[p] = v.z, g.Zl[p] = v.w;
    }
    // central pixel: row 2 PPL = lane-row (2 PPL) % 4 of pixel set (2 PPL) / 4
    constexpr int cp = (2 * PPL) / 4, clane = 4 + 8 * ((2 * PPL) % 4);
    const bool cvalid = __shfl_sync(FDX_FULL_MASK, g.valid[cp], clane);
    const int rl = cvalid ? clane : 0;
    const float rRh = cvalid ? g.Rh[cp] : g.Rh[0], rRl = cvalid ? g.Rl[cp] : g.Rl[0];
    const float rZh = cvalid ? g.Zh[cp] : g.Zh[0], rZl = cvalid ? g.Zl[cp] : g.Zl[0];
    g.Rrh = __shfl_sync(FDX_FULL_MASK, rRh, rl), g.Rrl = __shfl_sync(FDX_FULL_MASK, rRl, rl);
    g.Zrh = __shfl_sync(FDX_FULL_MASK, rZh, rl), g.Zrl = __shfl_sync(FDX_FULL_MASK, rZl, rl);
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        g.dRl[p] = (g.Rh[p] - g.Rrh) + (g.Rl[p] - g.Rrl);
        g.dZl[p] = (g.Zh[p] - g.Zrh) + (g.Zl[p] - g.Zrl);
    }
    return g;
}

struct PairAcc {
    ff s0;           // sum of w / prod den (Hosemann) or w * sinc product
    ff sb[3];        // adjoint: sum of (w / prod den) / den_i
    ff ss, sg;       // adjoint: sums of dw/dsigma / prod den and dw/dgamma / prod den
    int32_t cnt;     // count mode: in-support terms
};

__device__ __forceinline__ void clear(PairAcc &a) {
    a.s0 = a.sb[0] = a.sb[1] = a.sb[2] = a.ss = a.sg = ff{0.0f, 0.0f};
    a.cnt = 0;
}

// Evaluate the pair for all PPL pixels of every lane; `rec` is the reflection
// record in shared memory.  Node buffers of the warp (NB nodes each): `buf`
// (sigma_a, sigma_b, sigma_c, w), `buf2` (adjoint: dw/dsigma, dw/dgamma, as
// float2 per node), and for the Hosemann lineshape `bsc` (NB float4) and
// `bsc2` (NB/2 float4) for the scaled cos, sin of pi sigma_i.  Before the
// Hosemann walk the buffers are rearranged in place into node pairs u:
//   buf[2u]  = (-sigma_a, -sigma_a', -sigma_b, -sigma_b'),  buf[2u+1] = (-sigma_c, -sigma_c', w, w'),
//   bsc[2u]  = (C_a, C_a', S_a, S_a'),  bsc[2u+1] = (C_b, C_b', S_b, S_b'),  bsc2[u] = (C_c, C_c', S_c, S_c'),
//   buf2[u]  = (dw_s, dw_s', dw_g, dw_g')   (primes: the odd node of the pair),
// with C_i = sqrt(1 - beta_i^2) cos(pi sigma_i), S_i likewise with sin.
// In the Hosemann walks (forward and adjoint), nodes are staged in two lists:
// "core" nodes (slots [0, NB/2)) lie inside the support of every valid pixel
// of the warp, by a margin far above FP32 rounding, so their walk needs no
// support test (an invalid point's terms there are finite and weighted by 0 in
// the adjoint, never written in the forward); the others ("rim", slots
// [NB/2, NB)) are tested per pixel.  Returns false when no node can be
// in any pixel's support.
//
// Hosemann denominators by angle addition: with t = tau - sigma,
//   sin(pi t) = sin(pi tau) cos(pi sigma) - cos(pi tau) sin(pi sigma),
//   den_i = beta_i^2 + (1 - beta_i^2) sin^2(pi t_i),
// sin/cos(pi tau) once per pixel and pair, sin/cos(pi sigma) (scaled by
// sqrt(1 - beta_i^2)) once per staged node: one FMA per denominator on top of
// the two products.
// Query points of one warp for one reflection: per lane and point p, the
// offset (p - D)/r0 in the reflection frame (FP32, bounds only), tau_i =
// a_i . (p - p_ref) (small; 1e4 for invalid points, far outside any support),
// and the warp's reference offset (p_ref - D)/r0 in float-float.
template <int PPL>
struct QueryPts {
    float P[PPL][3];
    float tau[PPL][3];
    bool valid[PPL];
    ff dP[3];
    float cw[PPL];  // adjoint: weight of each point's sums (dL/dI x Lorentz factor)
};

// Pixel query points (reading R12): p = Z n + R e_R(D) for the lane's pixels.
template <int PPL>
__device__ __forceinline__ QueryPts<PPL> pixel_queries(const PatternParams &P, const PatchPix<PPL> &g, const float *rec) {
    QueryPts<PPL> q;
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        const float dZ = (g.Zh[p] - rec[REC_ZD]) + (g.Zl[p] - rec[REC_ZD + 1]);
        const float dR = (g.Rh[p] - rec[REC_RD]) + (g.Rl[p] - rec[REC_RD + 1]);
#pragma unroll
        for (int k = 0; k < 3; ++k) q.P[p][k] = fmaf(dZ, rec[REC_NFR + k], dR * rec[REC_EFR + k]);
        q.valid[p] = g.valid[p];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            q.tau[p][i] = g.valid[p] ? fmaf(g.dZl[p], P.AZ[i], g.dRl[p] * rec[REC_AR + i]) : 1.0e4f;
    }
    const ff dZr = ff_add(two_sum(g.Zrh, -rec[REC_ZD]), ff{g.Zrl, -rec[REC_ZD + 1]});
    const ff dRr = ff_add(two_sum(g.Rrh, -rec[REC_RD]), ff{g.Rrl, -rec[REC_RD + 1]});
#pragma unroll
    for (int k = 0; k < 3; ++k)
        q.dP[k] = ff_add(ff_mul(dZr, ff{rec[REC_NFR + k], rec[REC_NFR + 3 + k]}),
                         ff_mul(dRr, ff{rec[REC_EFR + k], rec[REC_EFR + 3 + k]}));
    return q;
}

template <int LS, int MODE, int NB, int PPL>
__device__ __forceinline__ bool eval_core(const PatternParams &P, const QueryPts<PPL> &qp, const float *rec,
                                          float4 *buf, float4 *buf2, float4 *bsc, float4 *bsc2, int lane,
                                          PairAcc (&acc)[PPL]) {
    constexpr bool PACKED = (LS == FDX_LINESHAPE_HOSEMANN && MODE != MODE_CNT);
    const int n = P.n_nodes;
    // Node rows/columns that can be in any point's support: the gnomonic
    // projection d = X_perp / X_0 of the 8 corners of the support box around
    // the reference point, X = (1, 0, 0) + (p_ref - D)/r0 + corner (one corner
    // per lane on lanes 0-7), widened for the other points.  A point at
    // p_ref + r0 delta, |delta| <= Dl, moves a corner's projection by at most
    // Dl (1 + |d_i|) / (X_0 - Dl) along d_i.  FP32, bounds only (the ranges get
    // one more node on each side).
    float Dl = 0.0f;
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        if (!qp.valid[p]) continue;
        const float e0 = qp.P[p][0] - qp.dP[0].hi, e1 = qp.P[p][1] - qp.dP[1].hi, e2 = qp.P[p][2] - qp.dP[2].hi;
        Dl = fmaxf(Dl, sqrtf(fmaf(e0, e0, fmaf(e1, e1, e2 * e2))));
    }
    Dl = warp_max(Dl) * 1.0001f + 1e-7f;
    int j0 = n, j1 = -1, m0 = n, m1 = -1;
    bool degenerate = false;
    if (lane < 8) {
        const int v = lane & 3;
        const float sg = (lane & 4) ? -1.0f : 1.0f;
        const float X0 = 1.0f + qp.dP[0].hi + sg * rec[REC_CR + 3 * v];
        const float X1 = qp.dP[1].hi + sg * rec[REC_CR + 3 * v + 1];
        const float X2 = qp.dP[2].hi + sg * rec[REC_CR + 3 * v + 2];
        const float den = X0 - Dl;
        degenerate = !(den > 0.05f);
        if (!degenerate) {
            const float inv = rcp_approx(X0), ivd = rcp_approx(den);  // bounds only
            const float d1 = X1 * inv, d2 = X2 * inv;
            const float w1 = Dl * (1.0f + fabsf(d1)) * ivd, w2 = Dl * (1.0f + fabsf(d2)) * ivd;
            const float T = P.T, ih = P.inv_h;
            j0 = max(0, (int)ceilf(fmaf(d1 - w1 + T, ih, -0.5f)) - 1);
            j1 = min(n - 1, (int)floorf(fmaf(d1 + w1 + T, ih, -0.5f)) + 1);
            m0 = max(0, (int)ceilf(fmaf(d2 - w2 + T, ih, -0.5f)) - 1);
            m1 = min(n - 1, (int)floorf(fmaf(d2 + w2 + T, ih, -0.5f)) + 1);
        }
    }
    if (__any_sync(FDX_FULL_MASK, degenerate)) j0 = 0, j1 = n - 1, m0 = 0, m1 = n - 1;
    const int J0 = __reduce_min_sync(FDX_FULL_MASK, j0), J1 = __reduce_max_sync(FDX_FULL_MASK, j1);
    const int M0 = __reduce_min_sync(FDX_FULL_MASK, m0), M1 = __reduce_max_sync(FDX_FULL_MASK, m1);
    if (J0 > J1 || M0 > M1) return false;

    float tau[PPL][3];
#pragma unroll
    for (int p = 0; p < PPL; ++p)
#pragma unroll
        for (int i = 0; i < 3; ++i) tau[p][i] = qp.tau[p][i];
    float st[PPL][3], ct[PPL][3];
    if (LS == FDX_LINESHAPE_HOSEMANN && MODE != MODE_CNT) {
#pragma unroll
        for (int p = 0; p < PPL; ++p)
#pragma unroll
            for (int i = 0; i < 3; ++i) sincospi_f(tau[p][i], st[p][i], ct[p][i]);
    }
    float la[3], tm[3], slb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) la[i] = rec[REC_LA + i], tm[i] = rec[REC_TM + i], slb[i] = rec[REC_SLB + i];
    const float hh[3] = {rec[REC_H], rec[REC_H + 1], rec[REC_H + 2]};
    const float E1[3] = {rec[REC_E1], rec[REC_E1 + 1], rec[REC_E1 + 2]};
    const float E2[3] = {rec[REC_E2], rec[REC_E2 + 1], rec[REC_E2 + 2]};

    // (p_ref - D)/r0 in the local frame, float-float
    const ff dP[3] = {qp.dP[0], qp.dP[1], qp.dP[2]};

    // warp-wide tau box: a node can be in some pixel's support only if sigma_i
    // lies within [min tau_i - tm_i, max tau_i + tm_i] for every i
    float tc[3], th[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float lo = 3.0e38f, hi = -3.0e38f;
#pragma unroll
        for (int p = 0; p < PPL; ++p)
            if (qp.valid[p]) lo = fminf(lo, tau[p][i]), hi = fmaxf(hi, tau[p][i]);
        lo = warp_min(lo), hi = warp_max(hi);
        tc[i] = 0.5f * (lo + hi);
        th[i] = 0.5f * (hi - lo) + tm[i] + 1e-5f;
    }
    const int nrows = J1 - J0 + 1, ncols = M1 - M0 + 1;
    // Block culling: the bounding box is cut into BR x BC-node blocks (32
    // nodes, the shape a tuning knob); a block is skipped when, at its centre,
    // sigma_i is farther from the warp's tau window than |a_i| r0 rho_b, rho_b
    // being the block's half-diagonal in the gnomonic plane (|d s / d d| <= r0,
    // so sigma_i varies by at most that).
    const int lr = P.blk_lr, lc = P.blk_lc, BR = 1 << lr, BC = 1 << lc;
    const int nbr = (nrows + BR - 1) >> lr, nbc = (ncols + BC - 1) >> lc, nblk = nbr * nbc;
    const float hgrid = 1.0f / P.inv_h;
    const float rho_b = hgrid * sqrtf(0.25f * (float)((BR - 1) * (BR - 1) + (BC - 1) * (BC - 1)));
    // (the block centres are evaluated in plain FP32 with an approximate rsqrt:
    // an error of a few 1e-7 in u, times the coefficients of sigma, is added)
    float bw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        bw[i] = th[i] + rec[REC_AR0 + i] * rho_b + 1e-4f + 1e-6f * (fabsf(hh[i]) + fabsf(E1[i]) + fabsf(E2[i]));
    // block index -> (row, column) without an integer division: blk < 2^13
    // and the quotient's fractional part is at least 0.5 / nbc from an integer
    const float inv_nbc = rcp_approx((float)nbc);
    const unsigned lt_mask = (1u << lane) - 1u;
    const int bj_lane = lane >> lc, bm_lane = lane & (BC - 1);  // this lane's node inside a block
    // staged counts: nr = rim nodes (all nodes when not PACKED), nc = core nodes
    int nr = 0, nc = 0;
    constexpr int NBH = NB / 2;                  // slots per list (PACKED)
    // core/rim split in both the forward and the adjoint (Hosemann).  The
    // adjoint's global gradients are differences of nearly equal sums over
    // reflections, so their FP32 rounding depends on the walk order; with the
    // split and 128-pair chunks the largest relative error against the FP64
    // adjoint on the seeded test models is 4e-5 (2.9e-5 without the split).
    constexpr bool SPLIT = PACKED;
    constexpr int RIM0 = SPLIT ? NBH : 0;        // first rim slot
    constexpr int RIM_CAP = SPLIT ? NBH : NB;
    static_assert(NB % 4 == 0, "node buffer must hold an even number of pairs per list");
    // core half-widths: |sigma_i - tc_i| <= ch_i puts the node inside every valid pixel's support
    float ch[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ch[i] = tm[i] - (th[i] - tm[i]) - 4e-5f;

    // Walk the compacted nodes (warp-uniform bounds) and empty the buffer.
    auto flush_scalar = [&]() {
        __syncwarp();
        for (int q0 = 0; q0 < nr; q0 += 32) {
            const int qe = min(q0 + 32, nr);
            float r0[PPL];
#pragma unroll
            for (int p = 0; p < PPL; ++p) r0[p] = 0.0f;
            // adjoint: the lane's points weighted by cw, six sums (absolute lineshapes)
            float x0 = 0.f, xa = 0.f, xb = 0.f, xc = 0.f, xs = 0.f, xg = 0.f;
#pragma unroll 2
            for (int q = q0; q < qe; ++q) {
                const float4 nq = buf[q];
#pragma unroll
                for (int p = 0; p < PPL; ++p) {
                    const float ta = tau[p][0] - nq.x, tb = tau[p][1] - nq.y, tcc = tau[p][2] - nq.z;
                    const bool in = (fabsf(ta) <= tm[0]) & (fabsf(tb) <= tm[1]) & (fabsf(tcc) <= tm[2]);
                    if (MODE == MODE_CNT) {
                        acc[p].cnt += in ? 1 : 0;
                    } else if (MODE == MODE_ADJ) {
                        if (in) {
                            float Ka, Kb, Kc, dKa, dKb, dKc;
                            if (LS == FDX_LINESHAPE_GAUSS) {
                                gauss_k_dk(ta, la[0], rec[REC_BETA], Ka, dKa);
                                gauss_k_dk(tb, la[1], rec[REC_BETA + 1], Kb, dKb);
                                gauss_k_dk(tcc, la[2], rec[REC_BETA + 2], Kc, dKc);
                            } else {
                                sinc_k_dk(ta, la[0], Ka, dKa);
                                sinc_k_dk(tb, la[1], Kb, dKb);
                                sinc_k_dk(tcc, la[2], Kc, dKc);
                            }
                            const float2 dw = reinterpret_cast<const float2 *>(buf2)[q];
                            const float c = qp.cw[p];
                            const float kbc = Kb * Kc, kp = Ka * kbc;
                            x0 = fmaf(c * nq.w, kp, x0);
                            xa = fmaf(c * nq.w, dKa * kbc, xa);
                            xb = fmaf(c * nq.w, Ka * dKb * Kc, xb);
                            xc = fmaf(c * nq.w, Ka * Kb * dKc, xc);
                            xs = fmaf(c * dw.x, kp, xs);
                            xg = fmaf(c * dw.y, kp, xg);
                        }
                    } else {
                        const float kv =
                            nq.w * (LS == FDX_LINESHAPE_GAUSS ? gauss_term(ta, tb, tcc, la) : sinc_term(ta, tb, tcc, la));
                        r0[p] += in ? kv : 0.0f;
                    }
                }
            }
            if (MODE == MODE_ADJ) {
                acc[0].s0 = ff_add_f(acc[0].s0, x0);
                acc[0].sb[0] = ff_add_f(acc[0].sb[0], xa);
                acc[0].sb[1] = ff_add_f(acc[0].sb[1], xb);
                acc[0].sb[2] = ff_add_f(acc[0].sb[2], xc);
                acc[0].ss = ff_add_f(acc[0].ss, xs);
                acc[0].sg = ff_add_f(acc[0].sg, xg);
            } else if (MODE != MODE_CNT) {
#pragma unroll
                for (int p = 0; p < PPL; ++p) acc[p].s0 = ff_add_f(acc[p].s0, r0[p]);
            }
        }
        nr = 0;
        __syncwarp();
    };

    // Hosemann walk on node pairs.  Per pixel and pair: t = tau - sigma (support
    // test), scaled sin(pi t) = sin(pi tau) C - cos(pi tau) S, den_i = beta_i^2 +
    // (scaled sin)^2, 1/prod den by one SFU reciprocal (the adjoint takes two:
    // 1/den_a and 1/(den_b den_c)); a node outside the pixel's support gets the
    // reciprocal of +inf, i.e. weight 0.
    float2 tau2[PPL][3], st2[PPL][3], ctn2[PPL][3], la2[3];
    if (PACKED) {
#pragma unroll
        for (int p = 0; p < PPL; ++p)
#pragma unroll
            for (int i = 0; i < 3; ++i) tau2[p][i] = f2(tau[p][i]), st2[p][i] = f2(st[p][i]), ctn2[p][i] = f2(-ct[p][i]);
#pragma unroll
        for (int i = 0; i < 3; ++i) la2[i] = f2(la[i]);
    }
    const float inf = __int_as_float(0x7f800000);
    // rearrange n staged nodes at slots [base, base + n) into pairs, 32 nodes
    // (16 pairs) at a time; a pair never straddles two such groups, so reading
    // the group before writing it is enough.  Padding node (odd n): weight 0,
    // and for the rim list far outside every support.
    auto pack_node = [&](int base, int n, bool rim) {
        float *bf = reinterpret_cast<float *>(buf);
        float *bs = reinterpret_cast<float *>(bsc);
        float *be = reinterpret_cast<float *>(bsc2);
        float *bd = reinterpret_cast<float *>(buf2);
        const int npad = (n + 1) & ~1;
        for (int q0 = 0; q0 < npad; q0 += 32) {
            const int q = q0 + lane;
            float4 nq = rim ? make_float4(-3.0e4f, -3.0e4f, -3.0e4f, 0.0f) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float2 dw = make_float2(0.0f, 0.0f);
            if (q < n && FDX_IN_BOUNDS(base + q, NB, DBG_PACK)) {
                nq = buf[base + q];
                if (MODE == MODE_ADJ) dw = reinterpret_cast<const float2 *>(buf2)[base + q];
            }
            __syncwarp();
            if (q < npad && FDX_IN_BOUNDS((base >> 1) + (q >> 1), NB / 2, DBG_PACK)) {
                float2 sab, cab;
                float sc, cc;
                sincospi_f2(make_float2(nq.x, nq.y), sab, cab);  // axes a, b on packed pairs
                sincospi_f(nq.z, sc, cc);
                const float sa = sab.x, ca = cab.x, sb = sab.y, cb = cab.y;
                const int u = (base >> 1) + (q >> 1), o = q & 1;
                bf[8 * u + o] = -nq.x, bf[8 * u + 2 + o] = -nq.y, bf[8 * u + 4 + o] = -nq.z, bf[8 * u + 6 + o] = nq.w;
                bs[8 * u + o] = slb[0] * ca, bs[8 * u + 2 + o] = slb[0] * sa;
                bs[8 * u + 4 + o] = slb[1] * cb, bs[8 * u + 6 + o] = slb[1] * sb;
                be[4 * u + o] = slb[2] * cc, be[4 * u + 2 + o] = slb[2] * sc;
                if (MODE == MODE_ADJ) bd[4 * u + o] = dw.x, bd[4 * u + 2 + o] = dw.y;
            }
            __syncwarp();
        }
    };
    // The same rearrangement with one pair per lane: lane k reads nodes 2k and
    // 2k + 1 of the list and writes the packed pair into the same two slots,
    // so no lane touches another's slots.  Fewer instructions per node, but
    // 32-byte-strided shared-memory accesses and half as many busy lanes: it
    // pays only with one point per lane, where staging weighs more.
    auto pack_pair = [&](int base, int n, bool rim) {
        const int npair = (n + 1) >> 1;
        for (int k = lane; k < npair; k += 32) {
            if (!FDX_IN_BOUNDS((base >> 1) + k, NB / 2, DBG_PACK)) continue;
            const float4 pad = rim ? make_float4(-3.0e4f, -3.0e4f, -3.0e4f, 0.0f) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const float4 n0 = buf[base + 2 * k];
            const float4 n1 = 2 * k + 1 < n ? buf[base + 2 * k + 1] : pad;
            float4 dw = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (MODE == MODE_ADJ) {
                const float2 d0 = reinterpret_cast<const float2 *>(buf2)[base + 2 * k];
                const float2 d1 =
                    2 * k + 1 < n ? reinterpret_cast<const float2 *>(buf2)[base + 2 * k + 1] : make_float2(0.0f, 0.0f);
                dw = make_float4(d0.x, d1.x, d0.y, d1.y);
            }
            float2 sa, ca, sb, cb, sc, cc;
            sincospi_f2(make_float2(n0.x, n1.x), sa, ca);
            sincospi_f2(make_float2(n0.y, n1.y), sb, cb);
            sincospi_f2(make_float2(n0.z, n1.z), sc, cc);
            const int u = (base >> 1) + k;
            buf[2 * u] = make_float4(-n0.x, -n1.x, -n0.y, -n1.y);
            buf[2 * u + 1] = make_float4(-n0.z, -n1.z, n0.w, n1.w);
            const float2 Ca = __fmul2_rn(f2(slb[0]), ca), Sa = __fmul2_rn(f2(slb[0]), sa);
            const float2 Cb = __fmul2_rn(f2(slb[1]), cb), Sb = __fmul2_rn(f2(slb[1]), sb);
            const float2 Cc = __fmul2_rn(f2(slb[2]), cc), Sc = __fmul2_rn(f2(slb[2]), sc);
            bsc[2 * u] = make_float4(Ca.x, Ca.y, Sa.x, Sa.y);
            bsc[2 * u + 1] = make_float4(Cb.x, Cb.y, Sb.x, Sb.y);
            bsc2[u] = make_float4(Cc.x, Cc.y, Sc.x, Sc.y);
            if (MODE == MODE_ADJ) buf2[u] = dw;
        }
        __syncwarp();
    };
    auto pack = [&](int base, int n, bool rim) {
        if constexpr (PPL == 1)
            pack_pair(base, n, rim);
        else
            pack_node(base, n, rim);
    };
    // walk npair pairs from pair slot ub; TEST: per-pixel support test (rim list)
    auto walk = [&](int ub, int npair, auto test_tag) {
        constexpr bool TEST = decltype(test_tag)::value;
        constexpr int CH = MODE == MODE_ADJ ? 128 : 32;  // node pairs per FP32 chunk sum (the adjoint folds six)
        for (int u0 = 0; u0 < npair; u0 += CH) {
            const int ue = ub + min(u0 + CH, npair);
            float2 r0[PPL], rb0[PPL], rb1[PPL], rb2[PPL], rss[PPL], rsg[PPL];
#pragma unroll
            for (int p = 0; p < PPL; ++p) r0[p] = rb0[p] = rb1[p] = rb2[p] = rss[p] = rsg[p] = f2(0.0f);
#pragma unroll 2
            for (int u = ub + u0; u < ue; ++u) {
                if (!FDX_IN_BOUNDS(u, NB / 2, DBG_WALK)) continue;
                const float4 A4 = buf[2 * u], B4 = buf[2 * u + 1];
                const float4 C4 = bsc[2 * u], D4 = bsc[2 * u + 1], E4 = bsc2[u];
                float4 W4;
                if (MODE == MODE_ADJ) W4 = buf2[u];
                const float2 nsa = make_float2(A4.x, A4.y), nsb = make_float2(A4.z, A4.w);
                const float2 nsc = make_float2(B4.x, B4.y), w = make_float2(B4.z, B4.w);
                const float2 Ca = make_float2(C4.x, C4.y), Sa = make_float2(C4.z, C4.w);
                const float2 Cb = make_float2(D4.x, D4.y), Sb = make_float2(D4.z, D4.w);
                const float2 Cc = make_float2(E4.x, E4.y), Sc = make_float2(E4.z, E4.w);
#pragma unroll
                for (int p = 0; p < PPL; ++p) {
                    const float2 xa = __ffma2_rn(st2[p][0], Ca, __fmul2_rn(ctn2[p][0], Sa));
                    const float2 xb = __ffma2_rn(st2[p][1], Cb, __fmul2_rn(ctn2[p][1], Sb));
                    const float2 xc = __ffma2_rn(st2[p][2], Cc, __fmul2_rn(ctn2[p][2], Sc));
                    const float2 da = __ffma2_rn(xa, xa, la2[0]);
                    const float2 db = __ffma2_rn(xb, xb, la2[1]);
                    const float2 dc = __ffma2_rn(xc, xc, la2[2]);
                    if constexpr (MODE == MODE_ADJ) {
                        // two reciprocals per node, ra = 1/den_a and rbc = 1/(den_b den_c):
                        // 1/prod den = ra rbc, and the three kv/den_i are kv ra,
                        // (kv rbc) den_c and (kv rbc) den_b -- two packed products fewer
                        // than dividing by the full product, for one more SFU operation
                        const float2 dbc = __fmul2_rn(db, dc);
                        float2 ra;
                        if constexpr (TEST) {
                            const float2 ta = __fadd2_rn(tau2[p][0], nsa);
                            const float2 tb = __fadd2_rn(tau2[p][1], nsb);
                            const float2 tc2 = __fadd2_rn(tau2[p][2], nsc);
                            ra = make_float2(rcp_approx(support_sel(ta.x, tb.x, tc2.x, tm[0], tm[1], tm[2], da.x, inf)),
                                             rcp_approx(support_sel(ta.y, tb.y, tc2.y, tm[0], tm[1], tm[2], da.y, inf)));
                        } else {
                            ra = make_float2(rcp_approx(da.x), rcp_approx(da.y));
                        }
                        const float2 rbc = make_float2(rcp_approx(dbc.x), rcp_approx(dbc.y));
                        const float2 rp = __fmul2_rn(ra, rbc);
                        const float2 kv = __fmul2_rn(w, rp);
                        r0[p] = __fadd2_rn(r0[p], kv);
                        rb0[p] = __ffma2_rn(kv, ra, rb0[p]);
                        const float2 q = __fmul2_rn(kv, rbc);
                        rb1[p] = __ffma2_rn(q, dc, rb1[p]);
                        rb2[p] = __ffma2_rn(q, db, rb2[p]);
                        rss[p] = __ffma2_rn(make_float2(W4.x, W4.y), rp, rss[p]);
                        rsg[p] = __ffma2_rn(make_float2(W4.z, W4.w), rp, rsg[p]);
                        continue;
                    }
                    const float2 dab = __fmul2_rn(da, db);
                    const float2 d = __fmul2_rn(dab, dc);
                    float2 rp;
                    if constexpr (TEST) {
                        const float2 ta = __fadd2_rn(tau2[p][0], nsa);
                        const float2 tb = __fadd2_rn(tau2[p][1], nsb);
                        const float2 tc2 = __fadd2_rn(tau2[p][2], nsc);
                        rp = make_float2(rcp_approx(support_sel(ta.x, tb.x, tc2.x, tm[0], tm[1], tm[2], d.x, inf)),
                                         rcp_approx(support_sel(ta.y, tb.y, tc2.y, tm[0], tm[1], tm[2], d.y, inf)));
                    } else {
                        rp = make_float2(rcp_approx(d.x), rcp_approx(d.y));
                    }
                    r0[p] = __ffma2_rn(w, rp, r0[p]);
                }
            }
            if (MODE == MODE_ADJ) {
                // adjoint: the lane's points weighted by cw, into one accumulator
                float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f, x4 = 0.f, x5 = 0.f;
#pragma unroll
                for (int p = 0; p < PPL; ++p) {
                    const float c = qp.cw[p];
                    x0 = fmaf(c, r0[p].x + r0[p].y, x0);
                    x1 = fmaf(c, rb0[p].x + rb0[p].y, x1);
                    x2 = fmaf(c, rb1[p].x + rb1[p].y, x2);
                    x3 = fmaf(c, rb2[p].x + rb2[p].y, x3);
                    x4 = fmaf(c, rss[p].x + rss[p].y, x4);
                    x5 = fmaf(c, rsg[p].x + rsg[p].y, x5);
                }
                acc[0].s0 = ff_add_f(acc[0].s0, x0);
                acc[0].sb[0] = ff_add_f(acc[0].sb[0], x1);
                acc[0].sb[1] = ff_add_f(acc[0].sb[1], x2);
                acc[0].sb[2] = ff_add_f(acc[0].sb[2], x3);
                acc[0].ss = ff_add_f(acc[0].ss, x4);
                acc[0].sg = ff_add_f(acc[0].sg, x5);
            } else {
#pragma unroll
                for (int p = 0; p < PPL; ++p) acc[p].s0 = ff_add_f(acc[p].s0, r0[p].x + r0[p].y);
            }
        }
    };
    auto flush_packed = [&]() {
        __syncwarp();
        if (SPLIT) {
            pack(0, nc, false);
            walk(0, (nc + 1) >> 1, std::integral_constant<bool, false>{});
        }
        pack(RIM0, nr, true);
        walk(RIM0 / 2, (nr + 1) >> 1, std::integral_constant<bool, true>{});
        nc = nr = 0;
        __syncwarp();
    };
    auto flush = [&]() {
        if constexpr (PACKED)
            flush_packed();
        else
            flush_scalar();
    };

    for (int blk0 = 0; blk0 < nblk; blk0 += 32) {
        bool blive = false;
        {
            const int blk = blk0 + lane;
            if (blk < nblk) {
                const int bj = (int)(((float)blk + 0.5f) * inv_nbc), bm = blk - bj * nbc;
                const float d1 = -P.T + (J0 + bj * BR + 0.5f * (BR - 1) + 0.5f) * hgrid;
                const float d2 = -P.T + (M0 + bm * BC + 0.5f * (BC - 1) + 0.5f) * hgrid;
                const float c = rsqrtf(1.0f + fmaf(d1, d1, d2 * d2));
                const float u0 = (c - 1.0f) - dP[0].hi;
                const float u1 = d1 * c - dP[1].hi, u2 = d2 * c - dP[2].hi;
                blive = true;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float sgc = fmaf(hh[i], u0, fmaf(E1[i], u1, E2[i] * u2));
                    blive &= fabsf(sgc - tc[i]) <= bw[i];
                }
            }
        }
        unsigned bmask = __ballot_sync(FDX_FULL_MASK, blive);
        // The live blocks of this round one after another; the node entries of
        // the next live block are loaded while the current one is staged.
        // Every lane loads an entry of the grid (clamped into it); lanes whose
        // node lies outside the bounding box drop theirs.
        auto node_of = [&](int blk, int &jj, int &mm) {
            const int bj = (int)(((float)blk + 0.5f) * inv_nbc), bm = blk - bj * nbc;
            jj = J0 + bj * BR + bj_lane, mm = M0 + bm * BC + bm_lane;
        };
        int jc = 0, mc = 0;
        float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na;
        float2 dn = make_float2(0.f, 0.f);
        bool have = bmask != 0;
        if (have) {
            node_of(blk0 + __ffs(bmask) - 1, jc, mc);
            bmask &= bmask - 1;
            const size_t k = (size_t)min(jc, J1) * n + min(mc, M1);
            if (FDX_IN_BOUNDS(k, (long long)n * n, DBG_NODES)) {
                na = P.nodes[2 * k], nb = P.nodes[2 * k + 1];
                if (MODE == MODE_ADJ) dn = P.dnodes[k];
            }
        }
        while (have) {
            int jn = 0, mn = 0;
            float4 na2 = make_float4(0.f, 0.f, 0.f, 0.f), nb2 = na2;
            float2 dn2 = make_float2(0.f, 0.f);
            const bool more = bmask != 0;
            if (more) {
                node_of(blk0 + __ffs(bmask) - 1, jn, mn);
                bmask &= bmask - 1;
                const size_t k = (size_t)min(jn, J1) * n + min(mn, M1);
                if (FDX_IN_BOUNDS(k, (long long)n * n, DBG_NODES)) {
                    na2 = P.nodes[2 * k], nb2 = P.nodes[2 * k + 1];
                    if (MODE == MODE_ADJ) dn2 = P.dnodes[k];
                }
            }
            bool live = false;
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            if (jc <= J1 && mc <= M1) {
                // u = s_k/r0 - p_ref/r0 in the local frame = (c - 1, c d1, c d2) - dP
                const float u0 = (na.x - dP[0].hi) + (na.y - dP[0].lo);
                const float u1 = (na.z - dP[1].hi) + (na.w - dP[1].lo);
                const float u2 = (nb.x - dP[2].hi) + (nb.y - dP[2].lo);
                float sg[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) sg[i] = fmaf(hh[i], u0, fmaf(E1[i], u1, E2[i] * u2));
                live = (fabsf(sg[0] - tc[0]) <= th[0]) & (fabsf(sg[1] - tc[1]) <= th[1]) &
                       (fabsf(sg[2] - tc[2]) <= th[2]);
                val = make_float4(sg[0], sg[1], sg[2], nb.z);
            }
            bool core = false;
            if (SPLIT)
                core = live & (fabsf(val.x - tc[0]) <= ch[0]) & (fabsf(val.y - tc[1]) <= ch[1]) &
                       (fabsf(val.z - tc[2]) <= ch[2]);
            const unsigned bal = __ballot_sync(FDX_FULL_MASK, live & !core);
            const unsigned balc = SPLIT ? __ballot_sync(FDX_FULL_MASK, core) : 0u;
            if (live) {
                const int pos = core ? nc + __popc(balc & lt_mask) : RIM0 + nr + __popc(bal & lt_mask);
                if (FDX_IN_BOUNDS(pos, NB, DBG_STAGE)) {
                    buf[pos] = val;
                    if (MODE == MODE_ADJ) reinterpret_cast<float2 *>(buf2)[pos] = dn;
                }
            }
            nr += __popc(bal);
            nc += __popc(balc);
            if (nr > RIM_CAP - 32 || nc > NBH - 32) flush();
            have = more, jc = jn, mc = mn, na = na2, nb = nb2, dn = dn2;
        }
    }
    if (nr > 0 || nc > 0) flush();
    return true;
}

// The pair (pixel patch, reflection) of the gather form.
template <int LS, int MODE, int NB, int PPL>
__device__ __forceinline__ bool eval_pair(const PatternParams &P, const PatchPix<PPL> &g, const float *rec,
                                          float4 *buf, float4 *buf2, float4 *bsc, float4 *bsc2, int lane,
                                          PairAcc (&acc)[PPL]) {
    return eval_core<LS, MODE, NB, PPL>(P, pixel_queries<PPL>(P, g, rec), rec, buf, buf2, bsc, bsc2, lane, acc);
}

// Copy a 64-float reflection record into the warp's shared slot.
__device__ __forceinline__ void load_record(const float *recs, int r, float *rec, int lane) {
    const float *grec = recs + (size_t)r * REC_SIZE;
    __syncwarp();
    rec[lane] = grec[lane];
    rec[lane + 32] = grec[lane + 32];
    __syncwarp();
}

}  // namespace fdx
