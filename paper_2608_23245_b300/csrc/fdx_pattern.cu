// Gather-form pattern kernel (Eq. direct_sum at every pixel's query point,
// times the Lorentz factor of Eq. lorentz).
//
// Work decomposition.  A CTA of 4 warps covers a 16 x 8 pixel block; each warp
// owns an 8 x 4 pixel patch, one pixel per lane, and accumulates its pixels in
// registers (no atomics).  The warp scans the reflection list 32 at a time
// with a conservative radial/polar test against its patch's (|S|, psi) bounds
// and processes the survivors in list order (deterministic).  For a surviving
// reflection each lane projects the 8 corners of its support box onto the
// gnomonic plane, which bounds the node rows/columns that can be in support;
// the warp takes the union.  For the nodes of that union the warp computes,
// one node per lane, sigma_i(k) = a_i . (s_k - p_ref) (p_ref = the query point
// of lane 0's pixel) with float-float differences so that the small offsets
// survive FP32 rounding, and keeps only the nodes that can lie in the support
// of some lane of the warp (sigma_i within the warp's range of tau_i widened
// by the support half-width); the survivors are compacted into the warp's
// shared-memory buffer.  Every lane then walks the buffer with warp-uniform
// bounds: t_i = tau_i - sigma_i, where tau_i = a_i . (p - p_ref) is the lane's
// own small offset, tests the support and accumulates w_k prod_i K_i(t_i).
// Sums of 32 nodes are folded into a float-float pair sum, pair sums into a
// float-float pixel sum.
#include "fdx_internal.cuh"

namespace fdx {

static constexpr int WARPS = 4;
static constexpr int NODE_BUF = 512;  // staged nodes per warp (float4 each)

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

// Hosemann denominators: den_i = beta_i^2 + (1 - beta_i^2) sin^2(pi t_i), with
// sin^2(pi t) = x Q(x), x = t^2, folded into one degree-6 polynomial in x whose
// coefficients cf[i][.] are scaled per reflection.  K_i = beta_i / den_i; the
// product of the beta_i is in the pair factor.
__device__ __forceinline__ float hosemann_den(float t, const float (&c)[7]) {
    const float x = t * t;
    float d = c[6];
#pragma unroll
    for (int k = 5; k >= 0; --k) d = fmaf(d, x, c[k]);
    return d;
}

// Sinc lineshape: K_i = N_i sinc^2(N_i t_i); with x = N t, y = x - rint(x):
// sinc^2(x) = Q(y^2) (y^2 / x^2) / pi^2, the ratio being 1 when rint(x) = 0.
// prod N_i / pi^6 is in the pair factor.
__device__ __forceinline__ float sinc_term(float ta, float tb, float tc, const float *la) {
    const float Qc[6] = FDX_SINPI2_C;
    float num = 1.0f, den = 1.0f, q = 1.0f;
    const float tt[3] = {ta, tb, tc};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float x = la[i] * tt[i];
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

template <int LS, bool COUNT>
__global__ void __launch_bounds__(WARPS * 32, 4) pattern_kernel(PatternParams P) {
    __shared__ float4 s_nodes[WARPS][NODE_BUF];
    __shared__ float s_rec[WARPS][REC_SIZE];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px0 = blockIdx.x * 16 + (warp & 1) * 8, py0 = blockIdx.y * 8 + (warp >> 1) * 4;
    const int px = px0 + (lane & 7), py = py0 + (lane >> 3);
    const bool valid = (px < P.nx) && (py < P.ny);
    if (__ballot_sync(FDX_FULL_MASK, valid) == 0) return;  // lane 0 is valid from here on

    const size_t pidx = valid ? (size_t)py * P.nx + px : (size_t)py0 * P.nx + px0;
    const float4 g = P.pixgeo[pidx];
    const float Rh = g.x, Rl = g.y, Zh = g.z, Zl = g.w;
    const float Rrh = __shfl_sync(FDX_FULL_MASK, Rh, 0), Rrl = __shfl_sync(FDX_FULL_MASK, Rl, 0);
    const float Zrh = __shfl_sync(FDX_FULL_MASK, Zh, 0), Zrl = __shfl_sync(FDX_FULL_MASK, Zl, 0);
    // offset of this pixel's (R, Z) from the reference pixel (exactly small)
    const float dRl = (Rh - Rrh) + (Rl - Rrl);
    const float dZl = (Zh - Zrh) + (Zl - Zrl);

    const float rlen = sqrtf(Rh * Rh + Zh * Zh), psi = atan2f(Rh, Zh);
    const float rmin = warp_min(valid ? rlen : 3.0e38f), rmax = warp_max(valid ? rlen : -3.0e38f);
    const float pmin = warp_min(valid ? psi : 3.0e38f), pmax = warp_max(valid ? psi : -3.0e38f);

    const int n = P.n_nodes;
    float *rec = s_rec[warp];
    float4 *buf = s_nodes[warp];
    ff acc = {0.0f, 0.0f};
    int32_t cnt = 0;

    for (int base = 0; base < P.n_refl; base += 32) {
        bool cand = false;
        const int rr = base + lane;
        if (rr < P.n_refl) {
            const float4 q = P.reach[rr];
            cand = (q.x - q.y <= rmax) && (q.x + q.y >= rmin) && (q.z - q.w <= pmax) && (q.z + q.w >= pmin);
        }
        unsigned mask = __ballot_sync(FDX_FULL_MASK, cand);
        while (mask) {
            const int b = __ffs(mask) - 1;
            mask &= mask - 1;
            const float *grec = P.recs + (size_t)(base + b) * REC_SIZE;
            __syncwarp();
            rec[lane] = grec[lane];
            rec[lane + 32] = grec[lane + 32];
            __syncwarp();

            // (p - D)/r0 in the local frame, FP32 (only bounds the node range)
            const float dZ = (Zh - rec[REC_ZD]) + (Zl - rec[REC_ZD + 1]);
            const float dR = (Rh - rec[REC_RD]) + (Rl - rec[REC_RD + 1]);
            const float P0 = fmaf(dZ, rec[REC_NFR], dR * rec[REC_EFR]);
            const float P1 = fmaf(dZ, rec[REC_NFR + 1], dR * rec[REC_EFR + 1]);
            const float P2 = fmaf(dZ, rec[REC_NFR + 2], dR * rec[REC_EFR + 2]);
            float d1lo = 3.0e38f, d1hi = -3.0e38f, d2lo = 3.0e38f, d2hi = -3.0e38f;
            bool degenerate = false;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const float sg = s ? -1.0f : 1.0f;
                    const float X0 = 1.0f + P0 + sg * rec[REC_CR + 3 * v];
                    const float X1 = P1 + sg * rec[REC_CR + 3 * v + 1];
                    const float X2 = P2 + sg * rec[REC_CR + 3 * v + 2];
                    degenerate |= !(X0 > 0.05f);
                    const float inv = 1.0f / X0;
                    const float d1 = X1 * inv, d2 = X2 * inv;
                    d1lo = fminf(d1lo, d1), d1hi = fmaxf(d1hi, d1);
                    d2lo = fminf(d2lo, d2), d2hi = fmaxf(d2hi, d2);
                }
            }
            int j0 = n, j1 = -1, m0 = n, m1 = -1;
            if (valid) {
                if (degenerate) {
                    j0 = 0, j1 = n - 1, m0 = 0, m1 = n - 1;
                } else {
                    const float T = P.T, ih = P.inv_h;
                    j0 = max(0, (int)ceilf(fmaf(d1lo + T, ih, -0.5f)) - 1);
                    j1 = min(n - 1, (int)floorf(fmaf(d1hi + T, ih, -0.5f)) + 1);
                    m0 = max(0, (int)ceilf(fmaf(d2lo + T, ih, -0.5f)) - 1);
                    m1 = min(n - 1, (int)floorf(fmaf(d2hi + T, ih, -0.5f)) + 1);
                }
            }
            const int J0 = __reduce_min_sync(FDX_FULL_MASK, j0), J1 = __reduce_max_sync(FDX_FULL_MASK, j1);
            const int M0 = __reduce_min_sync(FDX_FULL_MASK, m0), M1 = __reduce_max_sync(FDX_FULL_MASK, m1);
            if (J0 > J1 || M0 > M1) continue;

            // tau_i = a_i . (p - p_ref), small
            float tau[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) tau[i] = valid ? fmaf(dZl, P.AZ[i], dRl * rec[REC_AR + i]) : 3.0e30f;
            float la[3], tm[3], cf[3][7];
            {
                const float Qc[6] = FDX_SINPI2_C;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    la[i] = rec[REC_LA + i], tm[i] = rec[REC_TM + i];
                    const float lb = rec[REC_LB + i];
                    cf[i][0] = la[i];
#pragma unroll
                    for (int k = 1; k < 7; ++k) cf[i][k] = lb * Qc[k - 1];
                }
            }
            const float hh[3] = {rec[REC_H], rec[REC_H + 1], rec[REC_H + 2]};
            const float E1[3] = {rec[REC_E1], rec[REC_E1 + 1], rec[REC_E1 + 2]};
            const float E2[3] = {rec[REC_E2], rec[REC_E2 + 1], rec[REC_E2 + 2]};

            // (p_ref - D)/r0 in the local frame, float-float (all lanes compute it for lane 0's pixel)
            const ff dZr = ff_add(two_sum(Zrh, -rec[REC_ZD]), ff{Zrl, -rec[REC_ZD + 1]});
            const ff dRr = ff_add(two_sum(Rrh, -rec[REC_RD]), ff{Rrl, -rec[REC_RD + 1]});
            ff dP[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                dP[q] = ff_add(ff_mul(dZr, ff{rec[REC_NFR + q], rec[REC_NFR + 3 + q]}),
                               ff_mul(dRr, ff{rec[REC_EFR + q], rec[REC_EFR + 3 + q]}));
            }

            // Warp-wide tau box: a node can be in the support of some lane only if
            // sigma_i lies within [min tau_i - tm_i, max tau_i + tm_i] for every i.
            float tc[3], th[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float lo = warp_min(valid ? tau[i] : 3.0e38f), hi = warp_max(valid ? tau[i] : -3.0e38f);
                tc[i] = 0.5f * (lo + hi);
                th[i] = 0.5f * (hi - lo) + tm[i] + 1e-5f;
            }
            const int ncols = M1 - M0 + 1;
            const int total = (J1 - J0 + 1) * ncols;
            const unsigned lt_mask = (1u << lane) - 1u;
            const int step_r = 32 / ncols, step_c = 32 - step_r * ncols;
            int jj = J0 + lane / ncols, mm = M0 + lane % ncols;  // this lane's node in the batch
            ff pair = {0.0f, 0.0f};
            int nlive = 0;
            for (int b0 = 0; b0 < total; b0 += 32) {
                // stage: one node per lane, keep it if it passes the warp-wide test
                const int idx = b0 + lane;
                bool live = false;
                float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
                if (idx < total) {
                    const size_t k = (size_t)jj * n + mm;
                    const float4 na = P.nodes[2 * k], nb = P.nodes[2 * k + 1];
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
                jj += step_r, mm += step_c;
                if (mm > M1) mm -= ncols, ++jj;
                const unsigned bal = __ballot_sync(FDX_FULL_MASK, live);
                if (live) buf[nlive + __popc(bal & lt_mask)] = val;
                nlive += __popc(bal);
                if (nlive > NODE_BUF - 32 || (b0 + 32 >= total && nlive > 0)) {
                    __syncwarp();
                    // walk the live nodes: 32 at a time into a row sum, then into the pair sum
                    for (int q0 = 0; q0 < nlive; q0 += 32) {
                        const int qe = min(q0 + 32, nlive);
                        float rs = 0.0f;
#pragma unroll 4
                        for (int q = q0; q < qe; ++q) {
                            const float4 nq = buf[q];
                            const float ta = tau[0] - nq.x, tb = tau[1] - nq.y, tcc = tau[2] - nq.z;
                            const bool in = (fabsf(ta) <= tm[0]) & (fabsf(tb) <= tm[1]) & (fabsf(tcc) <= tm[2]);
                            if (COUNT) {
                                cnt += in ? 1 : 0;
                            } else if (LS == FDX_LINESHAPE_HOSEMANN) {
                                const float d = hosemann_den(ta, cf[0]) * hosemann_den(tb, cf[1]) *
                                                hosemann_den(tcc, cf[2]);
                                const float kv = nq.w * rcp_approx(d);
                                rs += in ? kv : 0.0f;
                            } else {
                                const float kv = nq.w * sinc_term(ta, tb, tcc, la);
                                rs += in ? kv : 0.0f;
                            }
                        }
                        if (!COUNT) pair = ff_add_f(pair, rs);
                    }
                    nlive = 0;
                    __syncwarp();
                }
            }
            if (!COUNT) acc = ff_add(acc, ff_mul_f(pair, rec[REC_FR]));
        }
    }
    if (!valid) return;
    const size_t out = (size_t)py * P.nx + px;
    if (COUNT) {
        P.counts[out] = cnt;
    } else {
        const double R = (double)Rh + (double)Rl;
        const double L = P.delta_L / (R + P.delta_L);
        P.image[out] = (float)(L * ((double)acc.hi + (double)acc.lo));
    }
}

cudaError_t launch_pattern(const PatternParams &p, int lineshape, bool count_mode, cudaStream_t s) {
    dim3 grid((p.nx + 15) / 16, (p.ny + 7) / 8);
    dim3 block(WARPS * 32);
    if (lineshape == FDX_LINESHAPE_HOSEMANN) {
        if (count_mode)
            pattern_kernel<FDX_LINESHAPE_HOSEMANN, true><<<grid, block, 0, s>>>(p);
        else
            pattern_kernel<FDX_LINESHAPE_HOSEMANN, false><<<grid, block, 0, s>>>(p);
    } else {
        if (count_mode)
            pattern_kernel<FDX_LINESHAPE_SINC, true><<<grid, block, 0, s>>>(p);
        else
            pattern_kernel<FDX_LINESHAPE_SINC, false><<<grid, block, 0, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace fdx
