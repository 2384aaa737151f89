// Ring-integrated cylindrical average (Eq. cyl-average): the pixel value is
// the average of the reciprocal-space intensity over the ring of the pixel's
// (R, Z) about the fiber axis, with no Lorentz factor,
//   I = sum_hkl M r0^2 (1/2pi) int dphi sum_k w_k prod_i K_i(a_i . (p(phi) - s_k)),
//   p(phi) = Z n + R (cos(phi) e_R + sin(phi) e_P),  e_P = n x e_R,
// with phi measured from the reflection's meridional half-plane, by the
// per-reflection midpoint rule over [-Phi_r, Phi_r] (N_r points; window and
// step from the reflection set-up kernel, reading R21).
//
// Work decomposition: as the gather form, a warp owns an 8 x 8 pixel patch
// (two pixels per lane, rows 0-3 and 4-7, so that the packed walk has two
// query points per node pair) and scans the reflections with the reach test (the ring points of a pixel
// have its |S| and polar angle, so the test is exact for every azimuth); for
// each azimuth point of a surviving reflection the patch's query points are
// the pixels' ring points p(phi_j), evaluated by eval_core (block culling,
// staging, packed walk) against a reference at the patch's centre pixel.  The
// azimuth points' sin(phi_j) and 1 - cos(phi_j) are computed in FP64, 32 at a
// time (one per lane), and broadcast; points whose ring arc cannot reach the
// support for any pixel of the patch are skipped.  A small detector region has
// too few patches to fill the GPU, so the points of every reflection are dealt
// round-robin to n_split warps per patch (grid z); each writes a float-float
// partial image and a second kernel sums them in split order.
#include "fdx_pair.cuh"

namespace fdx {

static constexpr int RING_NODE_BUF = 288;

template <int LS, int MODE, int PPL>
__device__ __forceinline__ void ring_warp(const RingParams &RP, int px0, int py0, float4 *buf, float4 *bsc,
                                          float4 *bsc2, float *rec, int lane) {
    const PatternParams &P = RP.P;
    const PatchPix<PPL> g = load_patch<PPL>(P.pixgeo, P.nx, P.ny, px0, py0, lane);
    float rmin = 3.0e38f, rmax = -3.0e38f, pmin = 3.0e38f, pmax = -3.0e38f;
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        if (!g.valid[p]) continue;
        const float rlen = sqrtf(g.Rh[p] * g.Rh[p] + g.Zh[p] * g.Zh[p]), psi = atan2f(g.Rh[p], g.Zh[p]);
        rmin = fminf(rmin, rlen), rmax = fmaxf(rmax, rlen), pmin = fminf(pmin, psi), pmax = fmaxf(pmax, psi);
    }
    rmin = warp_min(rmin), rmax = warp_max(rmax), pmin = warp_min(pmin), pmax = warp_max(pmax);
    ff acc[PPL];
    int32_t cnt[PPL];
#pragma unroll
    for (int p = 0; p < PPL; ++p) acc[p] = ff{0.0f, 0.0f}, cnt[p] = 0;

    for (int base = 0; base < P.n_refl; base += 32) {
        bool cand = false;
        const int rr = base + lane;
        if (rr < P.n_refl) {
            const float4 q = P.reach[rr];
            const float dw = q.w + RP.dpsi_extra;  // ring points leave the meridional plane
            cand = (q.x - q.y <= rmax) && (q.x + q.y >= rmin) && (q.z - dw <= pmax) && (q.z + dw >= pmin);
        }
        unsigned mask = __ballot_sync(FDX_FULL_MASK, cand);
        while (mask) {
            const int b = __ffs(mask) - 1;
            mask &= mask - 1;
            const int r = base + b;
            load_record(P.recs, r, rec, lane);
            const float *gr = RP.ring + (size_t)r * RING_REC;
            const int N = (int)gr[RING_N];
            const double Phi = (double)gr[RING_PHI] + (double)gr[RING_PHI + 1];
            const double hstep = 2.0 * Phi / N;
            const float hw = gr[RING_HW], rt = gr[RING_RT];
            float AT[3], tfrh[3], tfrl[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) AT[k] = gr[RING_AT + k], tfrh[k] = gr[RING_TFR + k], tfrl[k] = gr[RING_TFR + 3 + k];
            // this lane's pixels relative to D (float, bounds and reach of the arc)
            float dZ[PPL], dR[PPL];
#pragma unroll
            for (int p = 0; p < PPL; ++p) {
                dZ[p] = (g.Zh[p] - rec[REC_ZD]) + (g.Zl[p] - rec[REC_ZD + 1]);
                dR[p] = (g.Rh[p] - rec[REC_RD]) + (g.Rl[p] - rec[REC_RD + 1]);
            }
            const float RDf = rec[REC_RD];
            const float rt2 = rt * rt * (1.0f + 1e-4f) + 1e-12f;
            const ff dZr = ff_add(two_sum(g.Zrh, -rec[REC_ZD]), ff{g.Zrl, -rec[REC_ZD + 1]});
            const ff dRr = ff_add(two_sum(g.Rrh, -rec[REC_RD]), ff{g.Rrl, -rec[REC_RD + 1]});
            const ff RD = {rec[REC_RD], rec[REC_RD + 1]}, Rr = {g.Rrh, g.Rrl};
            ff pair[PPL];
#pragma unroll
            for (int p = 0; p < PPL; ++p) pair[p] = ff{0.0f, 0.0f};
            // this warp's share of the points: j = z + S m, m = 0, 1, ...
            const int S = RP.n_split, z = blockIdx.z;
            const int nz = N > z ? (N - z + S - 1) / S : 0;
            for (int m0 = 0; m0 < nz; m0 += 32) {
                // azimuth points of m0 .. m0 + 31, one per lane, in FP64
                float sh = 0.f, sl = 0.f, oh = 0.f, ol = 0.f;
                {
                    const double phi = -Phi + (z + (double)S * (m0 + lane) + 0.5) * hstep;
                    const double sh2 = sin(0.5 * phi);
                    split_double(sin(phi), sh, sl);
                    split_double(2.0 * sh2 * sh2, oh, ol);  // 1 - cos(phi) without cancellation
                }
                const int je = min(32, nz - m0);
                for (int jj = 0; jj < je; ++jj) {
                    const ff sp = {__shfl_sync(FDX_FULL_MASK, sh, jj), __shfl_sync(FDX_FULL_MASK, sl, jj)};
                    const ff om = {__shfl_sync(FDX_FULL_MASK, oh, jj), __shfl_sync(FDX_FULL_MASK, ol, jj)};
                    const float cp = 1.0f - om.hi;
                    // |p(phi) - D|^2 = dZ^2 + dR^2 + 2 R R_D (1 - cos phi): skip arcs out of reach
                    bool nearp = false;
#pragma unroll
                    for (int p = 0; p < PPL; ++p)
                        nearp |= g.valid[p] &&
                                 fmaf(dZ[p], dZ[p], fmaf(dR[p], dR[p], 2.0f * g.Rh[p] * RDf * om.hi)) <= rt2;
                    if (!__any_sync(FDX_FULL_MASK, nearp)) continue;
                    QueryPts<PPL> q;
#pragma unroll
                    for (int p = 0; p < PPL; ++p) {
                        q.valid[p] = g.valid[p];
                        // p - D = dZ n + (dR cos phi - R_D (1 - cos phi)) e_R + R sin phi e_P
                        const float er = fmaf(dR[p], cp, -RDf * om.hi), et = g.Rh[p] * sp.hi;
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            q.P[p][k] = fmaf(dZ[p], rec[REC_NFR + k], fmaf(er, rec[REC_EFR + k], et * tfrh[k]));
#pragma unroll
                        for (int i = 0; i < 3; ++i)
                            q.tau[p][i] = g.valid[p] ? fmaf(g.dZl[p], P.AZ[i],
                                                            g.dRl[p] * fmaf(cp, rec[REC_AR + i], sp.hi * AT[i]))
                                                     : 1.0e4f;
                    }
                    // reference (p_ref - D)/r0 in the reflection frame, float-float
                    const ff cpf = ff_add(ff{1.0f, 0.0f}, ff{-om.hi, -om.lo});
                    const ff erf_ = ff_sub(ff_mul(dRr, cpf), ff_mul(RD, om));
                    const ff etf = ff_mul(Rr, sp);
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        q.dP[k] = ff_add(ff_add(ff_mul(dZr, ff{rec[REC_NFR + k], rec[REC_NFR + 3 + k]}),
                                                ff_mul(erf_, ff{rec[REC_EFR + k], rec[REC_EFR + 3 + k]})),
                                         ff_mul(etf, ff{tfrh[k], tfrl[k]}));
                    PairAcc pa[PPL];
#pragma unroll
                    for (int p = 0; p < PPL; ++p) clear(pa[p]);
                    if (!eval_core<LS, MODE, RING_NODE_BUF, PPL>(P, q, rec, buf, nullptr, bsc, bsc2, lane, pa)) continue;
#pragma unroll
                    for (int p = 0; p < PPL; ++p) {
                        if (MODE == MODE_CNT)
                            cnt[p] += pa[p].cnt;
                        else
                            pair[p] = ff_add(pair[p], pa[p].s0);
                    }
                }
            }
            if (MODE != MODE_CNT) {
#pragma unroll
                for (int p = 0; p < PPL; ++p) acc[p] = ff_add(acc[p], ff_mul_f(pair[p], rec[REC_FR] * hw));
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        if (!g.valid[p]) continue;
        const int px = px0 + (lane & 7), py = py0 + (lane >> 3) + 4 * p;
        const size_t out = (size_t)py * P.nx + px;
        if (!FDX_IN_BOUNDS(out, (long long)P.nx * P.ny, DBG_IMAGE)) continue;
        if (RP.partial) {
            const size_t slot = (size_t)blockIdx.z * P.nx * P.ny + out;
            if (MODE == MODE_CNT)
                reinterpret_cast<int32_t *>(RP.partial)[slot] = cnt[p];
            else
                RP.partial[slot] = make_float2(acc[p].hi, acc[p].lo);
        } else if (MODE == MODE_CNT) {
            P.counts[out] = cnt[p];
        } else {
            P.image[out] = acc[p].hi + acc[p].lo;
        }
    }
}

// Sum of the n_split partial results of a pixel, in split order.
__global__ void ring_reduce_kernel(const float2 *partial, int n_split, int npix, float *image, int32_t *counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix) return;
    if (counts) {
        const int32_t *pc = reinterpret_cast<const int32_t *>(partial);
        int32_t c = 0;
        for (int z = 0; z < n_split; ++z) c += pc[(size_t)z * npix + i];
        counts[i] = c;
    } else {
        ff a = {0.0f, 0.0f};
        for (int z = 0; z < n_split; ++z) {
            const float2 v = partial[(size_t)z * npix + i];
            a = ff_add(a, ff{v.x, v.y});
        }
        image[i] = a.hi + a.lo;
    }
}

template <int LS, int MODE>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 4) ring_kernel(RingParams RP) {
    __shared__ float4 s_nodes[PAIR_WARPS][RING_NODE_BUF];
    __shared__ float4 s_sc[PAIR_WARPS][(LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? RING_NODE_BUF : 1];
    __shared__ float4 s_sc2[PAIR_WARPS][(LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? RING_NODE_BUF / 2 : 1];
    __shared__ float s_rec[PAIR_WARPS][REC_SIZE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px0 = blockIdx.x * 16 + (warp & 1) * 8, py0 = blockIdx.y * (8 * RING_PPL) + (warp >> 1) * (4 * RING_PPL);
    if (px0 >= RP.P.nx || py0 >= RP.P.ny) return;
    ring_warp<LS, MODE, RING_PPL>(RP, px0, py0, s_nodes[warp], s_sc[warp], s_sc2[warp], s_rec[warp], lane);
}

template <int LS>
static void launch_ring_ls(const RingParams &p, bool count_mode, cudaStream_t s) {
    dim3 grid((p.P.nx + 15) / 16, (p.P.ny + 8 * RING_PPL - 1) / (8 * RING_PPL), p.n_split);
    if (count_mode)
        ring_kernel<LS, MODE_CNT><<<grid, PAIR_WARPS * 32, 0, s>>>(p);
    else
        ring_kernel<LS, MODE_FWD><<<grid, PAIR_WARPS * 32, 0, s>>>(p);
    if (p.partial) {
        const int npix = p.P.nx * p.P.ny;
        ring_reduce_kernel<<<(npix + 255) / 256, 256, 0, s>>>(p.partial, p.n_split, npix,
                                                              count_mode ? nullptr : p.P.image,
                                                              count_mode ? p.P.counts : nullptr);
    }
}

cudaError_t launch_ring(const RingParams &p, int lineshape, bool count_mode, cudaStream_t s) {
    if (lineshape == FDX_LINESHAPE_HOSEMANN)
        launch_ring_ls<FDX_LINESHAPE_HOSEMANN>(p, count_mode, s);
    else if (lineshape == FDX_LINESHAPE_GAUSS)
        launch_ring_ls<FDX_LINESHAPE_GAUSS>(p, count_mode, s);
    else
        launch_ring_ls<FDX_LINESHAPE_SINC>(p, count_mode, s);
    return cudaGetLastError();
}

}  // namespace fdx
