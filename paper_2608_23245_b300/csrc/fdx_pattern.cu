// Gather-form pattern kernel (Eq. direct_sum at every pixel's query point,
// times the Lorentz factor of Eq. lorentz).
//
// Work decomposition.  A CTA of 4 warps covers a 16 x 8 pixel block; each warp
// owns an 8 x 4 pixel patch, one pixel per lane, and accumulates its pixels in
// registers (no atomics).  The warp scans the reflection list 32 at a time
// with a conservative radial/polar test against its patch's (|S|, psi) bounds
// and evaluates the surviving (patch, reflection) pairs in list order
// (deterministic) with eval_pair (fdx_pair.cuh).  Pair sums are weighted by
// the reflection's pair factor and folded into a float-float pixel sum; the
// epilogue applies the Lorentz factor in FP64.
#include "fdx_pair.cuh"

namespace fdx {

static constexpr int FWD_NODE_BUF = 288;  // staged nodes per warp; 4 warps x 288 x 40 B keeps static shared memory < 48 KB

template <int LS, int MODE>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 4) pattern_kernel(PatternParams P) {
    __shared__ float4 s_nodes[PAIR_WARPS][FWD_NODE_BUF];
    __shared__ float4 s_sc[PAIR_WARPS][(LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? FWD_NODE_BUF : 1];
    __shared__ float2 s_sc2[PAIR_WARPS][(LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? FWD_NODE_BUF : 1];
    __shared__ float s_rec[PAIR_WARPS][REC_SIZE];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px0 = blockIdx.x * 16 + (warp & 1) * 8, py0 = blockIdx.y * 8 + (warp >> 1) * 4;
    const bool lane_valid = (px0 + (lane & 7) < P.nx) && (py0 + (lane >> 3) < P.ny);
    if (__ballot_sync(FDX_FULL_MASK, lane_valid) == 0) return;  // lane 0 is valid from here on
    const PatchPix g = load_patch(P.pixgeo, P.nx, P.ny, px0, py0, lane);

    const float rlen = sqrtf(g.Rh * g.Rh + g.Zh * g.Zh), psi = atan2f(g.Rh, g.Zh);
    const float rmin = warp_min(g.valid ? rlen : 3.0e38f), rmax = warp_max(g.valid ? rlen : -3.0e38f);
    const float pmin = warp_min(g.valid ? psi : 3.0e38f), pmax = warp_max(g.valid ? psi : -3.0e38f);

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
            load_record(P.recs, base + b, rec, lane);
            PairAcc pa;
            pa.s0 = {0.0f, 0.0f};
            pa.cnt = 0;
            if (!eval_pair<LS, MODE, FWD_NODE_BUF>(P, g, rec, buf, nullptr, s_sc[warp], s_sc2[warp], lane, pa)) continue;
            if (MODE == MODE_CNT)
                cnt += pa.cnt;
            else
                acc = ff_add(acc, ff_mul_f(pa.s0, rec[REC_FR]));
        }
    }
    if (!g.valid) return;
    const int px = px0 + (lane & 7), py = py0 + (lane >> 3);
    const size_t out = (size_t)py * P.nx + px;
    if (MODE == MODE_CNT) {
        P.counts[out] = cnt;
    } else {
        const double R = (double)g.Rh + (double)g.Rl;
        const double L = P.delta_L / (R + P.delta_L);
        P.image[out] = (float)(L * ((double)acc.hi + (double)acc.lo));
    }
}

cudaError_t launch_pattern(const PatternParams &p, int lineshape, bool count_mode, cudaStream_t s) {
    dim3 grid((p.nx + 15) / 16, (p.ny + 7) / 8);
    dim3 block(PAIR_WARPS * 32);
    if (lineshape == FDX_LINESHAPE_HOSEMANN) {
        if (count_mode)
            pattern_kernel<FDX_LINESHAPE_HOSEMANN, MODE_CNT><<<grid, block, 0, s>>>(p);
        else
            pattern_kernel<FDX_LINESHAPE_HOSEMANN, MODE_FWD><<<grid, block, 0, s>>>(p);
    } else {
        if (count_mode)
            pattern_kernel<FDX_LINESHAPE_SINC, MODE_CNT><<<grid, block, 0, s>>>(p);
        else
            pattern_kernel<FDX_LINESHAPE_SINC, MODE_FWD><<<grid, block, 0, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace fdx
