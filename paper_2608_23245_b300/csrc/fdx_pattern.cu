// Gather-form pattern kernel (Eq. direct_sum at every pixel's query point,
// times the Lorentz factor of Eq. lorentz).
//
// Work decomposition.  A CTA of 4 warps covers a 16 x 16 pixel block; each warp
// owns an 8 x 8 pixel patch, two pixels per lane, and accumulates its pixels
// in registers (no atomics).  The warp scans the reflection list 32 at a time
// with a conservative radial/polar test against its patch's (|S|, psi) bounds
// and evaluates the surviving (patch, reflection) pairs in list order
// (deterministic) with eval_pair (fdx_pair.cuh).  Pair sums are weighted by
// the reflection's pair factor and folded into a float-float pixel sum; the
// epilogue applies the Lorentz factor in FP64.
#include "fdx_pair.cuh"

namespace fdx {

static constexpr int FWD_NODE_BUF = 288;  // staged nodes per warp (even); 4 warps x 288 x 40 B keeps static shared memory < 48 KB
// Pixels per lane (PPL): 2 (a warp owns 8 x 8 pixels, a CTA 16 x 16) when
// the patch spans a small fraction of a lattice period, else 1 (8 x 4, 16 x 8);
// chosen on the host from the pixel pitch and the cell.

// One warp's 8 x (4 PPL) patch with top-left pixel (px0, py0): scan the
// reflections, evaluate the surviving pairs, write the pixels.
template <int LS, int MODE, int PPL>
__device__ __forceinline__ void pattern_warp(const PatternParams &P, int px0, int py0, float4 *buf, float4 *bsc,
                                             float4 *bsc2, float *rec, int lane) {
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
            cand = (q.x - q.y <= rmax) && (q.x + q.y >= rmin) && (q.z - q.w <= pmax) && (q.z + q.w >= pmin);
        }
        unsigned mask = __ballot_sync(FDX_FULL_MASK, cand);
        while (mask) {
            const int b = __ffs(mask) - 1;
            mask &= mask - 1;
            load_record(P.recs, base + b, rec, lane);
            PairAcc pa[PPL];
#pragma unroll
            for (int p = 0; p < PPL; ++p) clear(pa[p]);
            if (!eval_pair<LS, MODE, FWD_NODE_BUF, PPL>(P, g, rec, buf, nullptr, bsc, bsc2, lane, pa)) continue;
#pragma unroll
            for (int p = 0; p < PPL; ++p) {
                if (MODE == MODE_CNT)
                    cnt[p] += pa[p].cnt;
                else
                    acc[p] = ff_add(acc[p], ff_mul_f(pa[p].s0, rec[REC_FR]));
            }
        }
    }
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        if (!g.valid[p]) continue;
        const int px = px0 + (lane & 7), py = py0 + (lane >> 3) + 4 * p;
        const size_t out = (size_t)py * P.nx + px;
        if (MODE == MODE_CNT) {
            P.counts[out] = cnt[p];
        } else {
            const double R = (double)g.Rh[p] + (double)g.Rl[p];
            const double L = P.delta_L / (R + P.delta_L);
            P.image[out] = (float)(L * ((double)acc[p].hi + (double)acc[p].lo));
        }
    }
}

#define FDX_PATTERN_SMEM(LS, MODE)                                                                  \
    __shared__ float4 s_nodes[PAIR_WARPS][FWD_NODE_BUF];                                            \
    __shared__ float4 s_sc[PAIR_WARPS][(LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? FWD_NODE_BUF : 1]; \
    __shared__ float4 s_sc2[PAIR_WARPS][(LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? FWD_NODE_BUF / 2 : 1]; \
    __shared__ float s_rec[PAIR_WARPS][REC_SIZE];

template <int LS, int MODE, int PPL>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 4) pattern_kernel(PatternParams P) {
    FDX_PATTERN_SMEM(LS, MODE)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px0 = blockIdx.x * 16 + (warp & 1) * 8, py0 = blockIdx.y * (8 * PPL) + (warp >> 1) * (4 * PPL);
    if (px0 >= P.nx || py0 >= P.ny) return;  // the whole patch is outside; its first pixel is valid otherwise
    pattern_warp<LS, MODE, PPL>(P, px0, py0, s_nodes[warp], s_sc[warp], s_sc2[warp], s_rec[warp], lane);
}

// Model of a flattened item index: the last m with prefix[m] <= item.
__device__ __forceinline__ int item_model(const long long *prefix, int n_models, long long item) {
    int lo = 0, hi = n_models - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Persistent forward over many models: CTAs take (model, tile) items from an
// atomic counter until the items of all models are done.  Every item is
// computed by one CTA start to finish, so the result does not depend on the
// order in which items are taken.
template <int LS>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 4) pattern_batch_kernel(BatchFwdParams B) {
    FDX_PATTERN_SMEM(LS, MODE_FWD)
    __shared__ long long s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(B.counter, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= B.total_items) break;
        const int m = item_model(B.item_prefix, B.n_models, item);
        const PatternParams &P = B.models[m];
        const int t = (int)(item - B.item_prefix[m]);
        const int ppl = P.ppl;
        const int tiles_x = (P.nx + 15) / 16;
        const int bx = t % tiles_x, by = t / tiles_x;
        const int px0 = bx * 16 + (warp & 1) * 8, py0 = by * (8 * ppl) + (warp >> 1) * (4 * ppl);
        if (px0 >= P.nx || py0 >= P.ny) continue;
        if (ppl == 2)
            pattern_warp<LS, MODE_FWD, 2>(P, px0, py0, s_nodes[warp], s_sc[warp], s_sc2[warp], s_rec[warp], lane);
        else
            pattern_warp<LS, MODE_FWD, 1>(P, px0, py0, s_nodes[warp], s_sc[warp], s_sc2[warp], s_rec[warp], lane);
    }
}

cudaError_t launch_pattern_batch(const BatchFwdParams &B, int n_ctas, cudaStream_t s) {
    pattern_batch_kernel<FDX_LINESHAPE_HOSEMANN><<<n_ctas, PAIR_WARPS * 32, 0, s>>>(B);
    return cudaGetLastError();
}

template <int LS, int PPL>
static void launch_ls(const PatternParams &p, bool count_mode, cudaStream_t s) {
    dim3 grid((p.nx + 15) / 16, (p.ny + 8 * PPL - 1) / (8 * PPL));
    dim3 block(PAIR_WARPS * 32);
    if (count_mode)
        pattern_kernel<LS, MODE_CNT, PPL><<<grid, block, 0, s>>>(p);
    else
        pattern_kernel<LS, MODE_FWD, PPL><<<grid, block, 0, s>>>(p);
}

template <int PPL>
static void launch_ppl(const PatternParams &p, int lineshape, bool count_mode, cudaStream_t s) {
    if (lineshape == FDX_LINESHAPE_HOSEMANN)
        launch_ls<FDX_LINESHAPE_HOSEMANN, PPL>(p, count_mode, s);
    else if (lineshape == FDX_LINESHAPE_GAUSS)
        launch_ls<FDX_LINESHAPE_GAUSS, PPL>(p, count_mode, s);
    else
        launch_ls<FDX_LINESHAPE_SINC, PPL>(p, count_mode, s);
}

cudaError_t launch_pattern(const PatternParams &p, int lineshape, bool count_mode, cudaStream_t s) {
    if (p.ppl == 2)
        launch_ppl<2>(p, lineshape, count_mode, s);
    else
        launch_ppl<1>(p, lineshape, count_mode, s);
    return cudaGetLastError();
}

}  // namespace fdx
