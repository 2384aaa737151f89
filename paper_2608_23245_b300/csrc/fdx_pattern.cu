// Gather-form pattern kernel (Eq. direct_sum at every pixel's query point,
// times the Lorentz factor of Eq. lorentz).
//
// Work decomposition.  A CTA of 4 warps covers a 16 x 16 pixel block; each warp
// owns an 8 x 8 pixel patch (the tile), two pixels per lane, and accumulates
// its pixels in registers (no atomics).  Binning is tile-major: the warp bins
// the reflections to its tile by the closed-form footprint of each one in
// (|S|, psi) -- the inverse-Ewald image of a pixel is its (R, Z), and a
// reflection reaches it only within its (r0 +- rho_B, psi_D +- dpsi) window --
// and stages the tile's list in shared memory, then evaluates the listed
// (tile, reflection) pairs in list order (deterministic) with eval_pair
// (fdx_pair.cuh).  Pair sums are weighted by the reflection's pair factor and
// folded into a float-float pixel sum; the epilogue applies the Lorentz
// factor in FP64.
#include "fdx_pair.cuh"

namespace fdx {

static constexpr int FWD_NODE_BUF = 288;  // staged nodes per warp (even): 54 KB per CTA, 4 CTAs per SM
static constexpr int TILE_SCAN = 512;     // reflections tested per refill of a tile's list
// Pixels per lane (PPL): 2 (a warp owns 8 x 8 pixels, a CTA 16 x 16) when
// the patch spans a small fraction of a lattice period, else 1 (8 x 4, 16 x 8);
// chosen on the host from the pixel pitch and the cell.

// One warp's 8 x (4 PPL) patch with top-left pixel (px0, py0): scan the
// reflections, evaluate the surviving pairs, write the pixels.
template <int LS, int MODE, int PPL>
__device__ __forceinline__ void pattern_warp(const PatternParams &P, int px0, int py0, float4 *buf, float4 *bsc,
                                             float4 *bsc2, float *rec, int *lst, int lane) {
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

    // The tile's reflection list, TILE_SCAN reflections at a time: the
    // closed-form footprint test (reflection's (|S|, psi) window against the
    // patch's) on 16 coalesced loads in flight, survivors staged in shared
    // memory in list order.  The list is then evaluated in order, each
    // candidate's record loaded into registers while the previous one is
    // evaluated.
    for (int base = 0; base < P.n_refl; base += TILE_SCAN) {
        int n = 0;
#pragma unroll
        for (int gq = 0; gq < TILE_SCAN / 32; ++gq) {
            const int rr = base + 32 * gq + lane;
            bool cand = false;
            if (rr < P.n_refl) {
                const float4 q = P.reach[rr];
                cand = (q.x - q.y <= rmax) && (q.x + q.y >= rmin) && (q.z - q.w <= pmax) && (q.z + q.w >= pmin);
            }
            const unsigned m = __ballot_sync(FDX_FULL_MASK, cand);
            const int slot = n + __popc(m & ((1u << lane) - 1u));
            if (cand && FDX_IN_BOUNDS(slot, TILE_SCAN, DBG_LIST)) lst[slot] = rr;
            n += __popc(m);
        }
        __syncwarp();
        if (n == 0) continue;
        float nx0 = 0.0f, nx1 = 0.0f;
        if (FDX_IN_BOUNDS(lst[0], P.n_refl, DBG_RECORD)) {
            const float *grec = P.recs + (size_t)lst[0] * REC_SIZE;
            nx0 = grec[lane], nx1 = grec[lane + 32];
        }
        for (int c = 0; c < n; ++c) {
            __syncwarp();
            rec[lane] = nx0, rec[lane + 32] = nx1;
            __syncwarp();
            if (c + 1 < n && FDX_IN_BOUNDS(lst[c + 1], P.n_refl, DBG_RECORD)) {
                const float *gn = P.recs + (size_t)lst[c + 1] * REC_SIZE;
                nx0 = gn[lane], nx1 = gn[lane + 32];
            }
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
        __syncwarp();
    }
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        if (!g.valid[p]) continue;
        const int px = px0 + (lane & 7), py = py0 + (lane >> 3) + 4 * p;
        const size_t out = (size_t)py * P.nx + px;
        if (!FDX_IN_BOUNDS(out, (long long)P.nx * P.ny, DBG_IMAGE)) continue;
        if (MODE == MODE_CNT) {
            P.counts[out] = cnt[p];
        } else {
            const double R = (double)g.Rh[p] + (double)g.Rl[p];
            const double L = P.delta_L / (R + P.delta_L);
            P.image[out] = (float)(L * ((double)acc[p].hi + (double)acc[p].lo));
        }
    }
}

// Shared memory of a pattern CTA (dynamic, so that it may exceed the 48 KB a
// kernel can declare statically), per warp: the staged nodes, the scaled
// sin/cos of the Hosemann walk, the reflection record and the tile's
// reflection list.
template <int LS, int MODE>
struct PatternSmem {
    static constexpr int SC = (LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? FWD_NODE_BUF : 1;
    static constexpr int SC2 = (LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? FWD_NODE_BUF / 2 : 1;
    static constexpr int PER_WARP = FWD_NODE_BUF + SC + SC2 + REC_SIZE / 4 + TILE_SCAN / 4;  // float4 units
    static constexpr size_t BYTES = sizeof(float4) * PAIR_WARPS * PER_WARP;
    float4 *nodes, *sc, *sc2;
    float *rec;
    int *lst;
    __device__ __forceinline__ PatternSmem(float4 *base, int warp) {
        float4 *w = base + (size_t)warp * PER_WARP;
        nodes = w, sc = nodes + FWD_NODE_BUF, sc2 = sc + SC;
        rec = reinterpret_cast<float *>(sc2 + SC2);
        lst = reinterpret_cast<int *>(sc2 + SC2 + REC_SIZE / 4);
    }
};

template <int LS, int MODE, int PPL>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 4) pattern_kernel(PatternParams P) {
    extern __shared__ float4 dsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px0 = blockIdx.x * 16 + (warp & 1) * 8, py0 = blockIdx.y * (8 * PPL) + (warp >> 1) * (4 * PPL);
    if (px0 >= P.nx || py0 >= P.ny) return;  // the whole patch is outside; its first pixel is valid otherwise
    const PatternSmem<LS, MODE> sm(dsm, warp);
    pattern_warp<LS, MODE, PPL>(P, px0, py0, sm.nodes, sm.sc, sm.sc2, sm.rec, sm.lst, lane);
}

// Persistent forward over the models of one tile shape: CTAs take (model,
// tile) items from an atomic counter until the items of all of them are done.
// Every item is computed by one CTA start to finish, so the result does not
// depend on the order in which items are taken; compiled for one PPL, like
// the per-model kernel.
template <int LS, int PPL>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 4) pattern_batch_kernel(BatchFwdParams B) {
    extern __shared__ float4 dsm[];
    __shared__ long long s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PatternSmem<LS, MODE_FWD> sm(dsm, warp);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = B.item0 + (long long)atomicAdd(B.counter, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= B.item_end) break;
        const int j = item_position(B.item_prefix, B.pos0, B.n_pos, item);
        if (!FDX_IN_BOUNDS(j - B.pos0, B.n_pos, DBG_BATCH)) continue;
        const PatternParams &P = B.models[B.item_model[j]];
        const int t = (int)(item - B.item_prefix[j]);
        const int tiles_x = (P.nx + 15) / 16;
        const int bx = t % tiles_x, by = t / tiles_x;
        const int px0 = bx * 16 + (warp & 1) * 8, py0 = by * (8 * PPL) + (warp >> 1) * (4 * PPL);
        if (px0 >= P.nx || py0 >= P.ny) continue;
        pattern_warp<LS, MODE_FWD, PPL>(P, px0, py0, sm.nodes, sm.sc, sm.sc2, sm.rec, sm.lst, lane);
    }
}

// Opt a kernel into `bytes` of dynamic shared memory (above 48 KB this must be
// requested; done once per kernel and device).
template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int PPL>
static cudaError_t launch_pattern_batch_ppl(const BatchFwdParams &B, int n_ctas, cudaStream_t s) {
    constexpr size_t bytes = PatternSmem<FDX_LINESHAPE_HOSEMANN, MODE_FWD>::BYTES;
    cudaError_t e = allow_smem(pattern_batch_kernel<FDX_LINESHAPE_HOSEMANN, PPL>, bytes);
    if (e != cudaSuccess) return e;
    pattern_batch_kernel<FDX_LINESHAPE_HOSEMANN, PPL><<<n_ctas, PAIR_WARPS * 32, bytes, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_pattern_batch(const BatchFwdParams &B, int ppl, int n_ctas, cudaStream_t s) {
    return ppl == 2 ? launch_pattern_batch_ppl<2>(B, n_ctas, s) : launch_pattern_batch_ppl<1>(B, n_ctas, s);
}

template <int LS, int PPL>
static cudaError_t launch_ls(const PatternParams &p, bool count_mode, cudaStream_t s) {
    dim3 grid((p.nx + 15) / 16, (p.ny + 8 * PPL - 1) / (8 * PPL));
    dim3 block(PAIR_WARPS * 32);
    if (count_mode) {
        constexpr size_t bytes = PatternSmem<LS, MODE_CNT>::BYTES;
        cudaError_t e = allow_smem(pattern_kernel<LS, MODE_CNT, PPL>, bytes);
        if (e != cudaSuccess) return e;
        pattern_kernel<LS, MODE_CNT, PPL><<<grid, block, bytes, s>>>(p);
    } else {
        constexpr size_t bytes = PatternSmem<LS, MODE_FWD>::BYTES;
        cudaError_t e = allow_smem(pattern_kernel<LS, MODE_FWD, PPL>, bytes);
        if (e != cudaSuccess) return e;
        pattern_kernel<LS, MODE_FWD, PPL><<<grid, block, bytes, s>>>(p);
    }
    return cudaGetLastError();
}

template <int PPL>
static cudaError_t launch_ppl(const PatternParams &p, int lineshape, bool count_mode, cudaStream_t s) {
    if (lineshape == FDX_LINESHAPE_HOSEMANN) return launch_ls<FDX_LINESHAPE_HOSEMANN, PPL>(p, count_mode, s);
    if (lineshape == FDX_LINESHAPE_GAUSS) return launch_ls<FDX_LINESHAPE_GAUSS, PPL>(p, count_mode, s);
    return launch_ls<FDX_LINESHAPE_SINC, PPL>(p, count_mode, s);
}

cudaError_t launch_pattern(const PatternParams &p, int lineshape, bool count_mode, cudaStream_t s) {
    return p.ppl == 2 ? launch_ppl<2>(p, lineshape, count_mode, s) : launch_ppl<1>(p, lineshape, count_mode, s);
}

}  // namespace fdx
