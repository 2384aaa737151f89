// Refinement path: loss, pattern adjoint, structure-factor adjoint, and the
// chain rule to the global disorder parameters.
//
// Loss (refinement loss of the scope): L = sum_px m_px w_px (I - I_t)^2,
// w = 1/(I_t + 1), optional mask m; dL/dI = 2 m w (I - I_t).
//
// Pattern adjoint.  I_px = L_px sum_r M_r r0^2 B_r S_r(px), B_r = prod_i beta_i,
// S_r(px) = sum_k w_k prod_i 1/den_i (Hosemann).  Per reflection:
//   dL/dM_r        = r0^2 B_r sum_px c_px S_r(px),                c_px = dL/dI_px L_px
//   dL/dbeta_{r,i} = M_r r0^2 B_r sum_px c_px (S/beta_i - 2 beta_i/(1 - beta_i^2) Sb_i),
//                    Sb_i = sum_k w_k prod 1/den (1/den_i - 1)  (from dK_i/dbeta_i)
//   dL/dsigma_r    = M_r r0^2 B_r sum_px c_px sum_k (dw_k/dsigma) prod 1/den, same for gamma.
// The profiles are recomputed, not stored.  Work decomposition is
// reflection-major so that per-reflection sums stay in one warp: a work item
// is (reflection, band of pixel-patch rows); its warp walks the band's 8 x 4
// patches that pass the reach test and evaluates each (patch, reflection) pair
// with the forward's eval_pair in adjoint mode.  Items write their six sums;
// a second kernel adds the bands of each reflection in fixed order.  No atomics.
//
// Structure-factor adjoint (M = |F|^2 P DW):
//   dL/dx_{j,c} = sum_r -4 pi h_c Im(c_r T_jr),  dL/dB_j = sum_r -(s_r^2/2) Re(c_r T_jr),
//   c_r = dL/dM_r P_r DW_r conj(F_r),  T_jr = occ_j f_j(s_r) exp(-B_j s_r^2/4) exp(2 pi i h_r . x_j).
// Chain rule (reading R4/R5, Eqs. Ah/Neff/Ipara): beta = min(1, |a_i|/L_i + tanh x),
// x = pi^2 g^2 h^2; dbeta/dL = -|a_i|/L_i^2, dbeta/dg = sech^2(x) 2 pi^2 g h^2 (0 when
// clamped); dP/dg_i = -P tanh(2x_i) 4 pi^2 g_i h_i^2.
#include "fdx_adjoint.cuh"
#include "fdx_pair.cuh"

namespace fdx {

static constexpr int ADJ_ITEM_VALS = 6;
// Staged nodes per warp: 384 (dynamic shared memory, 74.8 KB per CTA, 3 CTAs
// per SM at the kernels' register count); 224, the most that static shared
// memory allows, flushed twice as often and was 1.4 % slower.
static constexpr int ADJ_NODE_BUF = 384;
static constexpr int ADJ_PER_WARP = ADJ_NODE_BUF * 3 + REC_SIZE / 4;  // float4: nodes, dw (NB/2), sc, sc2 (NB/2), record
static constexpr size_t ADJ_SMEM_BYTES = sizeof(float4) * PAIR_WARPS * ADJ_PER_WARP;

__device__ __forceinline__ bool reach_overlap(float4 q, float4 b) {
    // q = (r0, rho_B, psi_D, dpsi); b = (rmin, rmax, psimin, psimax)
    return (q.x - q.y <= b.y) && (q.x + q.y >= b.x) && (q.z - q.w <= b.w) && (q.z + q.w >= b.z);
}

// Bounds (|S| min/max, psi min/max) of every 8 x 4 patch; one warp per patch.
__global__ void patch_bounds_kernel(AdjParams A) {
    const int warp_g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp_g >= A.npx * A.npy) return;
    const int pi = warp_g % A.npx, pj = warp_g / A.npx;
    const int px = 8 * pi + (lane & 7), py = 4 * pj + (lane >> 3);
    const bool valid = px < A.P.nx && py < A.P.ny;
    float r = 3.0e38f, rr = -3.0e38f, p = 3.0e38f, pp = -3.0e38f;
    if (valid) {
        const float4 g = A.P.pixgeo[(size_t)py * A.P.nx + px];
        r = rr = sqrtf(g.x * g.x + g.z * g.z);
        p = pp = atan2f(g.x, g.z);
    }
    r = warp_min(r), rr = warp_max(rr), p = warp_min(p), pp = warp_max(pp);
    if (lane == 0) A.patch_bounds[warp_g] = make_float4(r, rr, p, pp);
}

// Bounds of each band of patch rows; one block per band (min/max are exact).
__global__ void band_bounds_kernel(AdjParams A) {
    __shared__ float4 red[256];
    const int b = blockIdx.x;
    const int pj0 = b * A.rows_per_band, pj1 = min(A.npy, pj0 + A.rows_per_band);
    float4 acc = make_float4(3.0e38f, -3.0e38f, 3.0e38f, -3.0e38f);
    for (int k = threadIdx.x; k < (pj1 - pj0) * A.npx; k += blockDim.x) {
        const float4 v = A.patch_bounds[(size_t)pj0 * A.npx + k];
        acc.x = fminf(acc.x, v.x), acc.y = fmaxf(acc.y, v.y), acc.z = fminf(acc.z, v.z), acc.w = fmaxf(acc.w, v.w);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const float4 o = red[threadIdx.x + s];
            float4 &m = red[threadIdx.x];
            m.x = fminf(m.x, o.x), m.y = fmaxf(m.y, o.y), m.z = fminf(m.z, o.z), m.w = fmaxf(m.w, o.w);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) A.band_bounds[b] = red[0];
}

// One (reflection, band) item of the adjoint for one warp.  With PPL = 2 the
// warp's patch is 8 x 8 pixels (two rows of 8 x 4 bound patches; bands hold
// an even number of patch rows).  Per lane, the pair sums times the pixel's
// c = dL/dI L (applied to each 64-pair FP32 chunk sum) are accumulated in one
// float-float sum per quantity over the item's patches; the warp adds its
// lanes in FP64 once at the end.
template <int LS, int PPL>
__device__ __forceinline__ void adjoint_item(const AdjParams &A, long long item, float4 *buf, float4 *dn, float4 *sc,
                                             float4 *sc2, float *rec, int lane) {
    const int r = (int)(item / A.n_bands), b = (int)(item % A.n_bands);
    PairAcc tot[PPL];  // the item's sums, weighted by each pixel's c, in tot[0]
#pragma unroll
    for (int p = 0; p < PPL; ++p) clear(tot[p]);
    const float4 q = A.P.reach[r];
    if (reach_overlap(q, A.band_bounds[b])) {
        load_record(A.P.recs, r, rec, lane);
        const int pj0 = b * A.rows_per_band, pj1 = min(A.npy, pj0 + A.rows_per_band);
        const int nrow = (pj1 - pj0 + PPL - 1) / PPL;  // patch rows of this band, PPL bound rows each
        const int np = nrow * A.npx;
        const float dl = (float)A.P.delta_L;
        for (int base = 0; base < np; base += 32) {
            const int idx = base + lane;
            bool cand = false;
            if (idx < np) {
                const int pj = pj0 + PPL * (idx / A.npx), pi = idx % A.npx;
                float4 bb = make_float4(3.0e38f, -3.0e38f, 3.0e38f, -3.0e38f);  // empty: no overlap
                if (FDX_IN_BOUNDS((size_t)pj * A.npx + pi, (long long)A.npx * A.npy, DBG_PATCH))
                    bb = A.patch_bounds[(size_t)pj * A.npx + pi];
                if (PPL == 2 && pj + 1 < A.npy &&
                    FDX_IN_BOUNDS((size_t)(pj + 1) * A.npx + pi, (long long)A.npx * A.npy, DBG_PATCH)) {
                    const float4 b2 = A.patch_bounds[(size_t)(pj + 1) * A.npx + pi];
                    bb = make_float4(fminf(bb.x, b2.x), fmaxf(bb.y, b2.y), fminf(bb.z, b2.z), fmaxf(bb.w, b2.w));
                }
                cand = reach_overlap(q, bb);
            }
            unsigned mask = __ballot_sync(FDX_FULL_MASK, cand);
            while (mask) {
                const int bit = __ffs(mask) - 1;
                mask &= mask - 1;
                const int k = base + bit;
                const int px0 = 8 * (k % A.npx), py0 = 4 * (pj0 + PPL * (k / A.npx));
                const PatchPix<PPL> g = load_patch<PPL>(A.P.pixgeo, A.P.nx, A.P.ny, px0, py0, lane);
                QueryPts<PPL> qp = pixel_queries<PPL>(A.P, g, rec);
                bool any = false;
#pragma unroll
                for (int p = 0; p < PPL; ++p) {
                    qp.cw[p] = 0.0f;
                    if (g.valid[p]) {
                        const int px = px0 + (lane & 7), py = py0 + (lane >> 3) + 4 * p;
                        const size_t q = (size_t)py * A.P.nx + px;
                        if (FDX_IN_BOUNDS(q, (long long)A.P.nx * A.P.ny, DBG_GRAD_IN))
                            qp.cw[p] = A.gI[q] * (dl / ((g.Rh[p] + g.Rl[p]) + dl));
                    }
                    any |= qp.cw[p] != 0.0f;
                }
                if (__ballot_sync(FDX_FULL_MASK, any) == 0) continue;
                eval_core<LS, MODE_ADJ, ADJ_NODE_BUF, PPL>(A.P, qp, rec, buf, dn, sc, sc2, lane, tot);
            }
        }
    }
    const ff ia[ADJ_ITEM_VALS] = {tot[0].s0, tot[0].sb[0], tot[0].sb[1], tot[0].sb[2], tot[0].ss, tot[0].sg};
    double acc[ADJ_ITEM_VALS];
#pragma unroll
    for (int k = 0; k < ADJ_ITEM_VALS; ++k) acc[k] = warp_sum_d((double)ia[k].hi + (double)ia[k].lo);
    // Hosemann: the beta sums were accumulated as sum w / (den_i prod den);
    // subtract the profile sum for sum (w / prod den) (1/den_i - 1).  The
    // other lineshapes accumulate sum w dK_i/dbeta_i prod_{j != i} K_j directly.
    if (LS == FDX_LINESHAPE_HOSEMANN) {
#pragma unroll
        for (int k = 1; k <= 3; ++k) acc[k] -= acc[0];
    }
    if (lane < ADJ_ITEM_VALS) {
        double o = acc[0];
#pragma unroll
        for (int k = 1; k < ADJ_ITEM_VALS; ++k)
            if (lane == k) o = acc[k];
        if (FDX_IN_BOUNDS(item * ADJ_ITEM_VALS + lane, (long long)A.P.n_refl * A.n_bands * ADJ_ITEM_VALS, DBG_ITEM))
            A.item_out[item * ADJ_ITEM_VALS + lane] = o;
    }
}

// This warp's slice of the adjoint kernels' dynamic shared memory.
#define FDX_ADJ_SMEM                                                                           \
    extern __shared__ float4 adsm[];                                                           \
    float4 *const s_nodes = adsm + (size_t)(threadIdx.x >> 5) * ADJ_PER_WARP;                  \
    float4 *const s_dn = s_nodes + ADJ_NODE_BUF, *const s_sc = s_dn + ADJ_NODE_BUF / 2;        \
    float4 *const s_sc2 = s_sc + ADJ_NODE_BUF;                                                 \
    float *const s_rec = reinterpret_cast<float *>(s_sc2 + ADJ_NODE_BUF / 2);

// Single-model adjoint, persistent: each warp takes (reflection, band) items
// from the model's queue until none is left, so warps whose items end early
// (no overlap with the band) pick up more work instead of idling in their CTA.
template <int LS, int PPL>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 3) adjoint_kernel(AdjParams A) {
    FDX_ADJ_SMEM
    const int lane = threadIdx.x & 31;
    const long long total = (long long)A.P.n_refl * A.n_bands;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(A.counter, 1u);
        const long long item = (long long)__shfl_sync(FDX_FULL_MASK, it, 0);
        if (item >= total) break;
        adjoint_item<LS, PPL>(A, item, s_nodes, s_dn, s_sc, s_sc2, s_rec, lane);
    }
}

// Persistent adjoint over the models of one tile shape: each warp takes
// (model, reflection, band) items from an atomic counter; items are
// independent, so the order in which they are taken does not change any
// result.  Compiled for one PPL, like the per-model kernel.
template <int PPL>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 3) adjoint_batch_kernel(BatchAdjParams B) {
    FDX_ADJ_SMEM
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(B.counter, 1u);
        const long long item = B.item0 + (long long)__shfl_sync(FDX_FULL_MASK, it, 0);
        if (item >= B.item_end) break;
        const int j = item_position(B.item_prefix, B.pos0, B.n_pos, item);
        if (!FDX_IN_BOUNDS(j - B.pos0, B.n_pos, DBG_BATCH)) continue;
        adjoint_item<FDX_LINESHAPE_HOSEMANN, PPL>(B.models[B.item_model[j]], item - B.item_prefix[j], s_nodes, s_dn,
                                                  s_sc, s_sc2, s_rec, lane);
    }
}

// Per reflection: add the bands in order and form dL/dM, dL/dbeta, dL/dsigma,
// dL/dgamma; then chain to the global parameters and the structure-factor
// adjoint's coefficient c_r = dL/dM P DW conj(F).  FP64.
__global__ void adjoint_reflection_kernel(AdjParams A) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.P.n_refl) return;
    double s[ADJ_ITEM_VALS] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < A.n_bands; ++b)
        for (int k = 0; k < ADJ_ITEM_VALS; ++k) s[k] += A.item_out[((size_t)r * A.n_bands + b) * ADJ_ITEM_VALS + k];
    const float *rec = A.P.recs + (size_t)r * REC_SIZE;
    const double M = rec[REC_M];
    double G, dbeta[3], dsig, dgam;
    if (A.lineshape == FDX_LINESHAPE_HOSEMANN) {
        // sums relative to prod K_i = prod beta_i / den_i; r0^2 prod beta in the record
        const double r2b = rec[REC_R2B];
        G = r2b * s[0];
        for (int i = 0; i < 3; ++i)
            dbeta[i] = M * r2b * (s[0] / (double)rec[REC_BETA + i] - (double)rec[REC_DBF + i] * s[1 + i]);
        dsig = M * r2b * s[4], dgam = M * r2b * s[5];
    } else {
        // absolute sums: sum w prod K, sum w dK_i/dbeta_i prod_{j != i} K_j, weight derivatives
        double Dv[3];
        for (int q = 0; q < 3; ++q)
            Dv[q] = A.hkl[3 * r] * A.As[q] + A.hkl[3 * r + 1] * A.As[3 + q] + A.hkl[3 * r + 2] * A.As[6 + q];
        const double r2 = Dv[0] * Dv[0] + Dv[1] * Dv[1] + Dv[2] * Dv[2];
        G = r2 * s[0];
        for (int i = 0; i < 3; ++i) dbeta[i] = M * r2 * s[1 + i];
        dsig = M * r2 * s[4], dgam = M * r2 * s[5];
    }
    if (A.dM) A.dM[r] = (float)G;

    // chain rule to L_i, g_i; P and DW for the structure-factor adjoint
    double P = 1.0, dw = 0.0, x[3];
    int hk[3];
    for (int i = 0; i < 3; ++i) {
        hk[i] = A.hkl[3 * r + i];
        x[i] = FDX_PI * FDX_PI * A.g[i] * A.g[i] * (double)hk[i] * hk[i];
        if (A.intensity_model == FDX_INTENSITY_HOSEMANN) P *= 1.0 / cosh(2.0 * x[i]);
        const double sa = hk[i] / A.alen[i];
        dw += A.Bax[i] * sa * sa;
    }
    const double DW = exp(-0.25 * dw);
    const double Fr = A.F[2 * r], Fi = A.F[2 * r + 1];
    const double F2 = Fr * Fr + Fi * Fi;
    double *o = A.refl_out + (size_t)r * 8;
    for (int i = 0; i < 3; ++i) {
        const double braw = A.alen[i] / A.L[i] + tanh(x[i]);
        double dLi = 0.0, dgi = 0.0;
        if (braw < 1.0) {
            dLi = dbeta[i] * (-A.alen[i] / (A.L[i] * A.L[i]));
            const double sh = 1.0 / cosh(x[i]);
            dgi = dbeta[i] * sh * sh * 2.0 * FDX_PI * FDX_PI * A.g[i] * (double)hk[i] * hk[i];
        }
        if (A.intensity_model == FDX_INTENSITY_HOSEMANN)
            dgi += G * F2 * DW * (-P * tanh(2.0 * x[i]) * 4.0 * FDX_PI * FDX_PI * A.g[i] * (double)hk[i] * hk[i]);
        o[i] = dLi;
        o[3 + i] = dgi;
    }
    o[6] = dsig;
    o[7] = dgam;
    const double Gw = G * P * DW;
    double D[3];
    for (int q = 0; q < 3; ++q) D[q] = hk[0] * A.As[q] + hk[1] * A.As[3 + q] + hk[2] * A.As[6 + q];
    const double s2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    A.cF[r] = make_float4((float)(Gw * Fr), (float)(-Gw * Fi), (float)s2, 0.0f);  // Gw conj(F), s^2
    for (int e = 0; e < A.n_elem; ++e) {
        const float *f = A.ff + 9 * e;
        double v = f[8];
        for (int m = 0; m < 4; ++m) v += (double)f[m] * exp(-(double)f[4 + m] * s2 * 0.25);
        A.fe[(size_t)r * A.n_elem + e] = (float)v;
    }
}

// Sum the per-reflection global contributions in a fixed order (one block).
__global__ void adjoint_globals_kernel(AdjParams A) {
    __shared__ double red[256][8];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < A.P.n_refl; r += blockDim.x)
        for (int k = 0; k < 8; ++k) acc[k] += A.refl_out[(size_t)r * 8 + k];
    for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 8; ++k) red[threadIdx.x][k] += red[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x < 8 && A.dglobal) A.dglobal[threadIdx.x] = red[0][threadIdx.x];
}

// ---------------------------------------------------------------------------
// Structure-factor adjoint: one thread per atom, reflections staged through
// shared memory in tiles, reflection list split over blockIdx.y; partial sums
// per split reduced in a second kernel (fixed order).
// ---------------------------------------------------------------------------
static constexpr int SFA_THREADS = 128;
static constexpr int SFA_TILE = 128;

__device__ __forceinline__ void sincos_turns_adj(unsigned u, float &s, float &c) {
    const unsigned qd = (u + 0x20000000u) >> 30;
    const int rem = (int)(u - (qd << 30));
    const int rh = rem >> 8, rl = rem & 255;
    const float fh = __int_as_float(0x4B400000 + rh) - 12582912.0f;
    const float fl = __int_as_float(0x4B000000 + rl) - 8388608.0f;
    const float r = fmaf(fh, 5.9604644775390625e-08f, fl * 2.3283064365386963e-10f);
    const float Sc[4] = FDX_SIN2PI_C;
    const float Cc[5] = FDX_COS2PI_C;
    const float r2 = r * r;
    const float sn = r * horner(Sc, r2);
    const float cs = horner(Cc, r2);
    const float s1 = (qd & 1) ? cs : sn;
    const float c1 = (qd & 1) ? -sn : cs;
    s = (qd & 2) ? -s1 : s1;
    c = (qd & 2) ? -c1 : c1;
}

__global__ void __launch_bounds__(SFA_THREADS) sf_adjoint_kernel(SFAdjParams p) {
    __shared__ int4 s_h[SFA_TILE];           // h, k, l, -
    __shared__ float4 s_c[SFA_TILE];         // c re, c im, s^2, -
    extern __shared__ float s_fe[];          // [SFA_TILE][n_elem]
    const int j = blockIdx.x * SFA_THREADS + threadIdx.x;
    const bool active = j < p.n_atoms;
    uint4 aq = make_uint4(0, 0, 0, 0);
    float2 aw = make_float2(0.0f, -INFINITY);
    if (active) aq = p.atoms_q[j], aw = p.atoms_w[j];
    const int r_begin = blockIdx.y * p.refl_per_split, r_end = min(p.n_refl, r_begin + p.refl_per_split);
    ff ax = {0, 0}, ay = {0, 0}, az = {0, 0}, ab = {0, 0};
    for (int t0 = r_begin; t0 < r_end; t0 += SFA_TILE) {
        const int cnt = min(SFA_TILE, r_end - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < SFA_TILE; i += SFA_THREADS) {
            if (i < cnt) {
                const int r = t0 + i;
                s_h[i] = make_int4(p.hkl[3 * r], p.hkl[3 * r + 1], p.hkl[3 * r + 2], 0);
                s_c[i] = p.cF[r];
                for (int e = 0; e < p.n_elem; ++e) s_fe[i * p.n_elem + e] = p.fe[(size_t)r * p.n_elem + e];
            } else {
                s_h[i] = make_int4(0, 0, 0, 0);
                s_c[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                for (int e = 0; e < p.n_elem; ++e) s_fe[i * p.n_elem + e] = 0.0f;
            }
        }
        __syncthreads();
        const int cnt8 = (cnt + 7) & ~7;
        for (int i0 = 0; i0 < cnt8; i0 += 8) {
            float bx = 0.f, by = 0.f, bz = 0.f, bb = 0.f;
#pragma unroll
            for (int i = i0; i < i0 + 8; ++i) {
                const int4 hk = s_h[i];
                const float4 c = s_c[i];
                const unsigned ph = (unsigned)hk.x * aq.x + (unsigned)hk.y * aq.y + (unsigned)hk.z * aq.z;
                float sn, cs;
                sincos_turns_adj(ph, sn, cs);
                const float a = s_fe[i * p.n_elem + aq.w] * exp2f(fmaf(aw.x, c.z, aw.y));
                const float im = a * fmaf(c.x, sn, c.y * cs);
                const float re = a * fmaf(c.x, cs, -c.y * sn);
                bx = fmaf((float)hk.x, im, bx);
                by = fmaf((float)hk.y, im, by);
                bz = fmaf((float)hk.z, im, bz);
                bb = fmaf(c.z, re, bb);
            }
            ax = ff_add_f(ax, bx), ay = ff_add_f(ay, by), az = ff_add_f(az, bz), ab = ff_add_f(ab, bb);
        }
    }
    if (active) {
        double *o = p.partial + ((size_t)blockIdx.y * p.n_atoms + j) * 4;
        o[0] = (double)ax.hi + ax.lo;
        o[1] = (double)ay.hi + ay.lo;
        o[2] = (double)az.hi + az.lo;
        o[3] = (double)ab.hi + ab.lo;
    }
}

__global__ void sf_adjoint_reduce_kernel(SFAdjParams p) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.n_atoms) return;
    double s[4] = {0, 0, 0, 0};
    for (int sp = 0; sp < p.n_split; ++sp)
        for (int k = 0; k < 4; ++k) s[k] += p.partial[((size_t)sp * p.n_atoms + j) * 4 + k];
    if (p.dfrac) {
        p.dfrac[3 * j] = -4.0 * FDX_PI * s[0];
        p.dfrac[3 * j + 1] = -4.0 * FDX_PI * s[1];
        p.dfrac[3 * j + 2] = -4.0 * FDX_PI * s[2];
    }
    if (p.dB) p.dB[j] = -0.5 * s[3];
}

// ---------------------------------------------------------------------------
// Loss L = sum m w (I - I_t)^2, w = 1/(I_t + 1); dL/dI = 2 m w (I - I_t).
// Per-block partial sums in a fixed tree, then one block adds them in order.
// ---------------------------------------------------------------------------
__global__ void loss_kernel(LossParams p) {
    __shared__ double red[256];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < p.n) {
        const double It = p.It[i], I = p.I[i];
        const double m = p.mask ? (double)p.mask[i] : 1.0;
        const double w = m / (It + 1.0);
        const double d = I - It;
        v = w * d * d;
        if (p.gI) p.gI[i] = (float)(2.0 * w * d);
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) p.partial[blockIdx.x] = red[0];
}

__global__ void loss_final_kernel(LossParams p, int nblocks) {
    __shared__ double red[256];
    double v = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) v += p.partial[k];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *p.loss = red[0];
}

// ---------------------------------------------------------------------------
// The single-model adjoint kernel with its dynamic shared memory (above the
// 48 KB a launch gets without asking).
template <int LS, int PPL>
static cudaError_t launch_adj(const AdjParams &A, unsigned grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<LS, PPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ADJ_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    adjoint_kernel<LS, PPL><<<grid, PAIR_WARPS * 32, ADJ_SMEM_BYTES, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(AdjParams &A, int n_ctas, cudaStream_t s) {
    const int n_patch = A.npx * A.npy;
    patch_bounds_kernel<<<(n_patch * 32 + 127) / 128, 128, 0, s>>>(A);
    band_bounds_kernel<<<A.n_bands, 256, 0, s>>>(A);
    if (A.P.n_refl > 0) {
        const long long items = (long long)A.P.n_refl * A.n_bands;
        long long want = (items + PAIR_WARPS - 1) / PAIR_WARPS;
        const unsigned grid = (unsigned)(want < n_ctas ? want : n_ctas);
        if (cudaMemsetAsync(A.counter, 0, sizeof(unsigned), s) != cudaSuccess) return cudaGetLastError();
        const bool two = A.P.ppl == 2;
        cudaError_t e;
        if (A.lineshape == FDX_LINESHAPE_SINC)
            e = two ? launch_adj<FDX_LINESHAPE_SINC, 2>(A, grid, s) : launch_adj<FDX_LINESHAPE_SINC, 1>(A, grid, s);
        else if (A.lineshape == FDX_LINESHAPE_GAUSS)
            e = two ? launch_adj<FDX_LINESHAPE_GAUSS, 2>(A, grid, s) : launch_adj<FDX_LINESHAPE_GAUSS, 1>(A, grid, s);
        else
            e = two ? launch_adj<FDX_LINESHAPE_HOSEMANN, 2>(A, grid, s) : launch_adj<FDX_LINESHAPE_HOSEMANN, 1>(A, grid, s);
        if (e != cudaSuccess) return e;
        adjoint_reflection_kernel<<<(A.P.n_refl + 127) / 128, 128, 0, s>>>(A);
    }
    adjoint_globals_kernel<<<1, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <int PPL>
static cudaError_t launch_adj_batch(const BatchAdjParams &B, int n_ctas, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_batch_kernel<PPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ADJ_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    adjoint_batch_kernel<PPL><<<n_ctas, PAIR_WARPS * 32, ADJ_SMEM_BYTES, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_batch(const BatchAdjParams &B, int ppl, int n_ctas, cudaStream_t s) {
    return ppl == 2 ? launch_adj_batch<2>(B, n_ctas, s) : launch_adj_batch<1>(B, n_ctas, s);
}

cudaError_t launch_adjoint_post(AdjParams &A, cudaStream_t s) {
    if (A.P.n_refl > 0) adjoint_reflection_kernel<<<(A.P.n_refl + 127) / 128, 128, 0, s>>>(A);
    adjoint_globals_kernel<<<1, 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_bounds_only(AdjParams &A, cudaStream_t s) {
    const int n_patch = A.npx * A.npy;
    patch_bounds_kernel<<<(n_patch * 32 + 127) / 128, 128, 0, s>>>(A);
    band_bounds_kernel<<<A.n_bands, 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_globals_only(AdjParams &A, cudaStream_t s) {
    adjoint_globals_kernel<<<1, 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_sf_adjoint(SFAdjParams &p, cudaStream_t s) {
    dim3 grid((p.n_atoms + SFA_THREADS - 1) / SFA_THREADS, p.n_split);
    const size_t shm = sizeof(float) * SFA_TILE * p.n_elem;
    sf_adjoint_kernel<<<grid, SFA_THREADS, shm, s>>>(p);
    sf_adjoint_reduce_kernel<<<(p.n_atoms + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_loss(LossParams &p, cudaStream_t s) {
    const int nb = (int)((p.n + 255) / 256);
    loss_kernel<<<nb, 256, 0, s>>>(p);
    loss_final_kernel<<<1, 256, 0, s>>>(p, nb);
    return cudaGetLastError();
}

}  // namespace fdx
