// Scatter form of the projection: the paper's own pipeline (Sects. "Numerical
// evaluation: per-reflection shell quadrature", "Lorentz correction on a
// sampled reciprocal lattice", "Analytical Solution of the Ewald Diffraction
// Condition").  Each reflection is sampled on its shell, the intensity at
// every sample is the direct sum of Eq. direct_sum, the sample carries the
// Lorentz factor of Eq. lorentz, is rotated about the fiber axis into the
// diffraction condition with the closed form of Eqs. harmonic/solutions, and
// its two hits are added to the detector as spots of spot x spot pixels.
//
// Samples: normalised (x_r, x_1, x_2) in [-1, 1]^3 with quadrature weight q,
// shared by all reflections; for a reflection with radius r0 and support
// circumradius h_r = rho_B:  S = (r0 + x_r h_r) c (S^ + d1 e1 + d2 e2),
// d_i = x_i T, c = (1 + d^2)^(-1/2), volume element dV = q h_r T^2
// (r0 + x_r h_r)^2 c^3.  The pixel value is sum over hits of dV L I.
//
// Work decomposition: a warp evaluates 64 consecutive samples of one
// reflection (two per lane) with the same pair evaluation as the gather form
// (eval_core: block culling, live-node staging, packed walk); the query points
// are the samples, referred to the warp's sample nearest their centroid.  The
// per-sample Ewald rotation runs in float-float (one lane per sample) on seven
// projections of S, with Newton-refined reciprocals; the weights are FP32.
// The hits are added with FP64 atomics into an FP64 image that a last kernel
// rounds to FP32 (order effects far below FP32 resolution).
#include "fdx_pair.cuh"

namespace fdx {

static constexpr int SCAT_NODE_BUF = 288;
// Query points (samples) per lane of the scatter kernel.
static constexpr int SCAT_PPL = 2;

// Per-sample table from the normalised samples (FP64, once per call):
// (c - 1, c d1) and (c d2) as float-float, c, q T^2 c^3, x_r.
__global__ void scatter_table_kernel(ScatterParams p) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.n_s) return;
    const float4 x = p.samples[m];
    const double d1 = (double)x.y * p.T, d2 = (double)x.z * p.T;
    const double rho2 = d1 * d1 + d2 * d2;
    const double qn = sqrt(1.0 + rho2), c = 1.0 / qn;
    const double cm1 = -rho2 / (qn * (1.0 + qn));
    float4 a, b;
    split_double(cm1, a.x, a.y);
    split_double(c * d1, a.z, a.w);
    split_double(c * d2, b.x, b.y);
    b.z = (float)c;
    b.w = (float)((double)x.w * p.T * p.T * c * c * c);
    p.stab[3 * m] = a;
    p.stab[3 * m + 1] = b;
    p.stab[3 * m + 2] = make_float4(x.x, 0.0f, 0.0f, 0.0f);
}

// Per reflection: its frame vectors (S^, e1, e2) projected on the seven
// directions of the Ewald rotation and the detector map (n, u, v, b, u x n,
// v x n, b x n), so that every projection of a sample's S is three products
// of its frame coordinates; then r0, rho_B and rho_B / r0.  Computed in FP64,
// stored as float-float.
__global__ void scatter_proj_kernel(ScatterParams p) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.P.n_refl) return;
    const double *fr = p.frames + (size_t)r * 12;
    float2 *pr = p.proj + (size_t)r * SCAT_PROJ;
    float h, l;
    for (int j = 0; j < 7; ++j)
        for (int i = 0; i < 3; ++i) {
            split_double(fr[3 * i] * p.wdir[j][0] + fr[3 * i + 1] * p.wdir[j][1] + fr[3 * i + 2] * p.wdir[j][2], h, l);
            pr[3 * j + i] = make_float2(h, l);
        }
    split_double(fr[9], h, l);
    pr[21] = make_float2(h, l);
    split_double(fr[10], h, l);
    pr[22] = make_float2(h, l);
    pr[23] = make_float2((float)(fr[10] / fr[9]), 0.0f);
}

// Float-float reciprocal and reciprocal square root: the FP32 hardware value
// refined by one Newton step whose residual is formed in float-float, which
// squares the relative error (~1e-7 -> ~1e-14).  FP64 runs at a small
// fraction of the FP32 rate on this GPU, so the per-sample geometry is done in
// float-float (about 48 significant bits) instead.
__device__ __forceinline__ ff ffv(float2 v) { return ff{v.x, v.y}; }
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_rcp(ff x) {
    const float y = __frcp_rn(x.hi);
    const ff xy = ff_mul_f(x, y);
    const float r = (1.0f - xy.hi) - xy.lo;
    return fast_two_sum(y, y * r);
}
__device__ __forceinline__ ff ff_rsqrt(ff x) {
    const float y = rsqrtf(x.hi);
    const float y2 = y * y;
    const ff yy = {y2, fmaf(y, y, -y2)};  // y^2 exactly
    const ff xy2 = ff_mul(x, yy);
    const float r = (1.0f - xy2.hi) - xy2.lo;
    return fast_two_sum(y, 0.5f * y * r);
}
// floor of hi + lo (hi an integer and lo < 0: one below)
__device__ __forceinline__ float ff_floor(ff x) {
    float f = floorf(x.hi);
    if (f == x.hi && x.lo < 0.0f) f -= 1.0f;
    return f;
}

// Lorentz factor, Ewald rotation (both solutions) and splat of one sample,
// from its projections s = (S.n, S.u, S.v, S.b, S.(u x n), S.(v x n), S.(b x n))
// and |S| = rr, all float-float.  The rotation by phi about n is Rodrigues'
// formula, so for any direction w,  k_out . w = k_in . w + (S.w) cos phi
// + (S.(w x n)) sin phi + (n.w)(S.n)(1 - cos phi).
__device__ __forceinline__ void splat_sample(const ScatterParams &p, const ff *s, ff rr, float val) {
    const ff Z = s[0];
    // R^2 = |S|^2 - (S.n)^2 = (rr - Z)(rr + Z), without cancellation near the meridian
    const float R2 = ff_mul(ff_sub(rr, Z), ff_add(rr, Z)).hi;
    const float R = sqrtf(fmaxf(R2, 0.0f));
    const float dl = (float)p.delta_L;
    const double v = (double)(val * (dl / (R + dl)));  // Eq. lorentz (a weight: FP32 is enough)
    // Eqs. harmonic / solutions: P cos(phi) + Q sin(phi) = E with
    // P = k_in.S - D, Q = k_in.(n x S), D = (k_in.n)(n.S), E = -|S|^2/2 - D
    const ff D = ff_mul(ffv(p.kn_f), Z);
    const ff E = ff_sub(ff_mul_f(ff_mul(rr, rr), -0.5f), D);
    const ff Pp = ff_sub(ff_mul(ffv(p.il_f), s[3]), D), Qp = ff_mul(ffv(p.il_f), s[6]);
    const ff rpq2 = ff_add(ff_mul(Pp, Pp), ff_mul(Qp, Qp));
    if (!(rpq2.hi > 0.0f)) return;
    const ff inv = ff_rsqrt(rpq2);
    const ff cd = ff_mul(E, inv);
    // Eq. valid: no rotation reaches the Ewald sphere unless |cos(delta)| <= 1
    if (!(fabsf(cd.hi) < 1.0f || (fabsf(cd.hi) == 1.0f && cd.hi * cd.lo <= 0.0f))) return;
    // phi = phi0 +- delta with cos(phi0), sin(phi0) = (P, Q)/rpq, cos(delta) = cd
    const ff c0 = ff_mul(Pp, inv), s0 = ff_mul(Qp, inv);
    const ff t = ff_mul(ff_add_f(ff_neg(cd), 1.0f), ff_add_f(cd, 1.0f));
    const ff sd = t.hi > 1e-30f ? ff_mul(t, ff_rsqrt(t)) : ff{0.0f, 0.0f};
    const ff c0cd = ff_mul(c0, cd), s0sd = ff_mul(s0, sd), s0cd = ff_mul(s0, cd), c0sd = ff_mul(c0, sd);
    for (int br = 0; br < 2; ++br) {
        const ff cp = br == 0 ? ff_sub(c0cd, s0sd) : ff_add(c0cd, s0sd);
        const ff sp = br == 0 ? ff_add(s0cd, c0sd) : ff_sub(s0cd, c0sd);
        const ff zc = ff_mul(Z, ff_add_f(ff_neg(cp), 1.0f));
        const ff kb = ff_add(ff_add(ffv(p.kw_f[2]), ff_mul(s[3], cp)), ff_add(ff_mul(s[6], sp), ff_mul(ffv(p.nw_f[2]), zc)));
        if (!(kb.hi > 0.0f)) continue;
        const ff ku = ff_add(ff_add(ffv(p.kw_f[0]), ff_mul(s[1], cp)), ff_add(ff_mul(s[4], sp), ff_mul(ffv(p.nw_f[0]), zc)));
        const ff kv = ff_add(ff_add(ffv(p.kw_f[1]), ff_mul(s[2], cp)), ff_add(ff_mul(s[5], sp), ff_mul(ffv(p.nw_f[1]), zc)));
        const ff ib = ff_mul(ffv(p.dp_f), ff_rcp(kb));
        const float fi = ff_floor(ff_add(ff_mul(ku, ib), ffv(p.hx_f)));
        const float fj = ff_floor(ff_add(ff_mul(kv, ib), ffv(p.hy_f)));
        // detector spot: the spot x spot block centred on the hit pixel
        const int half = (p.spot - 1) >> 1;
        if (!(fi >= (float)-half) || !(fj >= (float)-half) || fi >= (float)(p.P.nx + half) ||
            fj >= (float)(p.P.ny + half))
            continue;
        const int ci = (int)fi, cj = (int)fj;
        if (half == 0) {
            if (FDX_IN_BOUNDS((size_t)cj * p.P.nx + (size_t)ci, (long long)p.P.nx * p.P.ny, DBG_SPLAT))
                atomicAdd(&p.img64[(size_t)cj * p.P.nx + (size_t)ci], v);
            continue;
        }
        const double share = v / (double)(p.spot * p.spot);
        for (int qj = max(cj - half, 0); qj <= min(cj + half, p.P.ny - 1); ++qj)
            for (int qi = max(ci - half, 0); qi <= min(ci + half, p.P.nx - 1); ++qi)
                if (FDX_IN_BOUNDS((size_t)qj * p.P.nx + (size_t)qi, (long long)p.P.nx * p.P.ny, DBG_SPLAT))
                    atomicAdd(&p.img64[(size_t)qj * p.P.nx + (size_t)qi], share);
    }
}

// (S - D)/r0 of sample m in the reflection frame: (1 + rho) (c, c d1, c d2) - (1, 0, 0),
// rho = x_r h_r / r0, float-float.
__device__ __forceinline__ void sample_offset(const ScatterParams &p, int m, float rho_r, ff &u0, ff &u1, ff &u2) {
    const float4 ta = p.stab[3 * m], tb = p.stab[3 * m + 1], tc = p.stab[3 * m + 2];
    const float rho = tc.x * rho_r;
    u0 = ff_add_f(ff{ta.x, ta.y}, rho * tb.z);
    u1 = ff_add_f(ff{ta.z, ta.w}, rho * ta.z);
    u2 = ff_add_f(ff{tb.x, tb.y}, rho * tb.x);
}

// A warp evaluates 32 SCAT_PPL consecutive samples of one reflection: sample
// chunk * 32 SCAT_PPL + 32 p + lane is the lane's query point p, so that the
// packed walk has SCAT_PPL query points per node pair (with bricks of 32
// samples, a warp's points are SCAT_PPL adjacent bricks).
template <int LS, int MODE>
__global__ void __launch_bounds__(PAIR_WARPS * 32, 4) scatter_kernel(ScatterParams p) {
    constexpr int PPL = SCAT_PPL, NW = 32 * PPL;
    __shared__ float4 s_nodes[PAIR_WARPS][SCAT_NODE_BUF];
    __shared__ float4 s_sc[PAIR_WARPS][(LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? SCAT_NODE_BUF : 1];
    __shared__ float4 s_sc2[PAIR_WARPS][(LS == FDX_LINESHAPE_HOSEMANN && MODE == MODE_FWD) ? SCAT_NODE_BUF / 2 : 1];
    __shared__ float s_rec[PAIR_WARPS][REC_SIZE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_chunks = (p.n_s + NW - 1) / NW;
    const long long item = (long long)blockIdx.x * PAIR_WARPS + warp;
    if (item >= (long long)p.P.n_refl * n_chunks) return;
    const int r = (int)(item / n_chunks), chunk = (int)(item % n_chunks);
    float *rec = s_rec[warp];
    load_record(p.P.recs, r, rec, lane);
    const float2 *pr = p.proj + (size_t)r * SCAT_PROJ;
    const float rho_r = pr[23].x;

    const int n_valid = min(NW, p.n_s - chunk * NW);
    bool valid[PPL];
    ff u0[PPL], u1[PPL], u2[PPL];
    float cx = 0.0f, cy = 0.0f, cz = 0.0f;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        valid[q] = 32 * q + lane < n_valid;
        u0[q] = u1[q] = u2[q] = ff{0.0f, 0.0f};
        if (valid[q] && FDX_IN_BOUNDS(chunk * NW + 32 * q + lane, p.n_s, DBG_SPLAT)) {
            sample_offset(p, chunk * NW + 32 * q + lane, rho_r, u0[q], u1[q], u2[q]);
            cx += u0[q].hi, cy += u1[q].hi, cz += u2[q].hi;
        }
    }
    // reference: the valid sample nearest the centroid of the warp's samples
    // (any order of the samples is correct; neighbours in a warp cull best)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cx += __shfl_xor_sync(FDX_FULL_MASK, cx, o);
        cy += __shfl_xor_sync(FDX_FULL_MASK, cy, o);
        cz += __shfl_xor_sync(FDX_FULL_MASK, cz, o);
    }
    const float inv_n = 1.0f / (float)n_valid;
    cx *= inv_n, cy *= inv_n, cz *= inv_n;
    // squared distances are >= 0, so their bit patterns order like the values;
    // the low 6 bits carry the point's index in the warp (ties and near-ties go
    // to either point)
    unsigned key = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        const float dx = u0[q].hi - cx, dy = u1[q].hi - cy, dz = u2[q].hi - cz;
        if (valid[q])
            key = min(key, (__float_as_uint(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) & ~63u) | (unsigned)(32 * q + lane));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) key = min(key, __shfl_xor_sync(FDX_FULL_MASK, key, o));
    const int rl = (int)(key & 31u), rq = (int)((key & 63u) >> 5);
    ff c0 = u0[0], c1 = u1[0], c2 = u2[0];
#pragma unroll
    for (int q = 1; q < PPL; ++q)
        if (rq == q) c0 = u0[q], c1 = u1[q], c2 = u2[q];
    const ff v0 = {__shfl_sync(FDX_FULL_MASK, c0.hi, rl), __shfl_sync(FDX_FULL_MASK, c0.lo, rl)};
    const ff v1 = {__shfl_sync(FDX_FULL_MASK, c1.hi, rl), __shfl_sync(FDX_FULL_MASK, c1.lo, rl)};
    const ff v2 = {__shfl_sync(FDX_FULL_MASK, c2.hi, rl), __shfl_sync(FDX_FULL_MASK, c2.lo, rl)};
    QueryPts<PPL> qp;
#pragma unroll
    for (int q = 0; q < PPL; ++q) {
        qp.valid[q] = valid[q];
        qp.P[q][0] = u0[q].hi, qp.P[q][1] = u1[q].hi, qp.P[q][2] = u2[q].hi;
        const float w0 = (u0[q].hi - v0.hi) + (u0[q].lo - v0.lo);
        const float w1 = (u1[q].hi - v1.hi) + (u1[q].lo - v1.lo);
        const float w2 = (u2[q].hi - v2.hi) + (u2[q].lo - v2.lo);
#pragma unroll
        for (int i = 0; i < 3; ++i)
            qp.tau[q][i] =
                valid[q] ? fmaf(rec[REC_H + i], w0, fmaf(rec[REC_E1 + i], w1, rec[REC_E2 + i] * w2)) : 1.0e4f;
    }
    qp.dP[0] = v0, qp.dP[1] = v1, qp.dP[2] = v2;

    PairAcc pa[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) clear(pa[q]);
    const bool any = eval_core<LS, MODE, SCAT_NODE_BUF, PPL>(p.P, qp, rec, s_nodes[warp], nullptr, s_sc[warp],
                                                             s_sc2[warp], lane, pa);
    if (MODE == MODE_CNT) {
        unsigned long long c = 0ull;
        if (any) {
#pragma unroll
            for (int q = 0; q < PPL; ++q) c += (unsigned long long)pa[q].cnt;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FDX_FULL_MASK, c, o);
        if (lane == 0 && c) atomicAdd(p.count, c);
        return;
    }
    if (!any) return;
    float Iq[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) Iq[q] = valid[q] ? rec[REC_FR] * (pa[q].s0.hi + pa[q].s0.lo) : 0.0f;
    const ff rr0 = ffv(pr[21]), rr1 = ffv(pr[22]);
#pragma unroll 1
    for (int q = 0; q < PPL; ++q) {
        float I = 0.0f;
#pragma unroll
        for (int k = 0; k < PPL; ++k)
            if (k == q) I = Iq[k];
        if (!(I != 0.0f)) continue;
        const int m = chunk * NW + 32 * q + lane;
        if (!FDX_IN_BOUNDS(m, p.n_s, DBG_SPLAT)) continue;
        // projections of S = (r0 + x_r h_r) (c, c d1, c d2) in the reflection frame
        // from the frame projections and the sample table, all float-float (the
        // hit position of a sample near the edge of the Ewald condition is
        // sensitive to S), and the volume element (a weight: FP32)
        const float4 ta = p.stab[3 * m], tb = p.stab[3 * m + 1], tc = p.stab[3 * m + 2];
        const ff rr = ff_add(rr0, ff_mul_f(rr1, tc.x));
        const ff U0 = ff_add_f(ff{ta.x, ta.y}, 1.0f), U1 = {ta.z, ta.w}, U2 = {tb.x, tb.y};
        ff sp[7];
#pragma unroll
        for (int j = 0; j < 7; ++j)
            sp[j] = ff_mul(rr, ff_add(ff_add(ff_mul(U0, ffv(pr[3 * j])), ff_mul(U1, ffv(pr[3 * j + 1]))),
                                      ff_mul(U2, ffv(pr[3 * j + 2]))));
        const float rrf = rr.hi + rr.lo;
        const float dV = tb.w * pr[22].x * rrf * rrf;
        splat_sample(p, sp, rr, dV * I);
    }
}

__global__ void scatter_finish_kernel(const double *img64, float *image, long long n) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) image[k] = (float)img64[k];
}

template <int LS>
static void launch_scatter_ls(const ScatterParams &p, bool count_mode, cudaStream_t s) {
    const long long items = (long long)p.P.n_refl * ((p.n_s + 32 * SCAT_PPL - 1) / (32 * SCAT_PPL));
    const unsigned grid = (unsigned)((items + PAIR_WARPS - 1) / PAIR_WARPS);
    if (grid == 0) return;
    if (count_mode)
        scatter_kernel<LS, MODE_CNT><<<grid, PAIR_WARPS * 32, 0, s>>>(p);
    else
        scatter_kernel<LS, MODE_FWD><<<grid, PAIR_WARPS * 32, 0, s>>>(p);
}

cudaError_t launch_scatter(const ScatterParams &p, int lineshape, bool count_mode, cudaStream_t s) {
    scatter_table_kernel<<<(p.n_s + 127) / 128, 128, 0, s>>>(p);
    scatter_proj_kernel<<<(p.P.n_refl + 127) / 128, 128, 0, s>>>(p);
    if (lineshape == FDX_LINESHAPE_HOSEMANN)
        launch_scatter_ls<FDX_LINESHAPE_HOSEMANN>(p, count_mode, s);
    else if (lineshape == FDX_LINESHAPE_GAUSS)
        launch_scatter_ls<FDX_LINESHAPE_GAUSS>(p, count_mode, s);
    else
        launch_scatter_ls<FDX_LINESHAPE_SINC>(p, count_mode, s);
    if (!count_mode) {
        const long long n = (long long)p.P.nx * p.P.ny;
        scatter_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.img64, p.image, n);
    }
    return cudaGetLastError();
}

}  // namespace fdx
