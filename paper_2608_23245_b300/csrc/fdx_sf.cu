// Structure factors by direct summation (Eq. structure_factor):
//   F_hkl = sum_j occ_j f_{e_j}(s) exp(-B_j s^2/4) exp(2 pi i (h x_j + k y_j + l z_j)).
//
// Phase reduction is exact: fractional coordinates are stored as 32-bit
// fixed-point turns X = round(x 2^32) mod 2^32, so h X + k Y + l Z computed in
// wrapping uint32 arithmetic is the phase modulo one turn with no rounding
// beyond the 2^-32 quantisation of x.  The phase is split into a half turn
// (a sign on the amplitude) and a remainder |r| <= 1/4 turn, converted to
// float once and fed to polynomials for sin(2 pi r), cos(2 pi r) fitted by
// fit_poly.py.
//
// Work decomposition: one thread per 4 consecutive reflections, evaluated as
// two packed FP32 pairs; atoms staged through shared memory in tiles; the
// atom list is split across blockIdx.y (sf_plan: whole waves of resident
// CTAs).  Each split writes a float-float partial (re, im) to the workspace; a
// second kernel adds the splits in a fixed order (deterministic, no atomics)
// and forms M = |F|^2 P DW.  Sums: 16 terms in plain FP32, then folded into a
// float-float accumulator.
#include "fdx_internal.cuh"

namespace fdx {

static constexpr int SF_THREADS = 128;
static constexpr int SF_TILE = 256;  // atoms per shared-memory tile (multiple of 16)

// Pack atoms: fixed-point coordinates, element, and the exponent terms
// Bq = -B log2(e) / 4 (so that exp(-B s^2/4) = exp2(Bq s^2)) and log2(occ).
__global__ void sf_pack_atoms_kernel(SFParams p) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.n_atoms) return;
    unsigned q[3];
    for (int c = 0; c < 3; ++c) {
        const double x = p.frac[3 * j + c];
        const double f = x - floor(x);  // [0, 1)
        const unsigned long long u = (unsigned long long)llrint(f * 4294967296.0);
        q[c] = (unsigned)(u & 0xffffffffull);
    }
    const unsigned e = (unsigned)p.elem[j];
    const bool bad = e >= (unsigned)p.n_elem;  // out-of-range element: poison F with NaN, never index past the table
    p.atoms_q[j] = make_uint4(q[0], q[1], q[2], bad ? 0u : e);
    const double occ = p.occ ? (double)p.occ[j] : 1.0;
    const float lo = bad ? __int_as_float(0x7fc00000) : (occ > 0.0 ? (float)log2(occ) : -INFINITY);
    p.atoms_w[j] = make_float2((float)(-(double)p.B[j] * 1.4426950408889634 / 4.0), lo);
}

// ex2.approx with flush-to-zero: one SFU op (amplitudes below 2^-126 are 0).
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Phase -> (sin, cos) for two reflections at once, on the half turn.  With
// the phase u (uint32 turns), rem = u sign-extended from its low 31 bits is
// u mod 1/2 turn in [-2^30, 2^30), and bit 31 of u - rem is the half turn (it
// flips the sign of both sin and cos; half_sign() returns it for the caller
// to apply to the amplitude).  r = rem 2^-32 in [-1/4, 1/4) turn (one
// rounding to 24 bits in the int -> float conversion: <= 2^-26 turn) feeds the
// half-turn polynomials.
__device__ __forceinline__ int half_rem(unsigned u) { return ((int)(u << 1)) >> 1; }
__device__ __forceinline__ unsigned half_sign(unsigned u, int rem) { return (u - (unsigned)rem) & 0x80000000u; }

__device__ __forceinline__ void sincos_half2(int rem0, int rem1, float2 &sn, float2 &cs) {
    const float2 r = __fmul2_rn(make_float2(__int2float_rn(rem0), __int2float_rn(rem1)),
                                make_float2(2.3283064365386963e-10f, 2.3283064365386963e-10f));
    const float2 r2 = __fmul2_rn(r, r);
    const float Sc[5] = FDX_SIN2PI_H_C;
    const float Cc[6] = FDX_COS2PI_H_C;
    float2 S = make_float2(Sc[4], Sc[4]);
#pragma unroll
    for (int k = 3; k >= 0; --k) S = __ffma2_rn(S, r2, make_float2(Sc[k], Sc[k]));
    float2 C = make_float2(Cc[5], Cc[5]);
#pragma unroll
    for (int k = 4; k >= 0; --k) C = __ffma2_rn(C, r2, make_float2(Cc[k], Cc[k]));
    sn = __fmul2_rn(r, S);
    cs = C;
}

// One thread per SF_RPT = 4 consecutive reflections (two packed pairs), atoms
// staged through shared memory; per atom and reflection: exact phase (3 IMAD
// in wrapping uint32),
// half-turn sin/cos, amplitude occ f_e(s) exp(-B s^2/4) = f_e(s) 2^(Bq s^2 +
// log2 occ) with one SFU exp2, half-turn sign folded into the amplitude.
// 16 atoms are summed in FP32, then folded into float-float.
static constexpr int SF_RPT = 4;
static constexpr int SF_FOLD = 16;  // atoms per FP32 partial sum (SF_TILE is a multiple)

__global__ void __launch_bounds__(SF_THREADS) sf_main_kernel(SFParams p) {
    __shared__ uint4 s_q[SF_TILE];
    __shared__ float4 s_w[SF_TILE];  // (Bq, Bq, log2 occ, log2 occ)
    extern __shared__ float4 s_fe[];  // [n_elem][SF_THREADS]: f_e(s) of this thread's 4 reflections

    const int r0 = (blockIdx.x * SF_THREADS + threadIdx.x) * SF_RPT;
    unsigned h[SF_RPT], k[SF_RPT], l[SF_RPT];
    float s2[SF_RPT];
#pragma unroll
    for (int j = 0; j < SF_RPT; ++j) {
        const int r = r0 + j;
        int hh = 0, kk = 0, ll = 0;
        if (r < p.n_refl) hh = p.hkl[3 * r], kk = p.hkl[3 * r + 1], ll = p.hkl[3 * r + 2];
        h[j] = (unsigned)hh, k[j] = (unsigned)kk, l[j] = (unsigned)ll;
        double D[3];
        for (int q = 0; q < 3; ++q) D[q] = hh * p.As[q] + kk * p.As[3 + q] + ll * p.As[6 + q];
        s2[j] = (float)(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    }
    for (int e = 0; e < p.n_elem; ++e) {
        const float *f = p.ff + 9 * e;
        float fe[SF_RPT];
#pragma unroll
        for (int j = 0; j < SF_RPT; ++j) {  // FP32 (expf, a few ulp): FP64 here would cost more than the sum
            float v = f[8];
            for (int i = 0; i < 4; ++i) v = fmaf(f[i], expf(-0.25f * f[4 + i] * s2[j]), v);
            fe[j] = v;
        }
        s_fe[e * SF_THREADS + threadIdx.x] = make_float4(fe[0], fe[1], fe[2], fe[3]);
    }
    const float2 s2a = make_float2(s2[0], s2[1]), s2b = make_float2(s2[2], s2[3]);

    const int a_begin = blockIdx.y * p.atoms_per_split;
    const int a_end = min(p.n_atoms, a_begin + p.atoms_per_split);
    ff re[SF_RPT], im[SF_RPT];
#pragma unroll
    for (int j = 0; j < SF_RPT; ++j) re[j] = im[j] = ff{0.0f, 0.0f};
    for (int t0 = a_begin; t0 < a_end; t0 += SF_TILE) {
        const int cnt = min(SF_TILE, a_end - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < SF_TILE; i += SF_THREADS) {
            if (i < cnt) {
                s_q[i] = p.atoms_q[t0 + i];
                const float2 w = p.atoms_w[t0 + i];
                s_w[i] = make_float4(w.x, w.x, w.y, w.y);
            } else {
                s_q[i] = make_uint4(0u, 0u, 0u, 0u);
                s_w[i] = make_float4(0.0f, 0.0f, -INFINITY, -INFINITY);  // zero amplitude padding
            }
        }
        __syncthreads();
        const int cntf = (cnt + SF_FOLD - 1) / SF_FOLD * SF_FOLD;
        for (int i0 = 0; i0 < cntf; i0 += SF_FOLD) {
            float2 ra = make_float2(0.0f, 0.0f), ia = ra, rb = ra, ib = ra;
#pragma unroll 4
            for (int i = i0; i < i0 + SF_FOLD; ++i) {
                const uint4 q = s_q[i];
                const float4 w = s_w[i];
                const float4 fe = s_fe[q.w * SF_THREADS + threadIdx.x];
                unsigned v[SF_RPT], sg[SF_RPT];
                int rm[SF_RPT];
#pragma unroll
                for (int j = 0; j < SF_RPT; ++j) {
                    v[j] = h[j] * q.x + k[j] * q.y + l[j] * q.z;
                    rm[j] = half_rem(v[j]);
                    sg[j] = half_sign(v[j], rm[j]);
                }
                float2 sa, ca, sb, cb;
                sincos_half2(rm[0], rm[1], sa, ca);
                sincos_half2(rm[2], rm[3], sb, cb);
                const float2 xa = __ffma2_rn(make_float2(w.x, w.y), s2a, make_float2(w.z, w.w));
                const float2 xb = __ffma2_rn(make_float2(w.x, w.y), s2b, make_float2(w.z, w.w));
                float2 aa = __fmul2_rn(make_float2(fe.x, fe.y), make_float2(ex2_ftz(xa.x), ex2_ftz(xa.y)));
                float2 ab = __fmul2_rn(make_float2(fe.z, fe.w), make_float2(ex2_ftz(xb.x), ex2_ftz(xb.y)));
                // half-turn sign of (sin, cos) onto the amplitude
                aa.x = __uint_as_float(__float_as_uint(aa.x) ^ sg[0]);
                aa.y = __uint_as_float(__float_as_uint(aa.y) ^ sg[1]);
                ab.x = __uint_as_float(__float_as_uint(ab.x) ^ sg[2]);
                ab.y = __uint_as_float(__float_as_uint(ab.y) ^ sg[3]);
                ra = __ffma2_rn(aa, ca, ra);
                ia = __ffma2_rn(aa, sa, ia);
                rb = __ffma2_rn(ab, cb, rb);
                ib = __ffma2_rn(ab, sb, ib);
            }
            re[0] = ff_add_f(re[0], ra.x), re[1] = ff_add_f(re[1], ra.y);
            re[2] = ff_add_f(re[2], rb.x), re[3] = ff_add_f(re[3], rb.y);
            im[0] = ff_add_f(im[0], ia.x), im[1] = ff_add_f(im[1], ia.y);
            im[2] = ff_add_f(im[2], ib.x), im[3] = ff_add_f(im[3], ib.y);
        }
    }
#pragma unroll
    for (int j = 0; j < SF_RPT; ++j)
        if (r0 + j < p.n_refl)
            p.partial[(size_t)blockIdx.y * p.n_refl + r0 + j] = make_float4(re[j].hi, re[j].lo, im[j].hi, im[j].lo);
}

// Sum the splits in order; F = (re, im); M = |F|^2 P DW (FP64 scalars).
__global__ void sf_reduce_kernel(SFParams p) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.n_refl) return;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < p.n_split; ++s) {
        const float4 v = p.partial[(size_t)s * p.n_refl + r];
        re += (double)v.x + (double)v.y;
        im += (double)v.z + (double)v.w;
    }
    p.F_out[2 * r] = (float)re;
    p.F_out[2 * r + 1] = (float)im;
    if (p.M_out) {
        double P = 1.0, dw = 0.0;
        if (p.has_br) {
            for (int i = 0; i < 3; ++i) {
                const double hi = (double)p.hkl[3 * r + i];
                const double x = FDX_PI * FDX_PI * p.g[i] * p.g[i] * hi * hi;
                if (p.intensity_model == FDX_INTENSITY_HOSEMANN) P *= 1.0 / cosh(2.0 * x);
                const double sa = hi / p.alen[i];  // S . a^_i at the reflection
                dw += p.Bax[i] * sa * sa;
            }
        }
        p.M_out[r] = (float)((re * re + im * im) * P * exp(-0.25 * dw));
    }
}

// Split of the atom list across blockIdx.y.  A CTA's time is proportional to
// its atoms (plus a fixed set-up of about SF_TILE / 4 atoms), and CTAs run in
// waves of `slots` (resident CTAs on the whole GPU), so the split count n
// minimises waves(n) x (atoms per split + set-up); splits hold a multiple of
// SF_TILE atoms, and there are at most max_split of them.
void sf_plan(int n_atoms, int n_refl, int n_elem, int max_split, int &n_split, int &per) {
    static int s_sm = 0;
    if (s_sm == 0) {
        int dev = 0, v = 148;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            s_sm = v;
        else
            s_sm = 148;
    }
    static size_t s_shm = (size_t)-1;
    static int s_per_sm = 1;
    const size_t shm = sizeof(float4) * SF_THREADS * (size_t)(n_elem > 0 ? n_elem : 1);
    if (shm != s_shm) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sf_main_kernel, SF_THREADS, shm) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        s_shm = shm, s_per_sm = v;
    }
    const int per_sm = s_per_sm;
    const long long slots = (long long)s_sm * per_sm;
    const long long refl_blocks = (n_refl + SF_THREADS * SF_RPT - 1) / (SF_THREADS * SF_RPT);
    const int tiles = (n_atoms + SF_TILE - 1) / SF_TILE;
    int best_n = 1, best_per = tiles * SF_TILE;
    double best_t = -1.0;
    for (int want = 1; want <= max_split && want <= tiles; ++want) {
        const int pt = (tiles + want - 1) / want;  // tiles per split
        const int n = (tiles + pt - 1) / pt;
        const long long ctas = (long long)n * refl_blocks;
        const long long waves = (ctas + slots - 1) / slots;
        const double t = (double)waves * (pt * SF_TILE + SF_TILE / 4);
        if (best_t < 0.0 || t < 0.98 * best_t) best_t = t, best_n = n, best_per = pt * SF_TILE;
    }
    n_split = best_n, per = best_per;
}

cudaError_t launch_sf_pack(SFParams &p, cudaStream_t s) {
    sf_pack_atoms_kernel<<<(p.n_atoms + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_structure_factors(SFParams &p, cudaStream_t s) {
    if (p.n_refl <= 0) return cudaSuccess;
    sf_pack_atoms_kernel<<<(p.n_atoms + 127) / 128, 128, 0, s>>>(p);
    dim3 grid((p.n_refl + SF_THREADS * SF_RPT - 1) / (SF_THREADS * SF_RPT), p.n_split);
    const size_t shm = sizeof(float4) * SF_THREADS * (size_t)p.n_elem;
    if (shm > 48 * 1024) {
        static size_t s_opted = 0;  // largest opt-in so far (the attribute is per function, process-wide)
        if (shm > s_opted) {
            if (cudaFuncSetAttribute(sf_main_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess)
                return cudaGetLastError();
            s_opted = shm;
        }
    }
    sf_main_kernel<<<grid, SF_THREADS, shm, s>>>(p);
    sf_reduce_kernel<<<(p.n_refl + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fdx
