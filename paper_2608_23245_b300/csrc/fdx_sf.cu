// Structure factors by direct summation (Eq. structure_factor):
//   F_hkl = sum_j occ_j f_{e_j}(s) exp(-B_j s^2/4) exp(2 pi i (h x_j + k y_j + l z_j)).
//
// Phase reduction is exact: fractional coordinates are stored as 32-bit
// fixed-point turns X = round(x 2^32) mod 2^32, so h X + k Y + l Z computed in
// wrapping uint32 arithmetic is the phase modulo one turn with no rounding
// beyond the 2^-32 quantisation of x.  The top two bits pick the quadrant;
// the remainder (|r| <= 1/8 turn) is converted to float exactly and fed to
// polynomials for sin(2 pi r), cos(2 pi r) fitted by fit_poly.py.
//
// Work decomposition: one thread per reflection, atoms staged through shared
// memory in tiles; the atom list is split across blockIdx.y so that small
// reflection counts still fill the GPU.  Each split writes a float-float
// partial (re, im) to the workspace; a second kernel adds the splits in a
// fixed order (deterministic, no atomics) and forms M = |F|^2 P DW.
// Sums: 8 terms in plain FP32, then folded into a float-float accumulator.
#include "fdx_internal.cuh"

namespace fdx {

static constexpr int SF_THREADS = 128;
static constexpr int SF_TILE = 256;  // atoms per shared-memory tile (multiple of 8)
static constexpr int SF_MAX_ELEM = 64;

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

__device__ __forceinline__ void sincos_turns(unsigned u, float &s, float &c) {
    // quadrant and remainder in [-2^29, 2^29)
    const unsigned qd = (u + 0x20000000u) >> 30;
    const int rem = (int)(u - (qd << 30));
    // exact int -> float of the 30-bit remainder via two 'magic number' conversions
    const int rh = rem >> 8, rl = rem & 255;
    const float fh = __int_as_float(0x4B400000 + rh) - 12582912.0f;
    const float fl = __int_as_float(0x4B000000 + rl) - 8388608.0f;
    const float r = fmaf(fh, 5.9604644775390625e-08f /* 2^-24 */, fl * 2.3283064365386963e-10f /* 2^-32 */);
    const float Sc[4] = FDX_SIN2PI_C;
    const float Cc[5] = FDX_COS2PI_C;
    const float r2 = r * r;
    const float sn = r * horner(Sc, r2);
    const float cs = horner(Cc, r2);
    // rotate by qd quarter turns
    const float s1 = (qd & 1) ? cs : sn;
    const float c1 = (qd & 1) ? -sn : cs;
    s = (qd & 2) ? -s1 : s1;
    c = (qd & 2) ? -c1 : c1;
}

__global__ void __launch_bounds__(SF_THREADS) sf_main_kernel(SFParams p) {
    __shared__ uint4 s_q[SF_TILE];
    __shared__ float2 s_w[SF_TILE];
    __shared__ float s_fe[SF_MAX_ELEM][SF_THREADS];

    const int r = blockIdx.x * SF_THREADS + threadIdx.x;
    const bool active = r < p.n_refl;
    int h = 0, k = 0, l = 0;
    if (active) h = p.hkl[3 * r], k = p.hkl[3 * r + 1], l = p.hkl[3 * r + 2];
    double D[3];
    for (int q = 0; q < 3; ++q) D[q] = h * p.As[q] + k * p.As[3 + q] + l * p.As[6 + q];
    const double s2d = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    const float s2 = (float)s2d;
    for (int e = 0; e < p.n_elem; ++e) {
        const float *f = p.ff + 9 * e;
        double v = f[8];
        for (int i = 0; i < 4; ++i) v += (double)f[i] * exp(-(double)f[4 + i] * s2d * 0.25);
        s_fe[e][threadIdx.x] = (float)v;
    }
    const unsigned uh = (unsigned)h, uk = (unsigned)k, ul = (unsigned)l;

    const int a_begin = blockIdx.y * p.atoms_per_split;
    const int a_end = min(p.n_atoms, a_begin + p.atoms_per_split);
    ff re = {0.0f, 0.0f}, im = {0.0f, 0.0f};
    for (int t0 = a_begin; t0 < a_end; t0 += SF_TILE) {
        const int cnt = min(SF_TILE, a_end - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < SF_TILE; i += SF_THREADS) {
            if (i < cnt) {
                s_q[i] = p.atoms_q[t0 + i];
                s_w[i] = p.atoms_w[t0 + i];
            } else {
                s_q[i] = make_uint4(0u, 0u, 0u, 0u);
                s_w[i] = make_float2(0.0f, -INFINITY);  // zero amplitude padding
            }
        }
        __syncthreads();
        const int cnt8 = (cnt + 7) & ~7;
        for (int i0 = 0; i0 < cnt8; i0 += 8) {
            float bre = 0.0f, bim = 0.0f;
#pragma unroll
            for (int i = i0; i < i0 + 8; ++i) {
                const uint4 q = s_q[i];
                const float2 w = s_w[i];
                const unsigned ph = uh * q.x + uk * q.y + ul * q.z;
                float sn, cs;
                sincos_turns(ph, sn, cs);
                const float amp = s_fe[q.w][threadIdx.x] * exp2f(fmaf(w.x, s2, w.y));
                bre = fmaf(amp, cs, bre);
                bim = fmaf(amp, sn, bim);
            }
            re = ff_add_f(re, bre);
            im = ff_add_f(im, bim);
        }
    }
    if (active) p.partial[(size_t)blockIdx.y * p.n_refl + r] = make_float4(re.hi, re.lo, im.hi, im.lo);
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

cudaError_t launch_sf_pack(SFParams &p, cudaStream_t s) {
    sf_pack_atoms_kernel<<<(p.n_atoms + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_structure_factors(SFParams &p, cudaStream_t s) {
    if (p.n_refl <= 0) return cudaSuccess;
    sf_pack_atoms_kernel<<<(p.n_atoms + 127) / 128, 128, 0, s>>>(p);
    dim3 grid((p.n_refl + SF_THREADS - 1) / SF_THREADS, p.n_split);
    sf_main_kernel<<<grid, SF_THREADS, 0, s>>>(p);
    sf_reduce_kernel<<<(p.n_refl + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fdx
