// Structure factors by direct summation (Eq. structure_factor):
//   F_hkl = sum_j occ_j f_{e_j}(s) exp(-B_j s^2/4) exp(2 pi i (h x_j + k y_j + l z_j)).
//
// Phase reduction is exact: fractional coordinates are stored as 32-bit
// fixed-point turns X = round(x 2^32) mod 2^32, so h X + k Y + l Z computed in
// wrapping uint32 arithmetic is the phase modulo one turn with no rounding
// beyond the 2^-32 quantisation of x.  A phase is split into a half turn (a
// sign) and a remainder |r| <= 1/4 turn, converted to float once and fed to
// polynomials for sin(2 pi r), cos(2 pi r) fitted by fit_poly.py.
//
// Runs of l.  Reflections are processed in groups of up to four with equal
// (h, k) and consecutive l (l = l0 .. l0 + 3), so that per atom
//   exp(2 pi i (h.x + (l0 + j) z)) = exp(2 pi i (h.x + l0 z)) exp(2 pi i j z):
// one exact phase and one polynomial sin/cos per group and atom, the other
// three terms by a complex rotation with exp(2 pi i j z), j = 1, 2, 3, which
// depends on the atom only and is tabulated (each from its own exact phase
// j Z) when the atom tile is staged.  A group starts at every run start of
// the reflection list and wherever l is a multiple of 4; three small kernels
// (flags and counts, a scan, a scatter) list the group starts, so any
// reflection order is valid and the lexicographic order of fdx_reflections
// gives runs of tens of reflections.
//
// Work decomposition: one thread per two groups (8 reflections, evaluated as
// packed FP32 pairs across the two groups); the atoms are packed sorted by
// element, each element's run padded to whole 64-atom chunks, so that the
// form factor f_e(s) multiplies a chunk's sum once instead of every term;
// atoms staged through shared memory in tiles; the atom list is cut into
// n_split splits; CTAs loop over (256-group block, split) items.  Each item
// writes float-float partials (re, im) per reflection; a second kernel adds
// the splits in a fixed order (deterministic, no atomics) and forms
// M = |F|^2 P DW.  Sums: one 64-atom chunk in plain FP32, then folded into a
// float-float accumulator.
#include "fdx_internal.cuh"

namespace fdx {

static constexpr int SF_THREADS = 128;
static constexpr int SF_TILE = 256;   // atoms per shared-memory tile (multiple of SF_FOLD)
static constexpr int SF_FOLD = 64;    // atoms per FP32 partial sum (one element)
static constexpr int SF_GROUP = 4;    // reflections per group (consecutive l)
static constexpr int SF_GPT = 2;      // groups per thread
static constexpr int SF_GPB = SF_THREADS * SF_GPT;  // groups per work item
static constexpr int SF_SCAN = 1024;  // reflections per block of the grouping kernels
static constexpr int SF_FE_MAX = 40;  // element types per pass (form-factor table in shared memory)
static constexpr int SF_ELEM_MAX = 64;  // element types of a model (the API's limit)

// Pack one atom: fixed-point coordinates, element, and the exponent terms
// Bq = -B log2(e) / 4 (so that exp(-B s^2/4) = exp2(Bq s^2)) and log2(occ).
// An element index out of range packs as element 0 with a NaN amplitude: F
// becomes NaN and no table is indexed past its end.
__device__ __forceinline__ void sf_pack_one(const SFParams &p, int j, int e, bool bad, int pos) {
    unsigned q[3];
    for (int c = 0; c < 3; ++c) {
        const double x = p.frac[3 * j + c];
        const double f = x - floor(x);  // [0, 1)
        const unsigned long long u = (unsigned long long)llrint(f * 4294967296.0);
        q[c] = (unsigned)(u & 0xffffffffull);
    }
    p.atoms_q[pos] = make_uint4(q[0], q[1], q[2], (unsigned)e);
    const double occ = p.occ ? (double)p.occ[j] : 1.0;
    const float lo = bad ? __int_as_float(0x7fc00000) : (occ > 0.0 ? log2f((float)occ) : -INFINITY);
    p.atoms_w[pos] = make_float2((float)(-(double)p.B[j] * 1.4426950408889634 / 4.0), lo);
}

__device__ __forceinline__ int sf_key(const SFParams &p, int j, bool &bad) {
    const unsigned e = (unsigned)p.elem[j];
    bad = e >= (unsigned)p.n_elem;
    return bad ? 0 : (int)e;
}

// Packed atoms in input order (the structure-factor adjoint indexes them by atom).
__global__ void sf_pack_atoms_kernel(SFParams p) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.n_atoms) return;
    bool bad;
    const int e = sf_key(p, j, bad);
    sf_pack_one(p, j, e, bad, j);
}

// ex2.approx with flush-to-zero: one SFU op (amplitudes below 2^-126 are 0).
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// With a phase u (uint32 turns), rem = u sign-extended from its low 31 bits
// is u mod 1/2 turn in [-2^30, 2^30), and bit 31 of u - rem is the half turn,
// which flips the sign of both sin and cos.  r = rem 2^-32 in [-1/4, 1/4)
// turn has one rounding to 24 bits in the int -> float conversion (<= 2^-26
// turn).
__device__ __forceinline__ int half_rem(unsigned u) { return ((int)(u << 1)) >> 1; }
__device__ __forceinline__ unsigned half_sign(unsigned u, int rem) { return (u - (unsigned)rem) & 0x80000000u; }
__device__ __forceinline__ float flip(float x, unsigned sign) { return __uint_as_float(__float_as_uint(x) ^ sign); }

// (sin, cos)(2 pi u) for one phase (scalar), sign of the half turn included.
__device__ __forceinline__ void sincos_turn(unsigned u, float &sn, float &cs) {
    const int rem = half_rem(u);
    const unsigned sg = half_sign(u, rem);
    const float r = __int2float_rn(rem) * 2.3283064365386963e-10f;
    const float r2 = r * r;
    const float Sc[5] = FDX_SIN2PI_H_C;
    const float Cc[6] = FDX_COS2PI_H_C;
    sn = flip(r * horner(Sc, r2), sg);
    cs = flip(horner(Cc, r2), sg);
}

// The same for two phases at once on packed pairs; the signs are returned
// for the caller to apply.
__device__ __forceinline__ void sincos_turn2(unsigned u0, unsigned u1, float2 &sn, float2 &cs) {
    const int m0 = half_rem(u0), m1 = half_rem(u1);
    const float2 r = __fmul2_rn(make_float2(__int2float_rn(m0), __int2float_rn(m1)),
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
    S = __fmul2_rn(r, S);
    const unsigned g0 = half_sign(u0, m0), g1 = half_sign(u1, m1);
    sn = make_float2(flip(S.x, g0), flip(S.y, g1));
    cs = make_float2(flip(C.x, g0), flip(C.y, g1));
}

// ---------------------------------------------------------------------------
// Grouping: group starts at run starts (first reflection, or (h, k) differ
// from the previous reflection, or l is not the previous l + 1) and where
// l = 0 mod 4.  A group holds the following reflections up to the next start.
// Meridional reflections (h = k = 0) are groups of their own: there the
// group's base phase l0 z and the rotation j z are multiples of the same
// angle, so the rounding and polynomial errors of the two factors are
// correlated instead of random, and over many atoms they add up to a bias
// (e.g. 5e-6 of |F| for (0, 0, 2) = (0, 0, 1) rotated by z, 20,000 atoms).
// Direct evaluation keeps their errors random; there are only ~2 l_max of them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool group_start(const int32_t *hkl, int r) {
    const int l = hkl[3 * r + 2];
    if (r == 0 || (l & 3) == 0) return true;
    if (hkl[3 * r] == 0 && hkl[3 * r + 1] == 0) return true;
    return hkl[3 * r] != hkl[3 * r - 3] || hkl[3 * r + 1] != hkl[3 * r - 2] || l != hkl[3 * r - 1] + 1;
}

// The same three kernels sort the atoms by element.  Blocks nblk.. of the
// count and write kernels take 1024-atom chunks, the scan kernel turns the
// per-chunk element counts into first entries (element-major, chunks in
// order: a stable sort) with each element's run padded to whole SF_FOLD
// chunks by zero-amplitude entries.  So every SF_FOLD-atom chunk of the list
// holds one element and its form factor multiplies the chunk's sum once.

// Chunk c of the atoms: element counts into acnt[c][*].
__device__ void sf_atom_count(const SFParams &p, int c) {
    __shared__ int s_h[SF_ELEM_MAX];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < SF_ELEM_MAX) s_h[tid] = 0;
    __syncthreads();
    const int j = c * SF_SCAN + tid;
    bool bad = false;
    const int e = j < p.n_atoms ? sf_key(p, j, bad) : SF_ELEM_MAX;
    const unsigned same = __match_any_sync(FDX_FULL_MASK, e);
    if (e < SF_ELEM_MAX && lane == __ffs(same) - 1) atomicAdd(&s_h[e], __popc(same));
    __syncthreads();
    if (tid < SF_ELEM_MAX) p.acnt[c * SF_ELEM_MAX + tid] = s_h[tid];
}

// Per block of SF_SCAN reflections: number of group starts.
__global__ void __launch_bounds__(SF_SCAN) sf_group_count_kernel(SFParams p, int nblk) {
    if ((int)blockIdx.x >= nblk) {
        sf_atom_count(p, blockIdx.x - nblk);
        return;
    }
    const int r = blockIdx.x * SF_SCAN + threadIdx.x;
    const int f = r < p.n_refl ? (int)group_start(p.hkl, r) : 0;
    const int cnt = __syncthreads_count(f);
    if (threadIdx.x == 0) p.gblk[blockIdx.x] = cnt;
}

// In-place exclusive scan of n values (value(i) read, put(i, excl) written)
// by one block of SF_SCAN threads; returns the total.
template <class Get, class Put>
__device__ int block_scan(int n, Get value, Put put) {
    __shared__ int s_warp[SF_SCAN / 32];
    __shared__ int s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < n; b0 += SF_SCAN) {
        const int b = b0 + threadIdx.x;
        const int v = b < n ? value(b) : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FDX_FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FDX_FULL_MASK, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int excl = s_carry + (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
        if (b < n) put(b, excl);
        __syncthreads();
        if (threadIdx.x == SF_SCAN - 1) s_carry = excl + v;
        __syncthreads();
    }
    return s_carry;
}

// Exclusive scan of the block counts (the total is the group count), then
// the atoms' first entries.
__global__ void __launch_bounds__(SF_SCAN) sf_group_scan_kernel(SFParams p, int nblk) {
    __shared__ int s_tot[SF_ELEM_MAX];
    const int G = block_scan(nblk, [&](int b) { return p.gblk[b]; }, [&](int b, int x) { p.gblk[b] = x; });
    if (threadIdx.x == 0) *p.n_groups = G;
    const int ne = p.n_elem, nch = p.n_achunks;
    if (threadIdx.x < SF_ELEM_MAX) s_tot[threadIdx.x] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < ne * nch; k += SF_SCAN) atomicAdd(&s_tot[k / nch], p.acnt[(k % nch) * SF_ELEM_MAX + k / nch]);
    __syncthreads();
    // entries (e, c), element-major; entry (e, nch) is the padding of element e
    const int total = block_scan(
        ne * (nch + 1),
        [&](int i) {
            const int e = i / (nch + 1), c = i % (nch + 1);
            return c < nch ? p.acnt[c * SF_ELEM_MAX + e] : (SF_FOLD - s_tot[e] % SF_FOLD) % SF_FOLD;
        },
        [&](int i, int x) {
            const int e = i / (nch + 1), c = i % (nch + 1);
            if (c < nch) p.acnt[c * SF_ELEM_MAX + e] = x;
            if (c == 0) p.elem_off[e] = x;
        });
    if (threadIdx.x < ne) p.elem_cnt[threadIdx.x] = s_tot[threadIdx.x];
    if (threadIdx.x == 0) p.elem_off[ne] = total;
}

// Chunk c of the atoms: pack each at its entry (first entry of its element
// in this chunk + its rank among the chunk's atoms of that element); chunk 0
// also writes the padding.
__device__ void sf_atom_write(const SFParams &p, int c) {
    __shared__ int s_wc[SF_SCAN / 32][SF_ELEM_MAX];  // per warp and element: atoms of this chunk
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = lane; k < SF_ELEM_MAX; k += 32) s_wc[warp][k] = 0;
    __syncwarp();
    const int j = c * SF_SCAN + tid;
    const bool valid = j < p.n_atoms;
    bool bad = false;
    const int e = valid ? sf_key(p, j, bad) : SF_ELEM_MAX;  // invalid lanes match only each other
    const unsigned same = __match_any_sync(FDX_FULL_MASK, e);
    if (valid && lane == __ffs(same) - 1) s_wc[warp][e] = __popc(same);
    __syncthreads();
    if (valid) {
        int pos = p.acnt[c * SF_ELEM_MAX + e] + __popc(same & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) pos += s_wc[w][e];
        sf_pack_one(p, j, e, bad, pos);
    }
    if (c == 0)
        for (int k = tid; k < p.n_elem * SF_FOLD; k += SF_SCAN) {
            const int ee = k / SF_FOLD, pos = p.elem_off[ee] + p.elem_cnt[ee] + k % SF_FOLD;
            if (pos < p.elem_off[ee + 1]) {
                p.atoms_q[pos] = make_uint4(0u, 0u, 0u, (unsigned)ee);
                p.atoms_w[pos] = make_float2(0.0f, -INFINITY);
            }
        }
}

// Scatter: groups[g] = first reflection of group g, in list order.
__global__ void __launch_bounds__(SF_SCAN) sf_group_write_kernel(SFParams p, int nblk) {
    if ((int)blockIdx.x >= nblk) {
        sf_atom_write(p, blockIdx.x - nblk);
        return;
    }
    __shared__ int s_warp[SF_SCAN / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * SF_SCAN + threadIdx.x;
    const bool f = r < p.n_refl && group_start(p.hkl, r);
    const unsigned bal = __ballot_sync(FDX_FULL_MASK, f);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        const int v = s_warp[lane];
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FDX_FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        s_warp[lane] = x - v;
    }
    __syncthreads();
    if (f) p.groups[p.gblk[blockIdx.x] + s_warp[warp] + __popc(bal & ((1u << lane) - 1u))] = r;
}

// Group g: first reflection r0 and count c (1..4; a group never crosses a
// multiple of 4 in l, so the next start is at most 4 entries later).
__device__ __forceinline__ void group_span(const SFParams &p, int G, int g, int &r0, int &c) {
    if (g >= G) {
        r0 = 0, c = 0;
        return;
    }
    r0 = p.groups[g];
    c = (g + 1 < G ? p.groups[g + 1] : p.n_refl) - r0;
}

// exp(y) in FP64 for |y| <= 700: y = n ln 2 + r with |r| <= ln(2)/2, exp(r)
// by its Taylor series through r^10/10! (truncation below 3e-13 relative),
// 2^n put in the exponent field.  Outside that range the library's exp.
__device__ __forceinline__ double exp_rr(double y) {
    if (!(fabs(y) <= 700.0)) return exp(y);
    const double n = rint(y * 1.4426950408889634);
    double r = fma(-n, 6.93147180559945286e-01, y);
    r = fma(-n, 2.319046813846299558e-17, r);
    double e = 1.0 / 3628800.0;
    const double inv_fact[10] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320,
                                 1.0 / 362880};
#pragma unroll
    for (int k = 9; k >= 0; --k) e = fma(e, r, inv_fact[k]);
    return e * __hiloint2double(((int)n + 1023) << 20, 0);
}

// P DW of reflection r: the paracrystal factor prod_i 1/cosh(2 x_i),
// x_i = pi^2 g_i^2 h_i^2 (Hosemann intensity model), times the axial
// Debye-Waller factor exp(-sum_i B_i h_i^2 / (4 |a_i|^2)), as one exponential
// (1/cosh z = 2 e^-z / (1 + e^-2z)):
//   P DW = exp(Y),  Y = sum_i [-B_i h_i^2 / (4 |a_i|^2) - 2 x_i + ln 2 - log1p(exp(-4 x_i))].
// Y is summed in FP64; the bounded terms log1p(exp(-4 x_i)) in [0, ln 2] are
// evaluated in FP32 (an absolute error ~1e-7 in Y is a relative error ~1e-7 in
// P DW); exp(Y) in FP64.  FP64 is slow on this GPU: one exponential per
// reflection instead of four, and no division.
__device__ __forceinline__ double refl_pdw(const SFParams &p, int r) {
    if (!p.has_br) return 1.0;
    const bool hos = p.intensity_model == FDX_INTENSITY_HOSEMANN;
    double y = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double hi = (double)p.hkl[3 * r + i], h2 = hi * hi;
        y = fma(p.dwc[i], h2, y);
        if (hos && p.hx[i] > 0.0) {
            const double x = p.hx[i] * h2;
            y = fma(-2.0, x, y) + (0.6931471805599453 - (double)log1pf(expf((float)(-4.0 * x))));
        }
    }
    return exp_rr(y);
}

// One CTA per (block of SF_GPB groups, atom split) item, looping over items.
// Thread t owns groups t and t + SF_THREADS of the block; every quantity of
// slot j (reflection l0 + j) is a packed pair over the two groups.  This pass
// covers element types e_lo .. e_lo + n_fe - 1: the entries elem_off[e_lo] ..
// elem_off[e_lo + n_fe] of the element-sorted atom list, cut into n_split
// ranges of whole SF_FOLD chunks.  A chunk holds one element, so its terms
// are summed without the form factor, which multiplies the chunk's sum.
__global__ void __launch_bounds__(SF_THREADS) sf_main_kernel(SFParams p) {
    __shared__ uint4 s_q[SF_TILE];
    __shared__ float4 s_w[SF_TILE];          // (Bq, Bq, log2 occ, log2 occ); log2 occ = -inf: not in this pass
    __shared__ float4 s_rot[3][SF_TILE];     // j = 1..3: (cos, cos, sin, sin)(2 pi j z)
    extern __shared__ float4 s_fe[];         // [n_fe][2][SF_THREADS]: f_e(s) pairs (slot 0, 1) and (slot 2, 3)
    const int tid = threadIdx.x;
    const int G = *p.n_groups;
    const int a_lo = p.elem_off[p.e_lo], a_hi = p.elem_off[p.e_lo + p.n_fe];
    const int per = ((a_hi - a_lo + p.n_split - 1) / p.n_split + SF_FOLD - 1) / SF_FOLD * SF_FOLD;
    const int n_gblk = (G + SF_GPB - 1) / SF_GPB;
    const long long n_items = (long long)n_gblk * p.n_split;
    for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int gb = (int)(item % n_gblk), split = (int)(item / n_gblk);
        int r0[SF_GPT], cnt[SF_GPT];
        unsigned h[SF_GPT], k[SF_GPT], l[SF_GPT];
        float s2[SF_GPT][SF_GROUP];
#pragma unroll
        for (int t = 0; t < SF_GPT; ++t) {
            group_span(p, G, gb * SF_GPB + t * SF_THREADS + tid, r0[t], cnt[t]);
            int hh = 0, kk = 0, ll = 0;
            if (cnt[t] > 0) hh = p.hkl[3 * r0[t]], kk = p.hkl[3 * r0[t] + 1], ll = p.hkl[3 * r0[t] + 2];
            h[t] = (unsigned)hh, k[t] = (unsigned)kk, l[t] = (unsigned)ll;
#pragma unroll
            for (int j = 0; j < SF_GROUP; ++j) {
                const double lj = (double)(ll + j);
                double D[3];
                for (int q = 0; q < 3; ++q) D[q] = hh * p.As[q] + kk * p.As[3 + q] + lj * p.As[6 + q];
                s2[t][j] = (float)(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
            }
        }
        // form factors of this thread's 8 reflections (0 for empty slots)
        for (int e = 0; e < p.n_fe; ++e) {
            const float *f = p.ff + 9 * (p.e_lo + e);
            float fe[SF_GPT][SF_GROUP];
#pragma unroll
            for (int t = 0; t < SF_GPT; ++t)
#pragma unroll
                for (int j = 0; j < SF_GROUP; ++j) {
                    float v = f[8];
                    for (int i = 0; i < 4; ++i) v = fmaf(f[i], expf(-0.25f * f[4 + i] * s2[t][j]), v);
                    fe[t][j] = j < cnt[t] ? v : 0.0f;
                }
            s_fe[(2 * e) * SF_THREADS + tid] = make_float4(fe[0][0], fe[1][0], fe[0][1], fe[1][1]);
            s_fe[(2 * e + 1) * SF_THREADS + tid] = make_float4(fe[0][2], fe[1][2], fe[0][3], fe[1][3]);
        }
        float2 s2p[SF_GROUP];
#pragma unroll
        for (int j = 0; j < SF_GROUP; ++j) s2p[j] = make_float2(s2[0][j], s2[1][j]);

        ff reF[SF_GPT][SF_GROUP], imF[SF_GPT][SF_GROUP];
#pragma unroll
        for (int t = 0; t < SF_GPT; ++t)
#pragma unroll
            for (int j = 0; j < SF_GROUP; ++j) reF[t][j] = imF[t][j] = ff{0.0f, 0.0f};
        const int a_begin = min(a_hi, a_lo + split * per);
        const int a_end = min(a_hi, a_begin + per);
        for (int t0 = a_begin; t0 < a_end; t0 += SF_TILE) {
            const int na = min(SF_TILE, a_end - t0);  // a multiple of SF_FOLD
            __syncthreads();
            for (int i = tid; i < na; i += SF_THREADS) {
                const uint4 q = p.atoms_q[t0 + i];
                const float2 w = p.atoms_w[t0 + i];
                s_q[i] = q;
                s_w[i] = make_float4(w.x, w.x, w.y, w.y);
#pragma unroll
                for (int j = 1; j <= 3; ++j) {
                    float sn, cs;
                    sincos_turn((unsigned)j * q.z, sn, cs);
                    s_rot[j - 1][i] = make_float4(cs, cs, sn, sn);
                }
            }
            __syncthreads();
            for (int i0 = 0; i0 < na; i0 += SF_FOLD) {
                float2 ra[SF_GROUP], ia[SF_GROUP];
#pragma unroll
                for (int j = 0; j < SF_GROUP; ++j) ra[j] = ia[j] = make_float2(0.0f, 0.0f);
#pragma unroll 2
                for (int i = i0; i < i0 + SF_FOLD; ++i) {
                    const uint4 q = s_q[i];
                    const float4 w = s_w[i];
                    const float2 wb = make_float2(w.x, w.y), wl = make_float2(w.z, w.w);
                    float2 sn, cs;
                    sincos_turn2(h[0] * q.x + k[0] * q.y + l[0] * q.z, h[1] * q.x + k[1] * q.y + l[1] * q.z, sn, cs);
                    const float2 nsn = make_float2(-sn.x, -sn.y);
                    float2 cr[SF_GROUP], ci[SF_GROUP];
                    cr[0] = cs, ci[0] = sn;
#pragma unroll
                    for (int j = 1; j < SF_GROUP; ++j) {
                        const float4 R = s_rot[j - 1][i];
                        const float2 C = make_float2(R.x, R.y), S = make_float2(R.z, R.w);
                        cr[j] = __ffma2_rn(cs, C, __fmul2_rn(nsn, S));
                        ci[j] = __ffma2_rn(cs, S, __fmul2_rn(sn, C));
                    }
#pragma unroll
                    for (int j = 0; j < SF_GROUP; ++j) {
                        const float2 x = __ffma2_rn(wb, s2p[j], wl);
                        const float2 a = make_float2(ex2_ftz(x.x), ex2_ftz(x.y));
                        ra[j] = __ffma2_rn(a, cr[j], ra[j]);
                        ia[j] = __ffma2_rn(a, ci[j], ia[j]);
                    }
                }
                // the chunk's element: its form factors at this thread's 8 reflections
                const int e = (int)s_q[i0].w - p.e_lo;
                const float4 fa = s_fe[(2 * e) * SF_THREADS + tid];
                const float4 fb = s_fe[(2 * e + 1) * SF_THREADS + tid];
                const float2 fe[SF_GROUP] = {make_float2(fa.x, fa.y), make_float2(fa.z, fa.w), make_float2(fb.x, fb.y),
                                             make_float2(fb.z, fb.w)};
#pragma unroll
                for (int j = 0; j < SF_GROUP; ++j) {
                    const float2 rf = __fmul2_rn(fe[j], ra[j]), im = __fmul2_rn(fe[j], ia[j]);
                    reF[0][j] = ff_add_f(reF[0][j], rf.x), reF[1][j] = ff_add_f(reF[1][j], rf.y);
                    imF[0][j] = ff_add_f(imF[0][j], im.x), imF[1][j] = ff_add_f(imF[1][j], im.y);
                }
            }
        }
        const size_t row = (size_t)(p.split_base + split) * p.n_refl;
#pragma unroll
        for (int t = 0; t < SF_GPT; ++t)
#pragma unroll
            for (int j = 0; j < SF_GROUP; ++j)
                if (j < cnt[t] && FDX_IN_BOUNDS(row + r0[t] + j, (long long)p.n_rows * p.n_refl, DBG_SF_PART))
                    p.partial[row + r0[t] + j] = make_float4(reF[t][j].hi, reF[t][j].lo, imF[t][j].hi, imF[t][j].lo);
    }
}

// Sum the partial rows in order (float-float); F = (re, im); M = |F|^2 P DW.
__global__ void sf_reduce_kernel(SFParams p) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.n_refl) return;
    ff re = {0.0f, 0.0f}, im = {0.0f, 0.0f};
    for (int s = 0; s < p.n_rows; ++s) {
        const float4 v = p.partial[(size_t)s * p.n_refl + r];
        re = ff_add(re, ff{v.x, v.y});
        im = ff_add(im, ff{v.z, v.w});
    }
    const double dre = (double)re.hi + (double)re.lo, dim = (double)im.hi + (double)im.lo;
    p.F_out[2 * r] = (float)dre;
    p.F_out[2 * r + 1] = (float)dim;
    if (p.M_out) p.M_out[r] = (float)((dre * dre + dim * dim) * refl_pdw(p, r));
}

static size_t sf_align(size_t x) { return (x + 255) / 256 * 256; }

int sf_passes(int n_elem) { return (n_elem + SF_FE_MAX - 1) / SF_FE_MAX; }

static int sm_count() {
    static int s_sm = 0;
    if (s_sm == 0) {
        int dev = 0, v = 148;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            s_sm = v;
        else
            s_sm = 148;
    }
    return s_sm;
}

// Resident CTAs of sf_main_kernel on the whole GPU for a form-factor table of
// n_fe element types (dynamic shared memory).
static int sf_slots(int n_fe) {
    static size_t s_shm = (size_t)-1;
    static int s_per_sm = 1;
    const size_t shm = sizeof(float4) * 2 * SF_THREADS * (size_t)(n_fe > 0 ? n_fe : 1);
    if (shm != s_shm) {
        int v = 0;
        if (shm > 48 * 1024 &&
            cudaFuncSetAttribute(sf_main_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess)
            cudaGetLastError();
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sf_main_kernel, SF_THREADS, shm) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        s_shm = shm, s_per_sm = v;
    }
    return sm_count() * s_per_sm;
}

// Split of the atom list: enough (group block, split) items for about four
// waves of resident CTAs (so that the last, partial wave costs little), with
// at least one tile of atoms per split and at most max_split rows of partials
// over all element passes.  The group count is estimated as 0.3 n_refl + 16
// (lexicographic lists give 0.26-0.35 groups per reflection); any other count
// only changes the balance, never the result.
void sf_plan(int n_atoms, int n_refl, int n_elem, int max_split, int &n_split, int &per) {
    const int passes = sf_passes(n_elem);
    const long long slots = sf_slots(n_elem < SF_FE_MAX ? n_elem : SF_FE_MAX);
    const long long gblk = ((long long)(0.3 * n_refl) + 16 + SF_GPB - 1) / SF_GPB;
    const int tiles = (n_atoms + SF_TILE - 1) / SF_TILE;
    long long want = (4 * slots + gblk - 1) / gblk;
    const int cap = max_split / passes;
    if (want > cap) want = cap;
    if (want > tiles) want = tiles;
    if (want < 1) want = 1;
    const int pt = (tiles + (int)want - 1) / (int)want;  // tiles per split
    per = pt * SF_TILE;
    n_split = (tiles + pt - 1) / pt;
}

// Workspace of the structure factors: packed atoms (element-sorted, with room
// for the padding of up to SF_ELEM_MAX element runs), the element offsets and
// counts, the per-chunk element counts, the group list and block offsets,
// the group count, and max_split rows of partials.  With ws null only the
// size is computed.
size_t sf_bind(SFParams *p, char *ws, int n_atoms, int n_refl, int max_split) {
    const int nr = n_refl > 0 ? n_refl : 1;
    const int nblk = (nr + SF_SCAN - 1) / SF_SCAN;
    size_t off = 0;
    const size_t na = (size_t)n_atoms + (size_t)SF_FOLD * SF_ELEM_MAX;  // room for the element runs' padding
    const size_t q = off;
    off += sf_align(sizeof(uint4) * na);
    const size_t w = off;
    off += sf_align(sizeof(float2) * na);
    const size_t eo = off;
    off += sf_align(sizeof(int) * (2 * SF_ELEM_MAX + 1));
    const size_t ac = off;
    off += sf_align(sizeof(int) * SF_ELEM_MAX * (size_t)((n_atoms + SF_SCAN - 1) / SF_SCAN));
    const size_t g = off;
    off += sf_align(sizeof(int) * (size_t)nr);
    const size_t b = off;
    off += sf_align(sizeof(int) * (size_t)(nblk + 1));
    const size_t part = off;
    off += sf_align(sizeof(float4) * (size_t)max_split * (size_t)nr);
    if (p && ws) {
        p->atoms_q = reinterpret_cast<uint4 *>(ws + q);
        p->atoms_w = reinterpret_cast<float2 *>(ws + w);
        p->elem_off = reinterpret_cast<int *>(ws + eo);
        p->elem_cnt = p->elem_off + SF_ELEM_MAX + 1;
        p->acnt = reinterpret_cast<int *>(ws + ac);
        p->groups = reinterpret_cast<int *>(ws + g);
        p->gblk = reinterpret_cast<int *>(ws + b);
        p->n_groups = p->gblk + nblk;
        p->partial = reinterpret_cast<float4 *>(ws + part);
    }
    return off;
}

cudaError_t launch_sf_pack(SFParams &p, cudaStream_t s) {
    sf_pack_atoms_kernel<<<(p.n_atoms + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_structure_factors(SFParams &p, cudaStream_t s) {
    if (p.n_refl <= 0) return cudaSuccess;
    if (p.n_elem < 1 || p.n_elem > SF_ELEM_MAX) return cudaErrorInvalidValue;
    const int nblk = (p.n_refl + SF_SCAN - 1) / SF_SCAN;
    p.n_achunks = (p.n_atoms + SF_SCAN - 1) / SF_SCAN;
    for (int i = 0; i < 3; ++i) {
        p.hx[i] = FDX_PI * FDX_PI * p.g[i] * p.g[i];
        p.dwc[i] = p.has_br ? -0.25 * p.Bax[i] / (p.alen[i] * p.alen[i]) : 0.0;
    }
    sf_group_count_kernel<<<nblk + p.n_achunks, SF_SCAN, 0, s>>>(p, nblk);
    sf_group_scan_kernel<<<1, SF_SCAN, 0, s>>>(p, nblk);
    sf_group_write_kernel<<<nblk + p.n_achunks, SF_SCAN, 0, s>>>(p, nblk);
    const int passes = sf_passes(p.n_elem);
    // items: at most (n_refl groups) / SF_GPB blocks x n_split; CTAs loop over items
    const long long items_ub = (long long)((p.n_refl + SF_GPB - 1) / SF_GPB) * p.n_split;
    p.n_rows = passes * p.n_split;
    for (int pass = 0; pass < passes; ++pass) {
        p.e_lo = pass * SF_FE_MAX;
        p.n_fe = min(SF_FE_MAX, p.n_elem - p.e_lo);
        p.split_base = pass * p.n_split;
        const long long slots = sf_slots(p.n_fe);
        const unsigned grid = (unsigned)(items_ub < slots ? items_ub : slots);
        const size_t shm = sizeof(float4) * 2 * SF_THREADS * (size_t)p.n_fe;
        sf_main_kernel<<<grid, SF_THREADS, shm, s>>>(p);
    }
    sf_reduce_kernel<<<(p.n_refl + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fdx
