// Internal declarations shared by the libfdx CUDA sources (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fdx.h"
#include "poly_coeffs.cuh"

#define FDX_FULL_MASK 0xffffffffu
#define FDX_PI 3.14159265358979323846

// ---------------------------------------------------------------------------
// Bounds checks of a debugging build (compiled with FDX_DEBUG and relocatable
// device code): an index outside its buffer sets the check's bit in a device
// status word, records the index and skips the access (no trap, no assert:
// the context stays usable); fdx_debug_status reads and clears the word.  In
// a normal build FDX_IN_BOUNDS is the constant true and changes no code.
// ---------------------------------------------------------------------------
#ifdef FDX_DEBUG
extern __device__ unsigned long long fdx_debug_word[2];  // [0]: bits of failed checks, [1]: last bad index
__device__ __forceinline__ bool fdx_in_bounds(long long i, long long n, int check) {
    if (i >= 0 && i < n) return true;
    atomicOr(&fdx_debug_word[0], 1ull << check);
    atomicExch(&fdx_debug_word[1], (unsigned long long)i);
    return false;
}
#define FDX_IN_BOUNDS(i, n, check) fdx_in_bounds((long long)(i), (long long)(n), (check))
#else
#define FDX_IN_BOUNDS(i, n, check) true
#endif

namespace fdx {

// The checks of a debugging build, one bit each in the status word.
enum DebugCheck {
    DBG_NODES = 0,    // node-table entry of a staged block
    DBG_STAGE = 1,    // slot of the warp's node buffer written by staging
    DBG_PACK = 2,     // node pair written by packing
    DBG_WALK = 3,     // node pair read by the walk
    DBG_LIST = 4,     // slot of a tile's reflection list
    DBG_RECORD = 5,   // reflection index of a list entry
    DBG_IMAGE = 6,    // pixel written by a pattern-family kernel
    DBG_PIXGEO = 7,   // pixel-geometry entry read
    DBG_PATCH = 8,    // adjoint patch bounds
    DBG_GRAD_IN = 9,  // dL/dI entry read by the adjoint
    DBG_ITEM = 10,    // adjoint item output
    DBG_SF_PART = 11, // structure-factor partial-sum row
    DBG_SPLAT = 12,   // scatter-form image entry
    DBG_BATCH = 13    // position-table entry of a batched launch
};

// ---------------------------------------------------------------------------
// Float-float ("double-float") arithmetic: a value is hi + lo with |lo| <=
// ulp(hi)/2.  Error-free transformations after Knuth (TwoSum), Dekker
// (FastTwoSum) and the FMA form of TwoProduct (Ogita, Rump, Oishi 2005).
// B300 runs FP64 at a small fraction of its FP32 rate, so the places that need
// more than 24 bits use these pairs instead.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    float e = s.lo + (a.lo + b.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.hi, -b.lo}); }

__host__ __device__ __forceinline__ void split_double(double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// Reciprocal on the SFU (rcp.approx.ftz.f32: max error 1 ulp for normal inputs).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Horner evaluation with coefficients in increasing order.
template <int N>
__device__ __forceinline__ float horner(const float (&c)[N], float x) {
    float acc = c[N - 1];
#pragma unroll
    for (int k = N - 2; k >= 0; --k) acc = fmaf(acc, x, c[k]);
    return acc;
}

// sin^2(pi t) for |t| <= 1/2: t^2 Q(t^2), Q fitted by fit_poly.py.
__device__ __forceinline__ float sinpi_sq(float t) {
    const float Q[6] = FDX_SINPI2_C;
    float x = t * t;
    return x * horner(Q, x);
}

// ---------------------------------------------------------------------------
// Per-reflection record of the pattern kernel (64 floats, 256 B), written by
// the reflection set-up kernel in FP64 and rounded once.
// Local frame: (S^, e1, e2) with e1 = normalize(n x S^) (or b x S^ on the
// axis), e2 = S^ x e1; e_R is the unit radial direction of D (e1 on the
// axis).  All "/r0" quantities are in units of r0 = |D|.
// ---------------------------------------------------------------------------
enum RecField {
    REC_RD = 0,    // R_D hi, lo
    REC_ZD = 2,    // Z_D hi, lo
    REC_NFR = 4,   // n . (S^, e1, e2) / r0, hi[3] then lo[3]
    REC_EFR = 10,  // e_R . (S^, e1, e2) / r0, hi[3] then lo[3]
    REC_AR = 16,   // a_i . e_R  (i = a, b, c)
    REC_H = 19,    // h_i as float (exact)
    REC_E1 = 22,   // r0 a_i . e1
    REC_E2 = 25,   // r0 a_i . e2
    REC_CR = 28,   // 4 box corners sum_i (+-) tmax_i a*_i in the local frame, / r0 (4 x 3)
    REC_LA = 40,   // Hosemann: beta_i^2;  sinc: N_i
    REC_LB = 43,   // Hosemann: 1 - beta_i^2
    REC_TM = 46,   // support half-widths tmax_i
    REC_FR = 49,   // pair factor: Hosemann M r0^2 prod beta_i; sinc M r0^2 prod N_i / pi^6
    REC_R2B = 50,  // r0^2 prod beta_i (Hosemann; dI/dM = L r0^2 prod beta_i S)
    REC_BETA = 51, // beta_i
    REC_M = 54,    // M
    REC_DBF = 55,  // 2 beta_i / (1 - beta_i^2), 0 when beta_i is clamped at 1 (adjoint)
    REC_AR0 = 58,  // |a_i| r0: Lipschitz constant of sigma_i along the gnomonic plane
    REC_SLB = 61,  // sqrt(1 - beta_i^2) (Hosemann)
    REC_SIZE = 64
};

struct PatternParams {
    int nx, ny, n_refl, n_nodes;
    int ppl;              // pixels per lane of the forward kernel (1 or 2)
    float T, inv_h;       // grid half-extent, 1 / node spacing
    int blk_lr, blk_lc;   // node blocks of the culling: 2^blk_lr rows x 2^blk_lc columns (blk_lr + blk_lc = 5)
    float AZ[3];          // a_i . n (cell constants)
    double delta_L;
    const float4 *pixgeo; // [ny*nx] (R hi, R lo, Z hi, Z lo)
    const float4 *reach;  // [n_refl] (r0, rho_B, psi_D, dpsi)
    const float *recs;    // [n_refl][REC_SIZE]
    const float4 *nodes;  // [n*n][2]: (cm1 hi, cm1 lo, cd1 hi, cd1 lo), (cd2 hi, cd2 lo, w, 0)
    const float2 *dnodes; // [n*n]: (dw/dsigma, dw/dgamma)
    float *image;         // [ny][nx]
    int32_t *counts;      // [ny][nx] (count mode)
};

// Forward over the models of one tile shape (pattern_batch_kernel<LS, PPL>):
// per-model parameters in device memory by model index; the models are
// ordered by tile shape in the position tables, and those of this launch take
// positions [pos0, pos0 + n_pos) and items [item0, item_end) (CTA tiles).
struct BatchFwdParams {
    const PatternParams *models;  // [n_models] device, by model index
    const long long *item_prefix; // [n_models] by position: the model's first item
    const int *item_model;        // [n_models] by position: the model index
    int pos0, n_pos;
    long long item0, item_end;
    unsigned *counter;            // zeroed before the launch
};

// First item of position j's model is item_prefix[j]; the position of `item`
// among [pos0, pos0 + n_pos): the last j with item_prefix[j] <= item (models
// without items share their successor's prefix and are passed over).
__device__ __forceinline__ int item_position(const long long *prefix, int pos0, int n_pos, long long item) {
    int lo = pos0, hi = pos0 + n_pos - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct ReflSetupParams {
    double A[9], As[9];   // real basis rows a, b, c and reciprocal rows a*, b*, c*
    double nh[3], bh[3];  // unit fiber and beam axes
    double alen[3];       // |a_i|
    double L[3], g[3], Bax[3];
    double T, K_z;
    int lineshape, intensity_model, n_refl, pad;
    const int32_t *hkl;
    const float *M;       // may be null (then M = 1)
    float *recs;
    float4 *reach;
    double *frames;       // may be null: [n_refl][12] (S^, e1, e2, r0, rho_B, 0) for the scatter form
    float *ring;          // may be null: [n_refl][RING_REC] ring-average record
    double alen3[3];      // |a_i| (ring-average step rule)
    int ring_max_n;       // cap on the ring-average azimuth points per reflection
};

// Ring-average record per reflection (fdx_ring.cu): e_P = n x e_R.
enum RingField {
    RING_TFR = 0,   // e_P . (S^, e1, e2) / r0, hi[3] then lo[3]
    RING_AT = 6,    // a_i . e_P
    RING_PHI = 9,   // window half-width Phi_r, hi, lo
    RING_N = 11,    // azimuth points N_r (exact integer as float)
    RING_HW = 12,   // quadrature weight (2 Phi_r / N_r) / (2 pi)
    RING_RT = 13,   // rho_tot = rho_B + sqrt(2) r0 T
    RING_REC = 16
};
// Pixels per lane of the ring average: a warp's patch is 8 x 4 RING_PPL pixels.
static constexpr int RING_PPL = 2;

struct NodeParams {
    int n;
    double T, h, sigma, gamma, sigma_r;
    float4 *nodes;
    float2 *dnodes;  // may be null
    double *nodes64; // may be null: [n*n][4] = w, c, dw/dsigma, dw/dgamma in FP64
};

struct PixelParams {
    int nx, ny;
    double lambda, dist, pix;
    double bh[3], uh[3], vh[3], nh[3];
    float4 *pixgeo;
};

// Weideman (1994) rational approximation of the Faddeeva function,
// w(z) ~ 2 p(Z) / (L - i z)^2 + 1 / (sqrt(pi) (L - i z)), Z = (L + i z)/(L - i z),
// for Im z >= 0; coefficients computed once on the host (fdx_setup.cu).
#define FDX_WEIDEMAN_N 40
struct WeidemanCoeffs {
    double a[FDX_WEIDEMAN_N];  // a_1 .. a_N
    double L;
};

// Host helpers (fdx_setup.cu)
void cell_basis(const fdx_cell &c, double A[9], double As[9]);
const WeidemanCoeffs &weideman_coeffs();

// Launchers
cudaError_t launch_pixel_geometry(const PixelParams &p, cudaStream_t s);
cudaError_t launch_nodes(const NodeParams &p, const WeidemanCoeffs &wc, cudaStream_t s);
cudaError_t launch_refl_setup(const ReflSetupParams &p, cudaStream_t s);
cudaError_t launch_pattern(const PatternParams &p, int lineshape, bool count_mode, cudaStream_t s);
cudaError_t launch_pattern_batch(const BatchFwdParams &B, int ppl, int n_ctas, cudaStream_t s);

struct SFParams {
    int n_atoms, n_elem, n_refl, n_split;
    double As[9];
    const double *frac;
    const float *B, *occ, *ff;
    const uint8_t *elem;
    uint4 *atoms_q;        // packed: X, Y, Z (fixed point), elem
    float2 *atoms_w;       // packed: Bq = -B log2(e)/4, log2(occ)
    int *elem_off;         // [n_elem + 1] element-sorted copy: first entry of each element, total
    int *elem_cnt;         // [64] atoms of each element
    int *acnt;             // [n_achunks][64] atoms of each element per 1024-atom chunk, then their first entries
    int n_achunks;         // ceil(n_atoms / 1024)
    const int32_t *hkl;
    int *groups;           // [<= n_refl] first reflection of each group (consecutive l, equal h, k)
    int *gblk;             // [n_refl / 1024 + 1] per-block group offsets
    int *n_groups;         // group count (device)
    float4 *partial;       // [rows][n_refl] (re hi, re lo, im hi, im lo)
    float *F_out, *M_out;
    int has_br, intensity_model;
    int e_lo, n_fe, split_base, n_rows;  // element pass and partial rows (set by the launcher)
    double g[3], Bax[3], alen[3];
    double hx[3], dwc[3];  // pi^2 g_i^2 and -B_i / (4 |a_i|^2) (set by the launcher)
};

cudaError_t launch_structure_factors(SFParams &p, cudaStream_t s);

// Scatter form (fdx_scatter.cu).
struct ScatterParams {
    PatternParams P;          // records, nodes (pixgeo/image unused)
    int n_s;                  // samples per reflection
    int spot;                 // detector spot size (odd): each hit covers spot x spot pixels
    const float4 *samples;    // [n_s] (x_r, x_1, x_2, q)
    float4 *stab;             // [n_s][3] per-sample table (set-up kernel)
    const double *frames;     // [n_refl][12]
    float2 *proj;             // [n_refl][SCAT_PROJ] float-float: frame vectors projected on wdir, r0, rho_B, (rho_B / r0, 0)
    double T, lambda, dist, pix, delta_L;
    double nh[3], bh[3], uh[3], vh[3];
    double wdir[7][3];        // n, u, v, b, u x n, v x n, b x n
    double il, kn, kw[3], nw[3], dp, hx, hy;  // 1/lambda, (b.n)/lambda, (b.w)/lambda and n.w for w = u, v, b,
                                              // distance / pixel, n_x / 2, n_y / 2
    float2 il_f, kn_f, kw_f[3], nw_f[3], dp_f, hx_f, hy_f;  // the same as float-float (hi, lo)
    double *img64;            // [ny][nx] accumulation
    float *image;             // [ny][nx] output
    unsigned long long *count;  // evaluation count (count mode)
};
static constexpr int SCAT_PROJ = 24;
cudaError_t launch_scatter(const ScatterParams &p, int lineshape, bool count_mode, cudaStream_t s);

// Ring-integrated cylindrical average (fdx_ring.cu).
struct RingParams {
    PatternParams P;          // pixel geometry, records, nodes; P.image / P.counts are the outputs
    const float *ring;        // [n_refl][RING_REC]
    int n_split;              // azimuth points of a reflection are dealt round-robin to n_split warps per patch
    float2 *partial;          // [n_split][n_y][n_x] float-float partial sums (int32 in count mode); null if n_split == 1
    float dpsi_extra;         // widening of the reach window for query points off the meridional plane
};
cudaError_t launch_ring(const RingParams &p, int lineshape, bool count_mode, cudaStream_t s);
void sf_plan(int n_atoms, int n_refl, int n_elem, int max_split, int &n_split, int &per);
// Element passes of the structure factors (form-factor tables of at most 40
// types in shared memory): each pass writes its own n_split rows of partials.
int sf_passes(int n_elem);

// Host-side argument checks shared by the entry points (fdx_api.cu).
int validate_cell(const fdx_cell *c);
int validate_broadening(const fdx_broadening *b);
size_t sf_bind(SFParams *p, char *ws, int n_atoms, int n_refl, int max_split);

}  // namespace fdx
