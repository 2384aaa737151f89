// Parameters of the refinement kernels (fdx_adjoint.cu).
#pragma once

#include "fdx_internal.cuh"

namespace fdx {

struct AdjParams {
    PatternParams P;           // geometry, records, node tables (image/counts unused)
    float4 *patch_bounds;      // [npy][npx] (|S| min, max, psi min, max)
    float4 *band_bounds;       // [n_bands]
    int npx, npy, n_bands, rows_per_band;
    const float *gI;           // [ny][nx] dL/dI
    double *item_out;          // [n_refl * n_bands][6]
    double *refl_out;          // [n_refl][8] per-reflection global contributions
    float4 *cF;                // [n_refl] (dL/dM P DW conj(F), s^2)
    float *fe;                 // [n_refl][n_elem] form factors at the reflection
    float *dM;                 // [n_refl] dL/dM (may be null)
    unsigned *counter;         // item queue of the single-model adjoint launch (zeroed by launch_adjoint)
    double *dglobal;           // [8] (may be null)
    const int32_t *hkl;
    const float *F;            // [n_refl][2]
    const float *ff;           // [n_elem][9]
    int n_elem, intensity_model;
    int lineshape;             // FDX_LINESHAPE_*: the Hosemann walk's sums are relative, the others absolute
    double As[9];
    double alen[3], L[3], g[3], Bax[3];
};

// Adjoint over the models of one tile shape (adjoint_batch_kernel<PPL>), with
// position tables as for the forward ((reflection, band) items).
struct BatchAdjParams {
    const AdjParams *models;       // [n_models] device, by model index
    const long long *item_prefix;  // [n_models] by position: the model's first item
    const int *item_model;         // [n_models] by position: the model index
    int pos0, n_pos;
    long long item0, item_end;
    unsigned *counter;             // zeroed before the launch
};

struct SFAdjParams {
    int n_atoms, n_elem, n_refl, n_split, refl_per_split;
    const uint4 *atoms_q;
    const float2 *atoms_w;
    const int32_t *hkl;
    const float4 *cF;
    const float *fe;
    double *partial;           // [n_split][n_atoms][4]
    double *dfrac, *dB;
};

struct LossParams {
    long long n;
    const float *I, *It, *mask;
    float *gI;
    double *partial;           // [n_blocks]
    double *loss;
};

struct Plain64Params {
    int nx, ny, n_refl, n, n_atoms, n_elem, npx, npy, n_bands, rows_per_band, intensity_model;
    double T, h, delta_L;
    double A[9], As[9], nh[3], bh[3], alen[3], L[3], g[3], Bax[3];
    const float4 *pixgeo, *reach, *patch_bounds, *band_bounds;
    double *recs64;          // [n_refl][48]
    const double *nodes64;   // [n*n][4]: w, -, dw/dsigma, dw/dgamma
    double *image64;         // [ny][nx]
    const double *It64;      // [ny][nx] target
    const float *mask;       // [ny][nx] or null
    double *gI, *loss, *loss_partial;
    const int32_t *hkl;
    double *F64, *M64, *Gw64;
    double *item_out, *refl_out;
    const double *frac;
    const float *B, *occ, *ff;
    const uint8_t *elem;
    double *dfrac, *dB;
};

cudaError_t launch_adjoint(AdjParams &A, int n_ctas, cudaStream_t s);
cudaError_t launch_bounds_only(AdjParams &A, cudaStream_t s);
cudaError_t launch_adjoint_batch(const BatchAdjParams &B, int ppl, int n_ctas, cudaStream_t s);
cudaError_t launch_adjoint_post(AdjParams &A, cudaStream_t s);
cudaError_t launch_globals_only(AdjParams &A, cudaStream_t s);
cudaError_t launch_plain64_forward(Plain64Params &p, cudaStream_t s);
cudaError_t launch_plain64_loss(Plain64Params &p, cudaStream_t s);
cudaError_t launch_plain64_backward(Plain64Params &p, AdjParams &A, cudaStream_t s);
cudaError_t launch_sf_adjoint(SFAdjParams &p, cudaStream_t s);
cudaError_t launch_loss(LossParams &p, cudaStream_t s);
cudaError_t launch_sf_pack(SFParams &p, cudaStream_t s);

}  // namespace fdx
