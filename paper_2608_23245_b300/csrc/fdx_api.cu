// C-ABI entry points of libfdx: argument validation on the host, workspace
// carving, and kernel launches on the caller's stream.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "fdx_adjoint.cuh"
#include "fdx_internal.cuh"

using namespace fdx;

namespace {

constexpr size_t kAlign = 256;

std::mutex g_tune_mu;
fdx_tuning g_tune = {2, 4, 3, 128, 1};

fdx_tuning tuning() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool finite3(const double *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

}  // namespace

namespace fdx {

int validate_cell(const fdx_cell *c) {
    if (!c) return FDX_ERR_ARG;
    const double v[6] = {c->a, c->b, c->c, c->alpha, c->beta, c->gamma};
    for (double x : v)
        if (!isfinite(x)) return FDX_ERR_ARG;
    if (c->a <= 0 || c->b <= 0 || c->c <= 0) return FDX_ERR_GEOMETRY;
    for (int k = 3; k < 6; ++k)
        if (v[k] <= 0 || v[k] >= FDX_PI) return FDX_ERR_GEOMETRY;
    // positive cell volume: 1 - cos^2 a - cos^2 b - cos^2 g + 2 cos a cos b cos g > 0
    const double ca = cos(c->alpha), cb = cos(c->beta), cg = cos(c->gamma);
    if (1 - ca * ca - cb * cb - cg * cg + 2 * ca * cb * cg <= 1e-12) return FDX_ERR_GEOMETRY;
    return FDX_OK;
}

int validate_broadening(const fdx_broadening *b) {
    if (!b) return FDX_ERR_ARG;
    for (int i = 0; i < 3; ++i) {
        if (!(b->L[i] > 0) || !isfinite(b->L[i])) return FDX_ERR_ARG;
        if (!(b->g[i] >= 0) || !isfinite(b->g[i])) return FDX_ERR_ARG;
        if (!isfinite(b->B_axis[i])) return FDX_ERR_ARG;
    }
    if (b->lineshape != FDX_LINESHAPE_SINC && b->lineshape != FDX_LINESHAPE_HOSEMANN &&
        b->lineshape != FDX_LINESHAPE_GAUSS)
        return FDX_ERR_ARG;
    if (b->intensity_model != FDX_INTENSITY_NONE && b->intensity_model != FDX_INTENSITY_HOSEMANN) return FDX_ERR_ARG;
    if (!(b->sigma >= 0) || !(b->gamma >= 0) || !isfinite(b->sigma) || !isfinite(b->gamma)) return FDX_ERR_ARG;
    if (b->gamma == 0 && !(b->sigma > 0)) return FDX_ERR_ARG;  // no angular shape
    if (!(b->sigma_r > 0) || !isfinite(b->sigma_r)) return FDX_ERR_ARG;
    if (!(b->T > 0) || !isfinite(b->T)) return FDX_ERR_ARG;
    if (b->n_nodes < 1 || b->n_nodes > 512) return FDX_ERR_ARG;
    if (!(b->K_z > 0) || !isfinite(b->K_z)) return FDX_ERR_ARG;
    return FDX_OK;
}

}  // namespace fdx

namespace {

int validate_geometry(const fdx_geometry *g) {
    if (!g) return FDX_ERR_ARG;
    if (!(g->wavelength > 0) || !(g->distance > 0) || !(g->pixel > 0) || !(g->delta_L > 0)) return FDX_ERR_ARG;
    if (!isfinite(g->wavelength) || !isfinite(g->distance) || !isfinite(g->pixel) || !isfinite(g->delta_L))
        return FDX_ERR_ARG;
    if (g->n_x < 1 || g->n_y < 1 || g->n_x > 16384 || g->n_y > 16384) return FDX_ERR_ARG;
    if (!finite3(g->fiber_axis) || !finite3(g->beam_axis)) return FDX_ERR_ARG;
    const double nf = sqrt(g->fiber_axis[0] * g->fiber_axis[0] + g->fiber_axis[1] * g->fiber_axis[1] +
                           g->fiber_axis[2] * g->fiber_axis[2]);
    const double nb = sqrt(g->beam_axis[0] * g->beam_axis[0] + g->beam_axis[1] * g->beam_axis[1] +
                           g->beam_axis[2] * g->beam_axis[2]);
    if (!(nf > 0) || !(nb > 0)) return FDX_ERR_ARG;
    const double c = (g->fiber_axis[0] * g->beam_axis[0] + g->fiber_axis[1] * g->beam_axis[1] +
                      g->fiber_axis[2] * g->beam_axis[2]) / (nf * nb);
    // any fiber tilt towards the beam (Sect. Experimental geometry: tilt); the
    // detector's vertical axis is the fiber axis projected onto it
    if (fabs(c) > 1.0 - 1e-6) return FDX_ERR_GEOMETRY;
    return FDX_OK;
}

int validate_problem(const fdx_problem *p) {
    if (!p) return FDX_ERR_ARG;
    int rc = validate_cell(&p->cell);
    if (rc) return rc;
    if ((rc = validate_broadening(&p->br))) return rc;
    if ((rc = validate_geometry(&p->geom))) return rc;
    if (p->n_refl < 0) return FDX_ERR_ARG;
    if (p->n_refl > 0 && (!p->hkl || !p->M)) return FDX_ERR_ARG;
    return FDX_OK;
}

struct Layout {
    size_t pixgeo, nodes, dnodes, recs, reach, total;
};

Layout layout_for(const fdx_problem *p) {
    Layout L;
    size_t off = 0;
    L.pixgeo = off;
    off += align_up(sizeof(float4) * (size_t)p->geom.n_x * p->geom.n_y);
    L.nodes = off;
    off += align_up(2 * sizeof(float4) * (size_t)p->br.n_nodes * p->br.n_nodes);
    L.dnodes = off;
    off += align_up(sizeof(float2) * (size_t)p->br.n_nodes * p->br.n_nodes);
    L.recs = off;
    off += align_up(sizeof(float) * REC_SIZE * (size_t)(p->n_refl > 0 ? p->n_refl : 1));
    L.reach = off;
    off += align_up(sizeof(float4) * (size_t)(p->n_refl > 0 ? p->n_refl : 1));
    L.total = off;
    return L;
}

void unit3(const double *v, double *o) {
    const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int q = 0; q < 3; ++q) o[q] = v[q] / n;
}

void cross3(const double *x, const double *y, double *z) {
    z[0] = x[1] * y[2] - x[2] * y[1];
    z[1] = x[2] * y[0] - x[0] * y[2];
    z[2] = x[0] * y[1] - x[1] * y[0];
}

// Two pixels per lane (8 x 8 warp patches) when the patch spans at most half
// a lattice period along every cell axis: pitch in S (largest at the beam
// centre) x 8 sqrt 2 x max |a_i| <= 0.5; otherwise one (8 x 4).
int pattern_ppl(const fdx_problem *p) {
    double A[9], As[9];
    cell_basis(p->cell, A, As);
    const double pitch = p->geom.pixel / (p->geom.wavelength * p->geom.distance);
    double amax = 0.0;
    for (int i = 0; i < 3; ++i) amax = fmax(amax, sqrt(A[3 * i] * A[3 * i] + A[3 * i + 1] * A[3 * i + 1] + A[3 * i + 2] * A[3 * i + 2]));
    return (pitch * 8.0 * sqrt(2.0) * amax <= 0.5 && tuning().ppl_max >= 2) ? 2 : 1;
}

// Queue the set-up kernels (pixel geometry, node table, reflection records)
// for one problem and fill the pattern kernel's parameters.
int setup_pattern(const fdx_problem *p, char *ws, cudaStream_t st, PatternParams &P, bool with_dnodes,
                  double *nodes64 = nullptr, double *frames = nullptr, float *ring = nullptr) {
    const Layout L = layout_for(p);
    double A[9], As[9];
    cell_basis(p->cell, A, As);
    double nh[3], bh[3], uh[3], vh[3];
    unit3(p->geom.fiber_axis, nh);
    unit3(p->geom.beam_axis, bh);
    cross3(nh, bh, uh);
    unit3(uh, uh);
    cross3(bh, uh, vh);

    PixelParams pp;
    pp.nx = p->geom.n_x, pp.ny = p->geom.n_y;
    pp.lambda = p->geom.wavelength, pp.dist = p->geom.distance, pp.pix = p->geom.pixel;
    for (int q = 0; q < 3; ++q) pp.bh[q] = bh[q], pp.uh[q] = uh[q], pp.vh[q] = vh[q], pp.nh[q] = nh[q];
    pp.pixgeo = reinterpret_cast<float4 *>(ws + L.pixgeo);
    if (launch_pixel_geometry(pp, st) != cudaSuccess) return FDX_ERR_CUDA;

    NodeParams np;
    np.n = p->br.n_nodes, np.T = p->br.T, np.h = 2.0 * p->br.T / p->br.n_nodes;
    np.sigma = p->br.sigma, np.gamma = p->br.gamma, np.sigma_r = p->br.sigma_r;
    np.nodes = reinterpret_cast<float4 *>(ws + L.nodes);
    np.dnodes = with_dnodes ? reinterpret_cast<float2 *>(ws + L.dnodes) : nullptr;
    np.nodes64 = nodes64;
    if (launch_nodes(np, weideman_coeffs(), st) != cudaSuccess) return FDX_ERR_CUDA;

    ReflSetupParams rp;
    memcpy(rp.A, A, sizeof A);
    memcpy(rp.As, As, sizeof As);
    for (int q = 0; q < 3; ++q) {
        rp.nh[q] = nh[q], rp.bh[q] = bh[q];
        rp.alen[q] = sqrt(A[3 * q] * A[3 * q] + A[3 * q + 1] * A[3 * q + 1] + A[3 * q + 2] * A[3 * q + 2]);
        rp.L[q] = p->br.L[q], rp.g[q] = p->br.g[q], rp.Bax[q] = p->br.B_axis[q];
    }
    rp.T = p->br.T, rp.K_z = p->br.K_z;
    rp.lineshape = p->br.lineshape, rp.intensity_model = p->br.intensity_model, rp.n_refl = p->n_refl, rp.pad = 0;
    rp.hkl = p->hkl, rp.M = p->M;
    rp.recs = reinterpret_cast<float *>(ws + L.recs);
    rp.reach = reinterpret_cast<float4 *>(ws + L.reach);
    rp.frames = frames;
    rp.ring = ring;
    rp.ring_max_n = FDX_RING_MAX_N;
    for (int q = 0; q < 3; ++q) rp.alen3[q] = rp.alen[q];
    if (launch_refl_setup(rp, st) != cudaSuccess) return FDX_ERR_CUDA;

    P.nx = p->geom.n_x, P.ny = p->geom.n_y, P.n_refl = p->n_refl, P.n_nodes = p->br.n_nodes;
    P.T = (float)p->br.T;
    P.inv_h = (float)(p->br.n_nodes / (2.0 * p->br.T));
    for (int i = 0; i < 3; ++i) P.AZ[i] = (float)(A[3 * i] * nh[0] + A[3 * i + 1] * nh[1] + A[3 * i + 2] * nh[2]);
    P.delta_L = p->geom.delta_L;
    P.ppl = pattern_ppl(p);
    // node blocks of the culling: 2^blk_lr rows x 2^blk_lc columns, 32 nodes
    {
        static const int lr[4] = {2, 3, 1, 4};
        const int nb = tuning().node_block;
        P.blk_lr = lr[nb], P.blk_lc = 5 - lr[nb];
    }
    P.pixgeo = pp.pixgeo;
    P.reach = rp.reach;
    P.recs = rp.recs;
    P.nodes = np.nodes;
    P.dnodes = np.dnodes;
    P.image = nullptr;
    P.counts = nullptr;
    return FDX_OK;
}

// Queue set-up kernels and the pattern kernel for one problem.
int run_pattern(const fdx_problem *p, float *image, int32_t *counts, char *ws, cudaStream_t st) {
    PatternParams P;
    int rc = setup_pattern(p, ws, st, P, false);
    if (rc) return rc;
    P.image = image;
    P.counts = counts;
    if (launch_pattern(P, p->br.lineshape, counts != nullptr, st) != cudaSuccess) return FDX_ERR_CUDA;
    return FDX_OK;
}

// Backward workspace: the forward layout followed by the adjoint buffers.
struct BackLayout {
    size_t fwd, patch_bounds, band_bounds, item_out, refl_out, cF, fe, atoms_q, atoms_w, sf_partial, counter, total;
    int npx, npy, n_bands, rows_per_band, sf_split, refl_per_split;
};

BackLayout back_layout(const fdx_problem *p, int n_atoms, int n_elem) {
    BackLayout B;
    const size_t nr = (size_t)(p->n_refl > 0 ? p->n_refl : 1);
    B.npx = (p->geom.n_x + 7) / 8, B.npy = (p->geom.n_y + 3) / 4;
    const int want_bands = tuning().adj_bands;
    B.n_bands = B.npy < want_bands ? B.npy : want_bands;
    B.rows_per_band = (B.npy + B.n_bands - 1) / B.n_bands;
    B.rows_per_band += B.rows_per_band & 1;  // even: 8 x 8 adjoint patches (two bound rows) never straddle bands
    B.n_bands = (B.npy + B.rows_per_band - 1) / B.rows_per_band;
    const int atom_blocks = (n_atoms + 127) / 128;
    int split = (600 + atom_blocks - 1) / atom_blocks;
    const int by_refl = (int)((nr + 255) / 256);
    if (split > by_refl) split = by_refl;
    if (split > 64) split = 64;
    if (split < 1) split = 1;
    int per = (int)((nr + split - 1) / split);
    per = (per + 127) / 128 * 128;
    split = (int)((nr + per - 1) / per);
    B.sf_split = split, B.refl_per_split = per;
    size_t off = layout_for(p).total;
    B.fwd = 0;
    B.patch_bounds = off;
    off += align_up(sizeof(float4) * (size_t)B.npx * B.npy);
    B.band_bounds = off;
    off += align_up(sizeof(float4) * (size_t)B.n_bands);
    B.item_out = off;
    off += align_up(sizeof(double) * 6 * nr * B.n_bands);
    B.refl_out = off;
    off += align_up(sizeof(double) * 8 * nr);
    B.cF = off;
    off += align_up(sizeof(float4) * nr);
    B.fe = off;
    off += align_up(sizeof(float) * nr * (size_t)(n_elem > 0 ? n_elem : 1));
    B.atoms_q = off;
    off += align_up(sizeof(uint4) * (size_t)n_atoms);
    B.atoms_w = off;
    off += align_up(sizeof(float2) * (size_t)n_atoms);
    B.sf_partial = off;
    off += align_up(sizeof(double) * 4 * (size_t)split * (size_t)n_atoms);
    B.counter = off;
    off += align_up(sizeof(unsigned));
    B.total = off;
    return B;
}

// Writes one model's parameter blocks and item prefixes into the batch tables
// (a kernel, so that the whole batch step can be captured in a CUDA graph).
// One model's parameter blocks (at its index) and its entries of the
// position tables (at its position; models are ordered by tile shape).
__global__ void batch_write_params(PatternParams *fdst, const PatternParams P, AdjParams *adst, const AdjParams A,
                                   long long *fpre, long long fp, long long *apre, long long ap, int *fmod, int *amod,
                                   int m) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *fdst = P;
        *adst = A;
        *fpre = fp;
        *apre = ap;
        *fmod = m;
        *amod = m;
    }
}

struct BatchLayout {
    size_t fwd_tab, adj_tab, fpre, apre, fmod, amod, counters, head;
    std::vector<size_t> region, back, sf, gI, loss;
    size_t total;
};

BatchLayout batch_layout(int n, const fdx_problem *const *probs, const fdx_atoms *const *atoms) {
    BatchLayout L;
    size_t off = 0;
    L.fwd_tab = off, off += align_up(sizeof(PatternParams) * n);
    L.adj_tab = off, off += align_up(sizeof(AdjParams) * n);
    L.fpre = off, off += align_up(sizeof(long long) * n);
    L.apre = off, off += align_up(sizeof(long long) * n);
    L.fmod = off, off += align_up(sizeof(int) * n);
    L.amod = off, off += align_up(sizeof(int) * n);
    L.counters = off, off += align_up(sizeof(unsigned) * 4);
    L.head = off;
    for (int m = 0; m < n; ++m) {
        const fdx_problem *p = probs[m];
        const size_t npx = (size_t)p->geom.n_x * p->geom.n_y;
        L.region.push_back(off);
        L.back.push_back(off), off += back_layout(p, atoms[m]->n_atoms, atoms[m]->n_elem).total;
        L.sf.push_back(off), off += align_up(fdx_sf_workspace_size(atoms[m]->n_atoms, p->n_refl > 0 ? p->n_refl : 1));
        L.gI.push_back(off), off += align_up(sizeof(float) * npx);
        L.loss.push_back(off), off += align_up(sizeof(double) * ((npx + 255) / 256));
    }
    L.total = off;
    return L;
}

// Scatter-form workspace: the pattern layout (records, nodes) followed by the
// FP64 reflection frames and their projections, the per-sample table and the
// FP64 image.
struct ScatterLayout {
    size_t frames, proj, stab, img64, total;
};

ScatterLayout scatter_layout(const fdx_problem *p, int n_s) {
    ScatterLayout S;
    size_t off = layout_for(p).total;
    S.frames = off, off += align_up(sizeof(double) * 12 * (size_t)(p->n_refl > 0 ? p->n_refl : 1));
    S.proj = off, off += align_up(sizeof(float2) * SCAT_PROJ * (size_t)(p->n_refl > 0 ? p->n_refl : 1));
    S.stab = off, off += align_up(sizeof(float4) * 3 * (size_t)n_s);
    S.img64 = off, off += align_up(sizeof(double) * (size_t)p->geom.n_x * p->geom.n_y);
    S.total = off;
    return S;
}

int run_scatter(const fdx_problem *prob, int32_t n_s, const float *samples, int32_t spot, float *image,
                int64_t *count, void *workspace, size_t ws_bytes, void *stream) {
    int rc = validate_problem(prob);
    if (rc) return rc;
    if (n_s < 1 || !samples || ((uintptr_t)samples % 16)) return FDX_ERR_ARG;
    if (spot < 1 || spot > 15 || spot % 2 == 0) return FDX_ERR_ARG;
    const ScatterLayout SL = scatter_layout(prob, n_s);
    if (!workspace || ws_bytes < SL.total || ((uintptr_t)workspace % kAlign)) return FDX_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    const size_t npx = (size_t)prob->geom.n_x * prob->geom.n_y;
    if (prob->n_refl == 0) {
        if (image && cudaMemsetAsync(image, 0, sizeof(float) * npx, st) != cudaSuccess) return FDX_ERR_CUDA;
        if (count && cudaMemsetAsync(count, 0, sizeof(int64_t), st) != cudaSuccess) return FDX_ERR_CUDA;
        return FDX_OK;
    }
    ScatterParams S;
    memset(&S, 0, sizeof S);
    rc = setup_pattern(prob, ws, st, S.P, false, nullptr, reinterpret_cast<double *>(ws + SL.frames));
    if (rc) return rc;
    S.n_s = n_s;
    S.spot = spot;
    S.samples = reinterpret_cast<const float4 *>(samples);
    S.stab = reinterpret_cast<float4 *>(ws + SL.stab);
    S.frames = reinterpret_cast<const double *>(ws + SL.frames);
    S.T = prob->br.T, S.lambda = prob->geom.wavelength, S.dist = prob->geom.distance, S.pix = prob->geom.pixel;
    S.delta_L = prob->geom.delta_L;
    unit3(prob->geom.fiber_axis, S.nh);
    unit3(prob->geom.beam_axis, S.bh);
    cross3(S.nh, S.bh, S.uh);
    unit3(S.uh, S.uh);
    cross3(S.bh, S.uh, S.vh);
    S.proj = reinterpret_cast<float2 *>(ws + SL.proj);
    const double *w3[3] = {S.uh, S.vh, S.bh};
    for (int q = 0; q < 3; ++q) S.wdir[0][q] = S.nh[q];
    for (int j = 0; j < 3; ++j) {
        for (int q = 0; q < 3; ++q) S.wdir[1 + j][q] = w3[j][q];
        cross3(w3[j], S.nh, S.wdir[4 + j]);
        S.kw[j] = (S.bh[0] * w3[j][0] + S.bh[1] * w3[j][1] + S.bh[2] * w3[j][2]) / S.lambda;
        S.nw[j] = S.nh[0] * w3[j][0] + S.nh[1] * w3[j][1] + S.nh[2] * w3[j][2];
    }
    S.il = 1.0 / S.lambda;
    S.kn = (S.bh[0] * S.nh[0] + S.bh[1] * S.nh[1] + S.bh[2] * S.nh[2]) / S.lambda;
    S.dp = S.dist / S.pix;
    S.hx = 0.5 * prob->geom.n_x, S.hy = 0.5 * prob->geom.n_y;
    auto ffv = [](double x) { float h, l; split_double(x, h, l); return make_float2(h, l); };
    S.il_f = ffv(S.il), S.kn_f = ffv(S.kn), S.dp_f = ffv(S.dp), S.hx_f = ffv(S.hx), S.hy_f = ffv(S.hy);
    for (int j = 0; j < 3; ++j) S.kw_f[j] = ffv(S.kw[j]), S.nw_f[j] = ffv(S.nw[j]);
    S.img64 = reinterpret_cast<double *>(ws + SL.img64);
    S.image = image;
    S.count = reinterpret_cast<unsigned long long *>(count);
    if (image && cudaMemsetAsync(S.img64, 0, sizeof(double) * npx, st) != cudaSuccess) return FDX_ERR_CUDA;
    if (count && cudaMemsetAsync(count, 0, sizeof(int64_t), st) != cudaSuccess) return FDX_ERR_CUDA;
    if (launch_scatter(S, prob->br.lineshape, count != nullptr, st) != cudaSuccess) return FDX_ERR_CUDA;
    return FDX_OK;
}

// Warps per 8 x 4 RING_PPL patch of the ring average: about 32768 warps in all
// (some fourteen waves of 16 resident warps on each of 148 SMs), at most 128;
// one per patch once the patches alone give 16384 warps (seven waves).
int ring_split(const fdx_problem *p) {
    const long long patches = (long long)((p->geom.n_x + 7) / 8) * ((p->geom.n_y + 4 * RING_PPL - 1) / (4 * RING_PPL));
    if (patches >= 16384) return 1;
    const long long s = (32768 + patches - 1) / (patches > 0 ? patches : 1);
    return (int)(s < 1 ? 1 : (s > 128 ? 128 : s));
}

// Ring-average workspace: the pattern layout followed by the ring records and,
// when the azimuth points are split, the partial images.
size_t ring_layout(const fdx_problem *p, size_t *ring_off, size_t *part_off = nullptr) {
    size_t off = layout_for(p).total;
    *ring_off = off;
    off += align_up(sizeof(float) * RING_REC * (size_t)(p->n_refl > 0 ? p->n_refl : 1));
    if (part_off) *part_off = off;
    const int S = ring_split(p);
    if (S > 1) off += align_up(sizeof(float2) * (size_t)S * p->geom.n_x * p->geom.n_y);
    return off;
}

int run_ring(const fdx_problem *prob, float *image, int32_t *counts, void *workspace, size_t ws_bytes, void *stream) {
    int rc = validate_problem(prob);
    if (rc) return rc;
    if (!image && !counts) return FDX_ERR_ARG;
    size_t roff = 0, poff = 0;
    const size_t need = ring_layout(prob, &roff, &poff);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign)) return FDX_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    RingParams R;
    memset(&R, 0, sizeof R);
    rc = setup_pattern(prob, ws, st, R.P, false, nullptr, nullptr, reinterpret_cast<float *>(ws + roff));
    if (rc) return rc;
    R.P.image = image;
    R.P.counts = counts;
    R.ring = reinterpret_cast<const float *>(ws + roff);
    R.n_split = ring_split(prob);
    R.dpsi_extra = (float)((atan(prob->br.T * sqrt(2.0)) - atan(prob->br.T)) * (1.0 + 1e-4) + 1e-6);
    R.partial = R.n_split > 1 ? reinterpret_cast<float2 *>(ws + poff) : nullptr;
    if (launch_ring(R, prob->br.lineshape, counts != nullptr, st) != cudaSuccess) return FDX_ERR_CUDA;
    return FDX_OK;
}

}  // namespace

// The debugging build's status word (declared in fdx_internal.cuh, C++
// linkage) and its probe kernel.
#ifdef FDX_DEBUG
__device__ unsigned long long fdx_debug_word[2];

// One check that fails on purpose (index 7 of a 3-entry range, check 63):
// nothing is accessed, only the status word is written.
__global__ void debug_probe_kernel() {
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)FDX_IN_BOUNDS(7, 3, 63);
}
#endif

extern "C" {

size_t fdx_batch_workspace_size(int32_t n_models, const fdx_problem *const *probs, const fdx_atoms *const *atoms) {
    if (n_models < 1 || !probs || !atoms) return 0;
    for (int m = 0; m < n_models; ++m)
        if (!probs[m] || !atoms[m] || atoms[m]->n_atoms < 1 || atoms[m]->n_elem < 1) return 0;
    return batch_layout(n_models, probs, atoms).total;
}

int fdx_batch_refine(int32_t n_models, const fdx_problem *const *probs, const fdx_atoms *const *atoms,
                     float *const *F, float *const *M, float *const *images, const float *const *targets,
                     const float *const *masks, double *losses, const fdx_grads *const *grads, void *workspace,
                     size_t ws_bytes, void *stream) {
    if (n_models < 1 || !probs || !atoms || !F || !M || !images) return FDX_ERR_ARG;
    if (targets && (!losses || !grads)) return FDX_ERR_ARG;
    for (int m = 0; m < n_models; ++m) {
        if (!probs[m] || !atoms[m] || !images[m]) return FDX_ERR_ARG;
        fdx_problem pr = *probs[m];
        pr.M = M[m];
        int rc = validate_problem(&pr);
        if (rc) return rc;
        if (pr.br.lineshape != FDX_LINESHAPE_HOSEMANN) return FDX_ERR_ARG;
        const fdx_atoms *a = atoms[m];
        if (a->n_atoms < 1 || a->n_elem < 1 || a->n_elem > 64 || !a->frac || !a->B || !a->elem || !a->ff)
            return FDX_ERR_ARG;
        if (pr.n_refl > 0 && (!F[m] || !M[m])) return FDX_ERR_ARG;
        if (targets && (!targets[m] || !grads[m])) return FDX_ERR_ARG;
    }
    const BatchLayout L = batch_layout(n_models, probs, atoms);
    if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace % kAlign)) return FDX_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    int dev = 0, n_sm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDX_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    unsigned *counters = reinterpret_cast<unsigned *>(ws + L.counters);
    if (cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned), st) != cudaSuccess) return FDX_ERR_CUDA;

    // Models ordered by tile shape (two pixels per lane first): each shape's
    // forward and adjoint run as persistent launches of their own, each
    // compiled for that shape.  Item counts and offsets per model, on the host.
    std::vector<int> ppl(n_models), pos(n_models);
    std::vector<long long> fitems(n_models), aitems(n_models), fstart(n_models), astart(n_models);
    int n_pos2 = 0;
    for (int m = 0; m < n_models; ++m) {
        fdx_problem pr = *probs[m];
        pr.M = M[m];
        ppl[m] = pattern_ppl(&pr);
        fitems[m] = (long long)((pr.geom.n_x + 15) / 16) * ((pr.geom.n_y + 8 * ppl[m] - 1) / (8 * ppl[m]));
        aitems[m] = (long long)pr.n_refl * back_layout(&pr, atoms[m]->n_atoms, atoms[m]->n_elem).n_bands;
        n_pos2 += ppl[m] == 2;
    }
    long long f_split = 0, a_split = 0, fsum = 0, asum = 0;  // items of the two-pixel models; totals
    for (int cls = 2, next = 0; cls >= 1; --cls) {
        if (cls == 1) f_split = fsum, a_split = asum;
        for (int m = 0; m < n_models; ++m) {
            if (ppl[m] != cls) continue;
            pos[m] = next++, fstart[m] = fsum, astart[m] = asum;
            fsum += fitems[m], asum += aitems[m];
        }
    }

    std::vector<AdjParams> adj(n_models);
    for (int m = 0; m < n_models; ++m) {
        fdx_problem pr = *probs[m];
        pr.M = M[m];
        const fdx_atoms *a = atoms[m];
        char *reg = ws + L.back[m];
        // structure factors -> F, M
        if (pr.n_refl > 0) {
            SFParams sp;
            memset(&sp, 0, sizeof sp);
            double Am[9], As[9];
            cell_basis(pr.cell, Am, As);
            memcpy(sp.As, As, sizeof As);
            sp.n_atoms = a->n_atoms, sp.n_elem = a->n_elem, sp.n_refl = pr.n_refl;
            int n_split = 1, per = 1;
            sf_plan(a->n_atoms, pr.n_refl, a->n_elem, 64, n_split, per);
            sp.n_split = n_split;
            sp.frac = a->frac, sp.B = a->B, sp.occ = a->occ, sp.ff = a->ff, sp.elem = a->elem;
            sf_bind(&sp, ws + L.sf[m], a->n_atoms, pr.n_refl, 64);
            sp.hkl = pr.hkl, sp.F_out = F[m], sp.M_out = M[m];
            sp.has_br = 1, sp.intensity_model = pr.br.intensity_model;
            for (int i = 0; i < 3; ++i) {
                sp.g[i] = pr.br.g[i], sp.Bax[i] = pr.br.B_axis[i];
                sp.alen[i] = sqrt(Am[3 * i] * Am[3 * i] + Am[3 * i + 1] * Am[3 * i + 1] + Am[3 * i + 2] * Am[3 * i + 2]);
            }
            if (launch_structure_factors(sp, st) != cudaSuccess) return FDX_ERR_CUDA;
        }
        // set-up kernels and parameter blocks
        PatternParams P;
        int rc = setup_pattern(&pr, reg, st, P, targets != nullptr);
        if (rc) return rc;
        P.image = images[m];
        P.counts = nullptr;
        const BackLayout B = back_layout(&pr, a->n_atoms, a->n_elem);
        AdjParams &A = adj[m];
        memset(&A, 0, sizeof A);
        A.P = P;
        double Am[9], As[9];
        cell_basis(pr.cell, Am, As);
        memcpy(A.As, As, sizeof As);
        for (int i = 0; i < 3; ++i) {
            A.alen[i] = sqrt(Am[3 * i] * Am[3 * i] + Am[3 * i + 1] * Am[3 * i + 1] + Am[3 * i + 2] * Am[3 * i + 2]);
            A.L[i] = pr.br.L[i], A.g[i] = pr.br.g[i], A.Bax[i] = pr.br.B_axis[i];
        }
        A.patch_bounds = reinterpret_cast<float4 *>(reg + B.patch_bounds);
        A.band_bounds = reinterpret_cast<float4 *>(reg + B.band_bounds);
        A.npx = B.npx, A.npy = B.npy, A.n_bands = B.n_bands, A.rows_per_band = B.rows_per_band;
        A.gI = reinterpret_cast<float *>(ws + L.gI[m]);
        A.item_out = reinterpret_cast<double *>(reg + B.item_out);
        A.refl_out = reinterpret_cast<double *>(reg + B.refl_out);
        A.cF = reinterpret_cast<float4 *>(reg + B.cF);
        A.fe = reinterpret_cast<float *>(reg + B.fe);
        A.dM = targets ? grads[m]->dM : nullptr;
        A.dglobal = targets ? grads[m]->dglobal : nullptr;
        A.hkl = pr.hkl, A.F = F[m], A.ff = a->ff, A.n_elem = a->n_elem, A.intensity_model = pr.br.intensity_model;
        A.lineshape = pr.br.lineshape;
        if (P.ppl != ppl[m] || B.n_bands * (long long)pr.n_refl != aitems[m]) return FDX_ERR_ARG;  // cannot happen
        const int j = pos[m];
        batch_write_params<<<1, 32, 0, st>>>(reinterpret_cast<PatternParams *>(ws + L.fwd_tab) + m, P,
                                             reinterpret_cast<AdjParams *>(ws + L.adj_tab) + m, A,
                                             reinterpret_cast<long long *>(ws + L.fpre) + j, fstart[m],
                                             reinterpret_cast<long long *>(ws + L.apre) + j, astart[m],
                                             reinterpret_cast<int *>(ws + L.fmod) + j,
                                             reinterpret_cast<int *>(ws + L.amod) + j, m);
        if (cudaGetLastError() != cudaSuccess) return FDX_ERR_CUDA;
    }
    // one persistent forward launch per tile shape over its models
    const fdx_tuning tu = tuning();
    for (int cls = 2; cls >= 1; --cls) {
        BatchFwdParams BF;
        BF.models = reinterpret_cast<const PatternParams *>(ws + L.fwd_tab);
        BF.item_prefix = reinterpret_cast<const long long *>(ws + L.fpre);
        BF.item_model = reinterpret_cast<const int *>(ws + L.fmod);
        BF.pos0 = cls == 2 ? 0 : n_pos2, BF.n_pos = cls == 2 ? n_pos2 : n_models - n_pos2;
        BF.item0 = cls == 2 ? 0 : f_split, BF.item_end = cls == 2 ? f_split : fsum;
        BF.counter = counters + (cls == 2 ? 0 : 1);
        if (BF.n_pos > 0 && BF.item_end > BF.item0 &&
            launch_pattern_batch(BF, cls, n_sm * tu.fwd_ctas_per_sm, st) != cudaSuccess)
            return FDX_ERR_CUDA;
    }
    if (!targets) return FDX_OK;

    for (int m = 0; m < n_models; ++m) {
        const fdx_problem *pr = probs[m];
        LossParams lp;
        lp.n = (long long)pr->geom.n_x * pr->geom.n_y, lp.I = images[m], lp.It = targets[m];
        lp.mask = masks ? masks[m] : nullptr, lp.gI = adj[m].gI == nullptr ? nullptr : const_cast<float *>(adj[m].gI);
        lp.partial = reinterpret_cast<double *>(ws + L.loss[m]);
        lp.loss = losses + m;
        if (launch_loss(lp, st) != cudaSuccess) return FDX_ERR_CUDA;
        if (launch_bounds_only(adj[m], st) != cudaSuccess) return FDX_ERR_CUDA;
    }
    // one persistent adjoint launch per tile shape over its models
    for (int cls = 2; cls >= 1; --cls) {
        BatchAdjParams BA;
        BA.models = reinterpret_cast<const AdjParams *>(ws + L.adj_tab);
        BA.item_prefix = reinterpret_cast<const long long *>(ws + L.apre);
        BA.item_model = reinterpret_cast<const int *>(ws + L.amod);
        BA.pos0 = cls == 2 ? 0 : n_pos2, BA.n_pos = cls == 2 ? n_pos2 : n_models - n_pos2;
        BA.item0 = cls == 2 ? 0 : a_split, BA.item_end = cls == 2 ? a_split : asum;
        BA.counter = counters + (cls == 2 ? 2 : 3);
        if (BA.n_pos > 0 && BA.item_end > BA.item0 &&
            launch_adjoint_batch(BA, cls, n_sm * tu.adj_ctas_per_sm, st) != cudaSuccess)
            return FDX_ERR_CUDA;
    }
    for (int m = 0; m < n_models; ++m) {
        const fdx_problem *pr = probs[m];
        const fdx_atoms *a = atoms[m];
        if (launch_adjoint_post(adj[m], st) != cudaSuccess) return FDX_ERR_CUDA;
        if (pr->n_refl > 0 && (grads[m]->dfrac || grads[m]->dB)) {
            const BackLayout B = back_layout(pr, a->n_atoms, a->n_elem);
            char *reg = ws + L.back[m];
            SFParams sp;
            memset(&sp, 0, sizeof sp);
            sp.n_atoms = a->n_atoms, sp.n_elem = a->n_elem;
            sp.frac = a->frac, sp.B = a->B, sp.occ = a->occ, sp.ff = a->ff, sp.elem = a->elem;
            sp.atoms_q = reinterpret_cast<uint4 *>(reg + B.atoms_q);
            sp.atoms_w = reinterpret_cast<float2 *>(reg + B.atoms_w);
            if (launch_sf_pack(sp, st) != cudaSuccess) return FDX_ERR_CUDA;
            SFAdjParams q;
            memset(&q, 0, sizeof q);
            q.n_atoms = a->n_atoms, q.n_elem = a->n_elem, q.n_refl = pr->n_refl;
            q.n_split = B.sf_split, q.refl_per_split = B.refl_per_split;
            q.atoms_q = sp.atoms_q, q.atoms_w = sp.atoms_w;
            q.hkl = pr->hkl, q.cF = adj[m].cF, q.fe = adj[m].fe;
            q.partial = reinterpret_cast<double *>(reg + B.sf_partial);
            q.dfrac = grads[m]->dfrac, q.dB = grads[m]->dB;
            if (launch_sf_adjoint(q, st) != cudaSuccess) return FDX_ERR_CUDA;
        } else if (pr->n_refl == 0) {
            if (grads[m]->dfrac && cudaMemsetAsync(grads[m]->dfrac, 0, sizeof(double) * 3 * a->n_atoms, st)) return FDX_ERR_CUDA;
            if (grads[m]->dB && cudaMemsetAsync(grads[m]->dB, 0, sizeof(double) * a->n_atoms, st)) return FDX_ERR_CUDA;
        }
    }
    return FDX_OK;
}

int fdx_version(void) { return 100; }

int fdx_debug_probe(void *stream) {
#ifdef FDX_DEBUG
    debug_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>();
    return cudaGetLastError() == cudaSuccess ? 1 : FDX_ERR_CUDA;
#else
    (void)stream;
    return 0;
#endif
}

int fdx_debug_status(unsigned long long *flags, long long *last_index) {
#ifdef FDX_DEBUG
    unsigned long long w[2] = {0ull, 0ull};
    const unsigned long long z[2] = {0ull, 0ull};
    if (cudaMemcpyFromSymbol(w, fdx_debug_word, sizeof w) != cudaSuccess) return FDX_ERR_CUDA;
    if (cudaMemcpyToSymbol(fdx_debug_word, z, sizeof z) != cudaSuccess) return FDX_ERR_CUDA;
    if (flags) *flags = w[0];
    if (last_index) *last_index = (long long)w[1];
    return 1;
#else
    if (flags) *flags = 0ull;
    if (last_index) *last_index = -1;
    return 0;
#endif
}

int fdx_status(void *stream, int *device_status) {
    const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (device_status) *device_status = (int)e;
    return e == cudaSuccess ? FDX_OK : FDX_ERR_CUDA;
}

int fdx_set_tuning(const fdx_tuning *t) {
    fdx_tuning v = {2, 4, 3, 128, 1};
    if (t) {
        if (t->ppl_max < 1 || t->ppl_max > 2 || t->fwd_ctas_per_sm < 1 || t->fwd_ctas_per_sm > 8 ||
            t->adj_ctas_per_sm < 1 || t->adj_ctas_per_sm > 8 || t->adj_bands < 1 || t->adj_bands > 256 ||
            t->node_block < 0 || t->node_block > 3)
            return FDX_ERR_ARG;
        v = *t;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = v;
    return FDX_OK;
}

int fdx_get_tuning(fdx_tuning *t) {
    if (!t) return FDX_ERR_ARG;
    *t = tuning();
    return FDX_OK;
}

const char *fdx_error_string(int code) {
    switch (code) {
        case FDX_OK: return "ok";
        case FDX_ERR_ARG: return "invalid argument";
        case FDX_ERR_GEOMETRY: return "invalid geometry (cell, resolution, or fiber axis parallel to the beam)";
        case FDX_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
        case FDX_ERR_CUDA: return "CUDA runtime error";
        case FDX_ERR_CAPACITY: return "output capacity too small";
        default: return "unknown error";
    }
}

int fdx_reflections(const fdx_cell *cell, double d_min, double d_max, int32_t capacity, int32_t *hkl_out,
                    int32_t *n_out) {
    int rc = validate_cell(cell);
    if (rc) return rc;
    if (!n_out || capacity < 0 || (capacity > 0 && !hkl_out)) return FDX_ERR_ARG;
    if (!(d_min > 0) || !isfinite(d_min) || !isfinite(d_max)) return FDX_ERR_GEOMETRY;
    double A[9], As[9];
    cell_basis(*cell, A, As);
    // |h| <= |D| |a| <= |a| / d_min
    const int H = (int)ceil(cell->a / d_min), K = (int)ceil(cell->b / d_min), Lm = (int)ceil(cell->c / d_min);
    const double s2max = (1.0 + 1e-12) / (d_min * d_min);
    const double s2min = d_max > 0 ? (1.0 - 1e-12) / (d_max * d_max) : 0.0;
    std::vector<int32_t> out;
    for (int h = -H; h <= H; ++h)
        for (int k = -K; k <= K; ++k)
            for (int l = -Lm; l <= Lm; ++l) {
                if (!h && !k && !l) continue;
                double D[3];
                for (int q = 0; q < 3; ++q) D[q] = h * As[q] + k * As[3 + q] + l * As[6 + q];
                const double s2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
                if (s2 > s2max || s2 < s2min) continue;
                out.push_back(h), out.push_back(k), out.push_back(l);
            }
    const int32_t n = (int32_t)(out.size() / 3);
    *n_out = n;
    if (capacity == 0) return FDX_OK;
    if (capacity < n) return FDX_ERR_CAPACITY;
    if (n == 0) return FDX_OK;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, hkl_out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    if (attr.type == cudaMemoryTypeDevice) {
        if (cudaMemcpy(hkl_out, out.data(), out.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
            return FDX_ERR_CUDA;
    } else {
        memcpy(hkl_out, out.data(), out.size() * sizeof(int32_t));
    }
    return FDX_OK;
}

size_t fdx_sf_workspace_size(int32_t n_atoms, int32_t n_refl) {
    if (n_atoms < 1 || n_refl < 0) return 0;
    return sf_bind(nullptr, nullptr, n_atoms, n_refl, 64);  // at most 64 rows of partials
}

int fdx_structure_factors(const fdx_cell *cell, const fdx_atoms *atoms, const fdx_broadening *br, int32_t n_refl,
                          const int32_t *hkl, float *F_out, float *M_out, void *workspace, size_t ws_bytes,
                          void *stream) {
    int rc = validate_cell(cell);
    if (rc) return rc;
    if (!atoms || atoms->n_atoms < 1 || atoms->n_elem < 1 || atoms->n_elem > 64) return FDX_ERR_ARG;
    if (!atoms->frac || !atoms->B || !atoms->elem || !atoms->ff) return FDX_ERR_ARG;
    if (n_refl < 0) return FDX_ERR_ARG;
    if (n_refl > 0 && (!hkl || !F_out)) return FDX_ERR_ARG;
    if (br && (rc = validate_broadening(br))) return rc;
    if (n_refl == 0) return FDX_OK;
    const size_t need = fdx_sf_workspace_size(atoms->n_atoms, n_refl);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign)) return FDX_ERR_WORKSPACE;

    SFParams p;
    memset(&p, 0, sizeof p);
    double A[9], As[9];
    cell_basis(*cell, A, As);
    memcpy(p.As, As, sizeof As);
    p.n_atoms = atoms->n_atoms, p.n_elem = atoms->n_elem, p.n_refl = n_refl;
    int n_split = 1, per = 1;
    sf_plan(atoms->n_atoms, n_refl, atoms->n_elem, 64, n_split, per);
    p.n_split = n_split;
    p.frac = atoms->frac, p.B = atoms->B, p.occ = atoms->occ, p.ff = atoms->ff, p.elem = atoms->elem;
    sf_bind(&p, static_cast<char *>(workspace), atoms->n_atoms, n_refl, 64);
    p.hkl = hkl, p.F_out = F_out, p.M_out = M_out;
    p.has_br = br ? 1 : 0;
    if (br) {
        p.intensity_model = br->intensity_model;
        for (int i = 0; i < 3; ++i) {
            p.g[i] = br->g[i], p.Bax[i] = br->B_axis[i];
            p.alen[i] = sqrt(A[3 * i] * A[3 * i] + A[3 * i + 1] * A[3 * i + 1] + A[3 * i + 2] * A[3 * i + 2]);
        }
    }
    if (launch_structure_factors(p, static_cast<cudaStream_t>(stream)) != cudaSuccess) return FDX_ERR_CUDA;
    return FDX_OK;
}

size_t fdx_workspace_size(int32_t n_models, const fdx_problem *const *probs) {
    if (n_models < 1 || !probs) return 0;
    size_t best = 0;
    for (int m = 0; m < n_models; ++m) {
        if (!probs[m]) return 0;
        const size_t t = layout_for(probs[m]).total;
        best = t > best ? t : best;
    }
    return best;
}

int fdx_pattern(int32_t n_models, const fdx_problem *const *probs, float *const *images, void *workspace,
                size_t ws_bytes, void *stream) {
    if (n_models < 1 || !probs || !images) return FDX_ERR_ARG;
    for (int m = 0; m < n_models; ++m) {
        int rc = validate_problem(probs[m]);
        if (rc) return rc;
        if (!images[m]) return FDX_ERR_ARG;
    }
    const size_t need = fdx_workspace_size(n_models, probs);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign)) return FDX_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int m = 0; m < n_models; ++m) {
        int rc = run_pattern(probs[m], images[m], nullptr, static_cast<char *>(workspace), st);
        if (rc) return rc;
    }
    return FDX_OK;
}

size_t fdx_backward_workspace_size(const fdx_problem *prob, int32_t n_atoms, int32_t n_elem) {
    if (!prob || n_atoms < 1 || n_elem < 1) return 0;
    return back_layout(prob, n_atoms, n_elem).total;
}

int fdx_pattern_backward(const fdx_problem *prob, const fdx_atoms *atoms, const float *F, const float *dL_dI,
                         const fdx_grads *grads, void *workspace, size_t ws_bytes, void *stream) {
    int rc = validate_problem(prob);
    if (rc) return rc;
    if (!atoms || atoms->n_atoms < 1 || atoms->n_elem < 1 || atoms->n_elem > 64) return FDX_ERR_ARG;
    if (!atoms->frac || !atoms->B || !atoms->elem || !atoms->ff) return FDX_ERR_ARG;
    if (!dL_dI || !grads || (prob->n_refl > 0 && !F)) return FDX_ERR_ARG;
    const BackLayout B = back_layout(prob, atoms->n_atoms, atoms->n_elem);
    if (!workspace || ws_bytes < B.total || ((uintptr_t)workspace % kAlign)) return FDX_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    if (prob->n_refl == 0) {
        if (grads->dfrac && cudaMemsetAsync(grads->dfrac, 0, sizeof(double) * 3 * atoms->n_atoms, st)) return FDX_ERR_CUDA;
        if (grads->dB && cudaMemsetAsync(grads->dB, 0, sizeof(double) * atoms->n_atoms, st)) return FDX_ERR_CUDA;
        if (grads->dglobal && cudaMemsetAsync(grads->dglobal, 0, sizeof(double) * 8, st)) return FDX_ERR_CUDA;
        return FDX_OK;
    }
    AdjParams A;
    memset(&A, 0, sizeof A);
    rc = setup_pattern(prob, ws, st, A.P, true);
    if (rc) return rc;
    double Am[9], As[9];
    cell_basis(prob->cell, Am, As);
    memcpy(A.As, As, sizeof As);
    for (int i = 0; i < 3; ++i) {
        A.alen[i] = sqrt(Am[3 * i] * Am[3 * i] + Am[3 * i + 1] * Am[3 * i + 1] + Am[3 * i + 2] * Am[3 * i + 2]);
        A.L[i] = prob->br.L[i], A.g[i] = prob->br.g[i], A.Bax[i] = prob->br.B_axis[i];
    }
    A.patch_bounds = reinterpret_cast<float4 *>(ws + B.patch_bounds);
    A.band_bounds = reinterpret_cast<float4 *>(ws + B.band_bounds);
    A.npx = B.npx, A.npy = B.npy, A.n_bands = B.n_bands, A.rows_per_band = B.rows_per_band;
    A.gI = dL_dI;
    A.item_out = reinterpret_cast<double *>(ws + B.item_out);
    A.refl_out = reinterpret_cast<double *>(ws + B.refl_out);
    A.cF = reinterpret_cast<float4 *>(ws + B.cF);
    A.fe = reinterpret_cast<float *>(ws + B.fe);
    A.dM = grads->dM;
    A.dglobal = grads->dglobal;
    A.hkl = prob->hkl;
    A.F = F;
    A.ff = atoms->ff;
    A.n_elem = atoms->n_elem;
    A.intensity_model = prob->br.intensity_model;
    A.lineshape = prob->br.lineshape;
    A.counter = reinterpret_cast<unsigned *>(ws + B.counter);
    int dev = 0, n_sm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDX_ERR_CUDA;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (launch_adjoint(A, n_sm * tuning().adj_ctas_per_sm, st) != cudaSuccess) return FDX_ERR_CUDA;

    if (grads->dfrac || grads->dB) {
        SFParams sp;
        memset(&sp, 0, sizeof sp);
        sp.n_atoms = atoms->n_atoms, sp.n_elem = atoms->n_elem;
        sp.frac = atoms->frac, sp.B = atoms->B, sp.occ = atoms->occ, sp.ff = atoms->ff, sp.elem = atoms->elem;
        sp.atoms_q = reinterpret_cast<uint4 *>(ws + B.atoms_q);
        sp.atoms_w = reinterpret_cast<float2 *>(ws + B.atoms_w);
        if (launch_sf_pack(sp, st) != cudaSuccess) return FDX_ERR_CUDA;
        SFAdjParams q;
        memset(&q, 0, sizeof q);
        q.n_atoms = atoms->n_atoms, q.n_elem = atoms->n_elem, q.n_refl = prob->n_refl;
        q.n_split = B.sf_split, q.refl_per_split = B.refl_per_split;
        q.atoms_q = sp.atoms_q, q.atoms_w = sp.atoms_w;
        q.hkl = prob->hkl, q.cF = A.cF, q.fe = A.fe;
        q.partial = reinterpret_cast<double *>(ws + B.sf_partial);
        q.dfrac = grads->dfrac, q.dB = grads->dB;
        if (launch_sf_adjoint(q, st) != cudaSuccess) return FDX_ERR_CUDA;
    }
    return FDX_OK;
}

// Plain FP64 path: the FP32 path's backward layout followed by FP64 buffers.
struct Plain64Layout {
    BackLayout B;
    size_t recs64, nodes64, F64, M64, Gw64, gI, loss_partial, total;
};

Plain64Layout plain64_layout(const fdx_problem *p, int n_atoms, int n_elem) {
    Plain64Layout L;
    L.B = back_layout(p, n_atoms, n_elem);
    const size_t nr = (size_t)(p->n_refl > 0 ? p->n_refl : 1);
    const size_t npx = (size_t)p->geom.n_x * p->geom.n_y;
    size_t off = L.B.total;
    L.recs64 = off, off += align_up(sizeof(double) * 48 * nr);
    L.nodes64 = off, off += align_up(sizeof(double) * 4 * (size_t)p->br.n_nodes * p->br.n_nodes);
    L.F64 = off, off += align_up(sizeof(double) * 2 * nr);
    L.M64 = off, off += align_up(sizeof(double) * nr);
    L.Gw64 = off, off += align_up(sizeof(double) * nr);
    L.gI = off, off += align_up(sizeof(double) * npx);
    L.loss_partial = off, off += align_up(sizeof(double) * ((npx + 255) / 256));
    L.total = off;
    return L;
}

size_t fdx_plain64_workspace_size(const fdx_problem *prob, int32_t n_atoms, int32_t n_elem) {
    if (!prob || n_atoms < 1 || n_elem < 1) return 0;
    return plain64_layout(prob, n_atoms, n_elem).total;
}

int fdx_plain64_refine(const fdx_problem *prob, const fdx_atoms *atoms, const double *I_target, const float *mask,
                       double *image, double *loss, const fdx_grads *grads, void *workspace, size_t ws_bytes,
                       void *stream) {
    if (!prob || !image) return FDX_ERR_ARG;
    fdx_problem pr = *prob;
    pr.M = nullptr;  // the FP64 path forms its own M
    int rc = validate_cell(&pr.cell);
    if (rc) return rc;
    if ((rc = validate_broadening(&pr.br)) || (rc = validate_geometry(&pr.geom))) return rc;
    if (pr.n_refl < 0 || (pr.n_refl > 0 && !pr.hkl)) return FDX_ERR_ARG;
    if (pr.br.lineshape != FDX_LINESHAPE_HOSEMANN) return FDX_ERR_ARG;
    if (!atoms || atoms->n_atoms < 1 || atoms->n_elem < 1 || atoms->n_elem > 64) return FDX_ERR_ARG;
    if (!atoms->frac || !atoms->B || !atoms->elem || !atoms->ff) return FDX_ERR_ARG;
    if (I_target && (!loss || !grads)) return FDX_ERR_ARG;
    const Plain64Layout L = plain64_layout(&pr, atoms->n_atoms, atoms->n_elem);
    if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace % kAlign)) return FDX_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    double *nodes64 = reinterpret_cast<double *>(ws + L.nodes64);
    PatternParams P;
    if ((rc = setup_pattern(&pr, ws, st, P, false, nodes64))) return rc;

    Plain64Params q;
    memset(&q, 0, sizeof q);
    q.nx = pr.geom.n_x, q.ny = pr.geom.n_y, q.n_refl = pr.n_refl, q.n = pr.br.n_nodes;
    q.n_atoms = atoms->n_atoms, q.n_elem = atoms->n_elem;
    q.npx = L.B.npx, q.npy = L.B.npy, q.n_bands = L.B.n_bands, q.rows_per_band = L.B.rows_per_band;
    q.intensity_model = pr.br.intensity_model;
    q.T = pr.br.T, q.h = 2.0 * pr.br.T / pr.br.n_nodes, q.delta_L = pr.geom.delta_L;
    double Am[9], As[9];
    cell_basis(pr.cell, Am, As);
    memcpy(q.A, Am, sizeof Am);
    memcpy(q.As, As, sizeof As);
    double bh[3];
    unit3(pr.geom.fiber_axis, q.nh);
    unit3(pr.geom.beam_axis, bh);
    for (int i = 0; i < 3; ++i) {
        q.bh[i] = bh[i];
        q.alen[i] = sqrt(Am[3 * i] * Am[3 * i] + Am[3 * i + 1] * Am[3 * i + 1] + Am[3 * i + 2] * Am[3 * i + 2]);
        q.L[i] = pr.br.L[i], q.g[i] = pr.br.g[i], q.Bax[i] = pr.br.B_axis[i];
    }
    q.pixgeo = P.pixgeo, q.reach = P.reach;
    q.patch_bounds = reinterpret_cast<float4 *>(ws + L.B.patch_bounds);
    q.band_bounds = reinterpret_cast<float4 *>(ws + L.B.band_bounds);
    q.recs64 = reinterpret_cast<double *>(ws + L.recs64);
    q.nodes64 = nodes64;
    q.image64 = image;
    q.It64 = I_target;
    q.mask = mask;
    q.gI = reinterpret_cast<double *>(ws + L.gI);
    q.loss = loss;
    q.loss_partial = reinterpret_cast<double *>(ws + L.loss_partial);
    q.hkl = pr.hkl;
    q.F64 = reinterpret_cast<double *>(ws + L.F64);
    q.M64 = reinterpret_cast<double *>(ws + L.M64);
    q.Gw64 = reinterpret_cast<double *>(ws + L.Gw64);
    q.item_out = reinterpret_cast<double *>(ws + L.B.item_out);
    q.refl_out = reinterpret_cast<double *>(ws + L.B.refl_out);
    q.frac = atoms->frac, q.B = atoms->B, q.occ = atoms->occ, q.ff = atoms->ff, q.elem = atoms->elem;
    q.dfrac = grads ? grads->dfrac : nullptr;
    q.dB = grads ? grads->dB : nullptr;
    if (launch_plain64_forward(q, st) != cudaSuccess) return FDX_ERR_CUDA;
    if (!I_target) return FDX_OK;
    if (launch_plain64_loss(q, st) != cudaSuccess) return FDX_ERR_CUDA;
    AdjParams A;
    memset(&A, 0, sizeof A);
    A.P = P;
    A.patch_bounds = const_cast<float4 *>(q.patch_bounds);
    A.band_bounds = const_cast<float4 *>(q.band_bounds);
    A.npx = q.npx, A.npy = q.npy, A.n_bands = q.n_bands, A.rows_per_band = q.rows_per_band;
    A.refl_out = q.refl_out;
    A.dglobal = grads->dglobal;
    if (launch_plain64_backward(q, A, st) != cudaSuccess) return FDX_ERR_CUDA;
    return FDX_OK;
}

size_t fdx_loss_workspace_size(int64_t n_px) {
    if (n_px < 1) return 0;
    return align_up(sizeof(double) * (size_t)((n_px + 255) / 256));
}

int fdx_loss(int64_t n_px, const float *I, const float *I_target, const float *mask, double *loss_out, float *dL_dI,
             void *workspace, size_t ws_bytes, void *stream) {
    if (n_px < 1 || !I || !I_target || !loss_out) return FDX_ERR_ARG;
    if (!workspace || ws_bytes < fdx_loss_workspace_size(n_px) || ((uintptr_t)workspace % kAlign))
        return FDX_ERR_WORKSPACE;
    LossParams lp;
    lp.n = n_px, lp.I = I, lp.It = I_target, lp.mask = mask, lp.gI = dL_dI;
    lp.partial = static_cast<double *>(workspace);
    lp.loss = loss_out;
    if (launch_loss(lp, static_cast<cudaStream_t>(stream)) != cudaSuccess) return FDX_ERR_CUDA;
    return FDX_OK;
}

size_t fdx_ring_workspace_size(const fdx_problem *prob) {
    if (!prob) return 0;
    size_t roff = 0;
    return ring_layout(prob, &roff);
}

int fdx_ring(const fdx_problem *prob, float *image, void *workspace, size_t ws_bytes, void *stream) {
    if (!image) return FDX_ERR_ARG;
    return run_ring(prob, image, nullptr, workspace, ws_bytes, stream);
}

int fdx_ring_evals(const fdx_problem *prob, int32_t *counts, void *workspace, size_t ws_bytes, void *stream) {
    if (!counts) return FDX_ERR_ARG;
    return run_ring(prob, nullptr, counts, workspace, ws_bytes, stream);
}

size_t fdx_scatter_workspace_size(const fdx_problem *prob, int32_t n_samples) {
    if (!prob || n_samples < 1) return 0;
    return scatter_layout(prob, n_samples).total;
}

int fdx_scatter(const fdx_problem *prob, int32_t n_samples, const float *samples, int32_t spot_size, float *image,
                void *workspace, size_t ws_bytes, void *stream) {
    if (!image) return FDX_ERR_ARG;
    return run_scatter(prob, n_samples, samples, spot_size, image, nullptr, workspace, ws_bytes, stream);
}

int fdx_scatter_evals(const fdx_problem *prob, int32_t n_samples, const float *samples, int64_t *count,
                      void *workspace, size_t ws_bytes, void *stream) {
    if (!count || ((uintptr_t)count % 8)) return FDX_ERR_ARG;
    return run_scatter(prob, n_samples, samples, 1, nullptr, count, workspace, ws_bytes, stream);
}

int fdx_pattern_evals(const fdx_problem *prob, int32_t *counts, void *workspace, size_t ws_bytes, void *stream) {
    int rc = validate_problem(prob);
    if (rc) return rc;
    if (!counts) return FDX_ERR_ARG;
    const fdx_problem *pp[1] = {prob};
    const size_t need = fdx_workspace_size(1, pp);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace % kAlign)) return FDX_ERR_WORKSPACE;
    return run_pattern(prob, nullptr, counts, static_cast<char *>(workspace), static_cast<cudaStream_t>(stream));
}

}  // extern "C"
