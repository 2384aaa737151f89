/*
 * fdx.h -- C-ABI of libfdx, the B300 (sm_103a) fiber-diffraction hot path.
 *
 * The library computes, on one GPU:
 *   1. the reflection list of a cell (Sect. "Structure factors and reflection
 *      list": every (h,k,l) != 0 with d_min <= d <= d_max);
 *   2. structure factors by direct summation over atoms (Eq. structure_factor,
 *      with the atomic form factor f(s) = sum_i a_i exp(-b_i s^2/4) + c and the
 *      isotropic Debye-Waller factor exp(-B s^2/4), B = 8 pi^2 <u^2>, Sect.
 *      "Paracrystalline disorder"), and per reflection M = |F|^2 P DW_axis with
 *      the Hosemann intensity factor P of Eq. Ipara and the axis damping
 *      D(S) = exp(-1/4 sum_i B_i (S . a^_i)^2);
 *   3. the detector image: per pixel, the shell-quadrature sum of Eq.
 *      direct_sum over the gnomonic nodes of Eq. gnomonic with the weights of
 *      Eq. node_weight (Gaussian, Lorentzian or Voigt angular shape, Sect.
 *      "Angular peak shapes"), the lattice factor of Eq. I_shape (sinc^2 with
 *      N_eff of Eq. Neff) or of Eq. Z (Hosemann), evaluated at the pixel's
 *      query point on the Ewald sphere, times the Lorentz factor of Eq.
 *      lorentz.
 *
 * Conventions
 *   - Units: lengths in Angstrom, reciprocal lengths in 1/Angstrom, angles in
 *     radians; detector distance and pixel size in one common unit (mm).
 *   - Cell frame (Sect. "Unit cell and reciprocal-space frame"): c along z,
 *     b in the yz-plane; fiber and beam axes are given in that frame.
 *   - Detector: pixel (i, j) has centre u = (i + 1/2 - n_x/2) p along
 *     u^ = normalize(n x b), v = (j + 1/2 - n_y/2) p along v^ = b x u^;
 *     image[j][i], row j along +v.  Tilt 0, beam centre at the detector centre.
 *   - Ownership: every array is owned by the caller.  Device arrays must stay
 *     valid until the work queued on `stream` has finished.  The library never
 *     allocates device memory: scratch comes from the caller's `workspace`.
 *     Host structs are read during the call only.
 *   - Errors: every entry point validates its arguments on the host before it
 *     queues any work and returns one of the FDX_* codes below; no C++
 *     exception crosses the ABI.  After validation the calls are asynchronous
 *     on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 *     stream), except fdx_reflections, which is synchronous.
 *   - Determinism: no result is accumulated with atomics; two calls with the
 *     same inputs produce bitwise identical outputs.
 */
#ifndef FDX_H
#define FDX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define FDX_OK 0
#define FDX_ERR_ARG (-1)       /* null pointer, non-positive size, NaN, bad enum */
#define FDX_ERR_GEOMETRY (-2)  /* fiber axis (nearly) parallel to the beam, d_min <= 0, bad cell */
#define FDX_ERR_WORKSPACE (-3) /* workspace too small or misaligned (256-byte alignment) */
#define FDX_ERR_CUDA (-4)      /* a CUDA runtime call or kernel launch failed */
#define FDX_ERR_CAPACITY (-5)  /* output capacity too small */

#define FDX_LINESHAPE_SINC 0     /* K = N sinc^2(N t), N = 1/beta, |t| <= min(K_z/N, 1/2) (Eq. I_shape) */
#define FDX_LINESHAPE_HOSEMANN 1 /* K = beta/(beta^2 + (1-beta^2) sin^2(pi t)), |t| <= 1/2 (Eq. Z) */
#define FDX_LINESHAPE_GAUSS 2    /* K = exp(-pi t^2/beta^2)/beta, |t| <= min(K_z beta, 1/2): the Gaussian of
                                    the same integral breadth as Eq. Z (Eq. breadth); forward only */
#define FDX_INTENSITY_NONE 0     /* P = 1 */
#define FDX_INTENSITY_HOSEMANN 1 /* P = prod_i 2A_i/(1 + A_i^2), A_i = exp(-2 pi^2 g_i^2 h_i^2) (Eq. Ipara) */

/* Unit cell: a, b, c in Angstrom; alpha, beta, gamma in radians. */
typedef struct fdx_cell {
    double a, b, c;
    double alpha, beta, gamma;
} fdx_cell;

/* Atoms of one model.  All pointers are device pointers. */
typedef struct fdx_atoms {
    int32_t n_atoms;      /* >= 1 */
    int32_t n_elem;       /* 1..64 element types */
    const double *frac;   /* [n_atoms][3] fractional coordinates (any real value) */
    const float *B;       /* [n_atoms] isotropic B (A^2) */
    const float *occ;     /* [n_atoms] occupancy, or NULL for 1 (the paper sets 1) */
    const uint8_t *elem;  /* [n_atoms] element index < n_elem (an index >= n_elem makes F NaN) */
    const float *ff;      /* [n_elem][9] form factor a1..a4, b1..b4, c: f(s) = sum a_i exp(-b_i s^2/4) + c */
} fdx_atoms;

/* Disorder and quadrature parameters (ParacrystalSpec and simulate(), Sect.
 * "Paracrystalline disorder and the simulation loop"). */
typedef struct fdx_broadening {
    double L[3];            /* crystallite size along a, b, c (A); N_base,i = L_i/|a_i| */
    double g[3];            /* Hosemann g along a, b, c (>= 0) */
    double B_axis[3];       /* axis damping B_a, B_b, B_c (A^2) */
    int32_t lineshape;      /* FDX_LINESHAPE_* */
    int32_t intensity_model;/* FDX_INTENSITY_* */
    double sigma;           /* Gaussian orientation width (rad); gamma == 0 selects the Gaussian */
    double gamma;           /* Lorentzian HWHM (rad); sigma < 1e-12 selects the Lorentzian */
    double sigma_r;         /* radial shell width (1/A); enters as sigma_r sqrt(2 pi) */
    double T;               /* patch half-extent in tangent units, > 0 */
    int32_t n_nodes;        /* nodes per axis of the midpoint grid, 1..512 */
    int32_t reserved;
    double K_z;             /* sinc support in zeros (> 0) */
} fdx_broadening;

/* Experiment geometry (params_experiment, Sect. "Experimental geometry"). */
typedef struct fdx_geometry {
    double wavelength;      /* A */
    double distance;        /* sample-detector distance */
    double pixel;           /* pixel size, same unit as distance */
    int32_t n_x, n_y;       /* detector size in pixels, 1..16384 each */
    double fiber_axis[3];   /* fiber (rotation) axis, need not be unit; tilted towards the beam by the
                               fiber tilt (Sect. Experimental geometry: tilt), not parallel to it */
    double beam_axis[3];    /* incident beam direction, need not be unit */
    double delta_L;         /* Lorentz regulariser delta of Eq. lorentz (1/A), > 0 */
} fdx_geometry;

/* One pattern problem. */
typedef struct fdx_problem {
    fdx_cell cell;
    fdx_broadening br;
    fdx_geometry geom;
    int32_t n_refl;         /* >= 0 */
    int32_t reserved;
    const int32_t *hkl;     /* [n_refl][3] device */
    const float *M;         /* [n_refl] device: M = |F|^2 P DW_axis */
} fdx_problem;

/*
 * fdx_reflections -- reflection list (Sect. "Structure factors and reflection
 * list").  Every (h,k,l) != (0,0,0) with d_min <= d <= d_max (d = 1/|D|,
 * D = h a* + k b* + l c*, Eq. recip_basis), Friedel mates included, in
 * lexicographic (h, k, l) order.  A reflection on the boundary within a
 * relative 1e-12 of 1/d^2 is kept.  d_max <= 0 means no upper cut.
 * Count/fill protocol: with capacity == 0 (hkl_out may be NULL) only *n_out
 * is written.  hkl_out ([capacity][3]) may be host or device memory.
 * Returns FDX_ERR_CAPACITY (and the needed count in *n_out) when capacity is
 * too small.  Synchronous.
 */
int fdx_reflections(const fdx_cell *cell, double d_min, double d_max, int32_t capacity, int32_t *hkl_out,
                    int32_t *n_out);

/* Bytes of workspace fdx_structure_factors needs for this size. */
size_t fdx_sf_workspace_size(int32_t n_atoms, int32_t n_refl);

/*
 * fdx_structure_factors -- Eq. structure_factor by direct summation:
 *   F_hkl = sum_j occ_j f_{e_j}(s) exp(-B_j s^2/4) exp(2 pi i (h x_j + k y_j + l z_j)),
 *   s = |D_hkl| = 1/d.
 * F_out ([n_refl][2] device, re/im) and, when M_out is not NULL,
 * M_out[r] = |F_r|^2 P_r DW_r (P and DW from `br`, which may be NULL for
 * P = DW = 1).  FP32 arithmetic with exact 32-bit fixed-point phase
 * reduction and compensated sums.  Asynchronous on `stream`.
 */
int fdx_structure_factors(const fdx_cell *cell, const fdx_atoms *atoms, const fdx_broadening *br, int32_t n_refl,
                          const int32_t *hkl, float *F_out, float *M_out, void *workspace, size_t ws_bytes,
                          void *stream);

/*
 * fdx_structure_factors_noalloc -- the same computation as
 * fdx_structure_factors, for callers that cannot allocate device memory at
 * call time (for example a plugin inside a host application whose caching
 * allocator owns all device memory, or a real-time loop that must not call
 * cudaMalloc after start-up because it can synchronise the device).  The paper
 * has no counterpart: this is a deployment convenience of the library.
 *   - No workspace argument: the kernels' scratch is a fixed array of
 *     FDX_NOALLOC_SF_SCRATCH_BYTES (8 MiB) in device memory that every GPU
 *     loading libfdx holds until the process exits.  Each piece of the layout
 *     is rounded up to 256 bytes; it must fit 24.25 bytes per atom (plus
 *     96 KiB of padding: the kernels keep the atoms sorted by element),
 *     4 bytes per reflection, and 16 bytes per reflection for every row of
 *     partial sums.  Each element pass writes its own rows (one pass for up to
 *     40 element types, two for 41-64), so at least `passes` rows must fit;
 *     the call uses as many rows as fit, at most 64.  Larger sizes return
 *     FDX_ERR_WORKSPACE before any work is queued.  The call allocates
 *     nothing.
 *   - The first call on a device looks up the array's address on that device
 *     and caches it; make that first call before any stream capture.
 *   - All calls share the array.  Calls whose work overlaps on the GPU race on
 *     it: serialise them (one stream, or events between streams).  Nothing in
 *     it needs to start at zero.
 * Inputs, outputs, argument checks and return codes as
 * fdx_structure_factors.  Asynchronous.
 */
#define FDX_NOALLOC_SF_SCRATCH_BYTES (8u << 20)
int fdx_structure_factors_noalloc(const fdx_cell *cell, const fdx_atoms *atoms, const fdx_broadening *br,
                                  int32_t n_refl, const int32_t *hkl, float *F_out, float *M_out, void *stream);

/* Bytes of workspace fdx_pattern / fdx_pattern_evals need for these problems. */
size_t fdx_workspace_size(int32_t n_models, const fdx_problem *const *probs);

/*
 * fdx_pattern -- detector images.  For every pixel (R, Z from the Ewald
 * construction, Eq. laue) and every reflection, the query point is the
 * pixel's ring point in the reflection's meridional half-plane,
 * p = Z n + R e_R(D), and
 *   I_pix = L(R) sum_hkl M_hkl r0^2 sum_{k: |t_i| <= t_max,i} w_k prod_i K_i(t_i),
 *   t_i = a_i . (p - s_k),  L(R) = delta_L / (R + delta_L),
 * with s_k the gnomonic shell nodes (Eq. gnomonic) and w_k their weights
 * (Eq. node_weight).  images[m] is [n_y][n_x] float (device).  Models are
 * processed one after another on `stream`.  Asynchronous.
 */
int fdx_pattern(int32_t n_models, const fdx_problem *const *probs, float *const *images, void *workspace,
                size_t ws_bytes, void *stream);

/*
 * fdx_pattern_evals -- the number of (reflection, node) terms inside the
 * support for each pixel of one problem (the unit of the throughput metric),
 * written to counts ([n_y][n_x] int32, device).  Asynchronous.
 */
int fdx_pattern_evals(const fdx_problem *prob, int32_t *counts, void *workspace, size_t ws_bytes, void *stream);

/* Cap on the azimuth points per reflection of the ring average. */
#define FDX_RING_MAX_N 1024

/* Bytes of workspace fdx_ring / fdx_ring_evals need. */
size_t fdx_ring_workspace_size(const fdx_problem *prob);

/*
 * fdx_ring -- the ring-integrated cylindrical average (Eq. cyl-average), the
 * other projection the paper describes: every pixel's value is the average of
 * the reciprocal-space intensity over the ring of its (R, Z) about the fiber
 * axis, with no Lorentz factor,
 *   I_pix = sum_hkl M r0^2 (1/2pi) int dphi sum_k w_k prod_i K_i(a_i . (p(phi) - s_k)),
 *   p(phi) = Z n + R (cos(phi) e_R + sin(phi) e_P),  e_P = n x e_R(D),
 * by the midpoint rule in phi over [-Phi_r, Phi_r] with N_r points per
 * reflection: Phi_r is the half-width outside which the ring stays farther
 * than rho_tot = rho_B + sqrt(2) r0 T from D, N_r = clamp(ceil(2 Phi_r /
 * dphi), 4, FDX_RING_MAX_N) with dphi = w_min / (4 (R_D + rho_tot)) and
 * w_min = min_i beta_i / |a_i|.  image is [n_y][n_x] float (device).  Every
 * lineshape.  Asynchronous.  The cost is about N_r times that of fdx_pattern.
 */
int fdx_ring(const fdx_problem *prob, float *image, void *workspace, size_t ws_bytes, void *stream);

/* fdx_ring_evals -- per-pixel in-support (reflection, azimuth point, node)
 * term counts of fdx_ring, [n_y][n_x] int32 (device). */
int fdx_ring_evals(const fdx_problem *prob, int32_t *counts, void *workspace, size_t ws_bytes, void *stream);

/* Bytes of workspace fdx_scatter / fdx_scatter_evals need. */
size_t fdx_scatter_workspace_size(const fdx_problem *prob, int32_t n_samples);

/*
 * fdx_scatter -- the scatter form of the projection, the paper's own pipeline
 * (Sects. "Numerical evaluation: per-reflection shell quadrature", "Lorentz
 * correction on a sampled reciprocal lattice", "Analytical Solution of the
 * Ewald Diffraction Condition").  samples is [n_samples][4] float (device,
 * 16-byte aligned): normalised (x_r, x_1, x_2) in [-1, 1]^3 and a quadrature
 * weight q, shared by all reflections.  For each reflection (radius r0,
 * support circumradius h_r) and sample:
 *   S  = (r0 + x_r h_r) c (S^ + d1 e1 + d2 e2),  d_i = x_i T,  c = (1 + d^2)^(-1/2)  (Eq. gnomonic)
 *   dV = q h_r T^2 (r0 + x_r h_r)^2 c^3,
 *   I  = M r0^2 sum_{k: |t_i| <= t_max,i} w_k prod_i K_i(a_i . (S - s_k))           (Eq. direct_sum)
 *   L  = delta_L / (R + delta_L),  R = |S - (S . n) n|                              (Eq. lorentz)
 * S is rotated about the fiber axis into the diffraction condition (Eqs.
 * harmonic, solutions; no contribution when Eq. valid fails); each of the two
 * hits with k_out . b > 0 is rendered as a detector spot (the paper's
 * simulate() parameter of that name): the spot_size x spot_size block of
 * pixels centred on the pixel the hit falls in each receive dV L I /
 * spot_size^2, the parts off the detector being lost (spot_size odd, 1..15;
 * 1 = the pixel itself; FDX_ERR_ARG otherwise).  The samples may reach past
 * [-1, 1] (heavy-tailed sampling of the angular coordinates: S and dV are the
 * same formulae for any x).  image is [n_y][n_x] float (device), overwritten.
 * Every lineshape.  Accumulation is in FP64 (atomics): the result does not
 * depend on the order at FP32 resolution.  Asynchronous.
 */
int fdx_scatter(const fdx_problem *prob, int32_t n_samples, const float *samples, int32_t spot_size, float *image,
                void *workspace, size_t ws_bytes, void *stream);

/* fdx_scatter_evals -- the number of in-support (sample, node) terms of the
 * scatter form over all reflections, written to *count (int64, device). */
int fdx_scatter_evals(const fdx_problem *prob, int32_t n_samples, const float *samples, int64_t *count,
                      void *workspace, size_t ws_bytes, void *stream);

/* Gradients written by fdx_pattern_backward; every pointer is a device pointer
 * or NULL (not written). */
typedef struct fdx_grads {
    double *dfrac;    /* [n_atoms][3] dLoss/d(fractional coordinates) */
    double *dB;       /* [n_atoms] dLoss/dB */
    double *dglobal;  /* [8] dLoss/d(L_a, L_b, L_c, g_a, g_b, g_c, sigma, gamma) */
    float *dM;        /* [n_refl] dLoss/dM */
} fdx_grads;

/* Bytes of workspace fdx_pattern_backward needs. */
size_t fdx_backward_workspace_size(const fdx_problem *prob, int32_t n_atoms, int32_t n_elem);

/*
 * fdx_pattern_backward -- hand-written adjoint of fdx_structure_factors +
 * fdx_pattern for an upstream gradient dL_dI ([n_y][n_x] float, device).
 * Recomputes the profiles (nothing is stored by the forward); takes the
 * forward's F ([n_refl][2], device) and the problem's M.  Writes the
 * gradients requested in `grads` with respect to the fractional coordinates,
 * isotropic B, crystallite sizes L_i, Hosemann g_i, sigma and gamma (T held
 * fixed; the pure-Gaussian branch reports 0 for gamma).  Every lineshape:
 * for the sinc (Eq. I_shape) and Gaussian ones the sums carry dK_i/dbeta_i at
 * fixed t (the sinc support's moving edge adds nothing: K and dK/dt vanish
 * there; the Gaussian's truncated tail is below 1e-12 of its peak).
 * Deterministic (no atomics).  Asynchronous.
 */
int fdx_pattern_backward(const fdx_problem *prob, const fdx_atoms *atoms, const float *F, const float *dL_dI,
                         const fdx_grads *grads, void *workspace, size_t ws_bytes, void *stream);

/* Bytes of workspace fdx_loss needs for n_px pixels. */
size_t fdx_loss_workspace_size(int64_t n_px);

/*
 * fdx_loss -- refinement loss L = sum_px m_px (I - I_t)^2 / (I_t + 1) (mask m
 * optional, NULL = 1) into *loss_out (device double) and, when dL_dI is not
 * NULL, dL/dI = 2 m (I - I_t)/(I_t + 1) (device float).  FP64 reduction in a
 * fixed order.  Asynchronous.
 */
int fdx_loss(int64_t n_px, const float *I, const float *I_target, const float *mask, double *loss_out,
             float *dL_dI, void *workspace, size_t ws_bytes, void *stream);

/* Bytes of workspace fdx_plain64_refine needs. */
size_t fdx_plain64_workspace_size(const fdx_problem *prob, int32_t n_atoms, int32_t n_elem);

/*
 * fdx_plain64_refine -- the same method in plain FP64 on the GPU (the
 * comparison form of the refinement-throughput metric): FP64 structure
 * factors, FP64 pattern (every term of each pixel's node range evaluated
 * directly with sinpi), and, when I_target is not NULL, the FP64 loss of
 * fdx_loss (mask optional) into *loss and the FP64 adjoint into `grads`
 * (dfrac, dB, dglobal; dM is not written).  image and I_target are
 * [n_y][n_x] double (device).  prob->M is ignored.  Hosemann lineshape only.
 * Asynchronous.
 */
int fdx_plain64_refine(const fdx_problem *prob, const fdx_atoms *atoms, const double *I_target, const float *mask,
                       double *image, double *loss, const fdx_grads *grads, void *workspace, size_t ws_bytes,
                       void *stream);

/* Bytes of workspace fdx_batch_refine needs for these models. */
size_t fdx_batch_workspace_size(int32_t n_models, const fdx_problem *const *probs, const fdx_atoms *const *atoms);

/*
 * fdx_batch_refine -- one refinement step for many models at once (batched
 * refinement of candidate models): per model the structure factors (into
 * F[m], M[m]; probs[m]->M is ignored), the pattern (images[m]), and, when
 * targets is not NULL, the loss of fdx_loss (losses[m], masks optional) and
 * the adjoint of fdx_pattern_backward (grads[m]).  The pattern of all models
 * runs in one persistent launch per tile shape (pixels per lane; at most two)
 * and the adjoint likewise; they take (model, tile) or (model, reflection,
 * band) items from an atomic
 * counter in the workspace, and each item is computed by one CTA or warp from
 * start to finish, so results do not depend on the order items are taken.
 * Every operation is a kernel launch or an asynchronous memset on `stream`,
 * so the step can be captured in a CUDA graph and replayed while the
 * problems' host parameters stay the same (atom coordinates and B, being
 * device arrays, may change between replays).  Hosemann lineshape only.
 */
int fdx_batch_refine(int32_t n_models, const fdx_problem *const *probs, const fdx_atoms *const *atoms,
                     float *const *F, float *const *M, float *const *images, const float *const *targets,
                     const float *const *masks, double *losses, const fdx_grads *const *grads, void *workspace,
                     size_t ws_bytes, void *stream);

/* Launch-shape settings (process-wide; chosen by the autotuner of the Python
 * package or set by hand).  They change speed only, never results beyond
 * the summation order of the adjoint's bands. */
typedef struct fdx_tuning {
    int32_t ppl_max;         /* 1 or 2: pixels per lane of the pattern kernels (2 is used only where the
                                8 x 8 patch spans <= 0.5 lattice periods, which keeps FP32 t accurate) */
    int32_t fwd_ctas_per_sm; /* persistent forward CTAs per SM in fdx_batch_refine, 1..8 */
    int32_t adj_ctas_per_sm; /* persistent adjoint CTAs per SM in fdx_batch_refine and fdx_pattern_backward, 1..8 */
    int32_t adj_bands;       /* detector bands per reflection in the adjoint work items, 1..256 */
    int32_t node_block;      /* 0..3: shape of the quadrature-node blocks that the pattern-family kernels
                                cull and stage as one unit, rows x columns of the node grid:
                                0 = 4 x 8, 1 = 8 x 4 (default), 2 = 2 x 16, 3 = 16 x 2.  Changes the order of the
                                node sums (results agree to rounding), not the set of terms */
} fdx_tuning;

/* Set the tuning (NULL restores the defaults 2, 4, 3, 128, 1).  Workspace sizes
 * depend on adj_bands: query them after setting. */
int fdx_set_tuning(const fdx_tuning *t);
int fdx_get_tuning(fdx_tuning *t);

/*
 * fdx_status -- wait for the work queued on `stream` (NULL: the legacy
 * default stream) and report how it ended.  The library's calls are
 * asynchronous after validation, so a fault inside a kernel surfaces only
 * here (or at the caller's next synchronisation).  *device_status (may be
 * NULL) receives the CUDA error code of the stream's work (0 = success).
 * Returns FDX_OK, or FDX_ERR_CUDA when that work failed.  No kernel of the
 * library waits on another kernel, a flag or a peer (the persistent kernels
 * take independent work items from an atomic counter), so there is no
 * device-side wait that could time out.
 */
int fdx_status(void *stream, int *device_status);

/* Human-readable text for a return code (static storage). */
/*
 * fdx_debug_status -- bounds checks of a debugging build.  A library compiled
 * with FDX_DEBUG defined and relocatable device code (the package's build
 * script writes it as libfdx_debug.so) checks its kernels' main indexing (node table, staging buffers, tile lists,
 * reflection records, pixel and gradient images, adjoint items,
 * structure-factor partial rows, batched position tables): an index outside
 * its buffer sets a bit in a device status word (bit k for check k, see
 * DebugCheck in the sources), records the index and skips the access.  This
 * call waits for the device, copies the word into *flags and the last bad
 * index into *last_index (either may be NULL), clears both, and returns 1.
 * A normal build has no checks: it sets *flags = 0, *last_index = -1 and
 * returns 0.  FDX_ERR_CUDA if the device copy fails.
 */
int fdx_debug_status(unsigned long long *flags, long long *last_index);

/* fdx_debug_probe -- in a debugging build, queue on `stream` one check that
 * fails on purpose (check 63, index 7; no memory but the status word is
 * touched), so that a caller can see fdx_debug_status report it; returns 1.
 * A normal build does nothing and returns 0. */
int fdx_debug_probe(void *stream);

const char *fdx_error_string(int code);

/* Library version as major*10000 + minor*100 + patch. */
int fdx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FDX_H */
