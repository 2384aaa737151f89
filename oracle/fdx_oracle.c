/*
 * FP64 CPU oracle for the fiber-diffraction hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference the GPU
 * path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the GPU library.
 *
 * What it computes (paper sections / equations):
 *   cell and reciprocal basis ........ Eq. recip_basis; Sect. "Unit cell and
 *                                      reciprocal-space frame" (c || z, b in
 *                                      the yz-plane)
 *   reflection list .................. Sect. "Structure factors and reflection
 *                                      list" (d_min <= d <= d_max, (000) out)
 *   structure factors ................ Eq. structure_factor with atomic form
 *                                      factor f(s) = sum a_i exp(-b_i s^2/4) + c
 *                                      and isotropic Debye-Waller exp(-B s^2/4)
 *                                      (Sect. "Paracrystalline disorder",
 *                                      B = 8 pi^2 <u^2>)
 *   per-reflection disorder .......... Eqs. Ah, breadth, Neff, Ipara; the
 *                                      anisotropic axis damping of Sect.
 *                                      "Paracrystalline disorder"
 *   lineshapes ....................... Eq. I_shape (sinc^2 with N_eff),
 *                                      Eq. Z (Hosemann) with the combined
 *                                      breadth of Eq. Neff, and the Gaussian
 *                                      of the same integral breadth (Eq.
 *                                      breadth)
 *   angular shapes ................... Sect. "Angular peak shapes": Gaussian,
 *                                      Lorentzian, Voigt normalised to g(0)=1;
 *                                      the Voigt is the convolution integral
 *                                      itself, evaluated by adaptive
 *                                      Gauss-Legendre quadrature
 *   shell nodes and weights .......... Eqs. gnomonic and node_weight on a
 *                                      midpoint grid
 *   ring average ..................... Eq. cyl-average by a per-reflection
 *                                      midpoint rule over the ring azimuth
 *   scatter form ..................... per-reflection samples of the shell
 *                                      (Eq. gnomonic), Eq. direct_sum at each,
 *                                      Eq. lorentz per sample, Ewald rotation
 *                                      by Eqs. harmonic/solutions, splat into
 *                                      the hit pixel
 *   pixel value ...................... Eq. direct_sum at the pixel's query
 *                                      point, Lorentz factor of Eq. lorentz,
 *                                      pixel -> scattering vector from the
 *                                      Ewald construction (Eq. laue)
 *   adjoint .......................... analytic derivatives of the above
 *
 * Readings where the paper is silent (numbered as in the design notes):
 *   R1  every hkl in the resolution sphere, Friedel mates included; a
 *       reflection exactly on d = d_min is kept (tolerance 1e-12 relative).
 *   R3  form-factor and Debye-Waller argument s^2/4 = (sin theta / lambda)^2.
 *   R4  N_base,i = L_i / |a_i| is real valued (not rounded).
 *   R5  beta_i = min(1, 1/N_base,i + tanh(pi^2 g_i^2 h_i^2)).
 *   R6  SINC: K = N sinc^2(N t), N = 1/beta, support |t| <= min(K_z/N, 1/2);
 *       HOSEMANN: Eq. Z with |phi| = (1-beta)/(1+beta), support |t| <= 1/2.
 *   R9  e1 = normalize(n x S^); if |n x S^| < 1e-12, e1 = normalize(b x S^).
 *   R10 n x n midpoint grid on [-T, T]^2, n nodes per axis.
 *   R12 the query point is the pixel's ring point in the reflection's
 *       meridional half-plane: p = Z n + R e_R(D); e_R = e1 if R_D ~ 0.
 *   R13 no polarisation, solid-angle or obliquity factor.
 *   R14 tilt 0; beam centre at the detector centre; pixel centres at
 *       half-integers.
 *
 * Parity pins live in tests/test_oracle_*.py.  The pattern value itself has
 * no printed worked example in the paper ("parity unpinned" for the readings
 * R6, R8, R10, R12 as definitions); its parts are pinned individually.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

typedef struct {
    double cell[6];          /* a, b, c (A); alpha, beta, gamma (rad) */
    double L[3];             /* crystallite size along a, b, c (A) */
    double g[3];             /* Hosemann g along a, b, c */
    double B_axis[3];        /* axis damping B_a, B_b, B_c (A^2) */
    int32_t lineshape;       /* 0 = sinc, 1 = Hosemann, 2 = Gaussian of matched breadth */
    int32_t intensity_model; /* 0 = none, 1 = Hosemann */
    double sigma, gamma;     /* orientation widths (rad) */
    double sigma_r;          /* radial shell width (1/A) */
    double T;                /* patch half-extent (tangent units) */
    int32_t n_nodes;         /* nodes per axis */
    int32_t pad0;
    double K_z;              /* sinc support in zeros */
    double wavelength, distance, pixel;
    int32_t n_x, n_y;
    double fiber[3], beam[3];
    double delta_L;
} or_params;

/* ------------------------------------------------------------------ */
/* small vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double *x, const double *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; }
static void cross3(const double *x, const double *y, double *z) {
    z[0] = x[1] * y[2] - x[2] * y[1];
    z[1] = x[2] * y[0] - x[0] * y[2];
    z[2] = x[0] * y[1] - x[1] * y[0];
}
static double norm3(const double *x) { return sqrt(dot3(x, x)); }

/* ------------------------------------------------------------------ */
/* Cell and reciprocal basis (Eq. recip_basis; UC_FULL convention)      */
/* A rows: a, b, c.  As rows: a*, b*, c*.                               */
/* ------------------------------------------------------------------ */
void or_basis(const double cell[6], double A[9], double As[9]) {
    double a = cell[0], b = cell[1], c = cell[2];
    double al = cell[3], be = cell[4], ga = cell[5];
    double *av = A, *bv = A + 3, *cv = A + 6;
    cv[0] = 0.0; cv[1] = 0.0; cv[2] = c;
    bv[0] = 0.0; bv[1] = b * sin(al); bv[2] = b * cos(al);
    av[2] = a * cos(be);
    av[1] = a * (cos(ga) - cos(al) * cos(be)) / sin(al);
    av[0] = sqrt(a * a - av[1] * av[1] - av[2] * av[2]);
    double bxc[3], cxa[3], axb[3];
    cross3(bv, cv, bxc);
    cross3(cv, av, cxa);
    cross3(av, bv, axb);
    double V = dot3(av, bxc);
    for (int k = 0; k < 3; k++) {
        As[k] = bxc[k] / V;
        As[3 + k] = cxa[k] / V;
        As[6 + k] = axb[k] / V;
    }
}

static void recip_vector(const double *As, int h, int k, int l, double *D) {
    for (int q = 0; q < 3; q++) D[q] = h * As[q] + k * As[3 + q] + l * As[6 + q];
}

/* ------------------------------------------------------------------ */
/* Reflection list: all (h,k,l) != 0 with d_min <= d <= d_max,          */
/* lexicographic order.  Returns the count; writes at most cap triples. */
/* ------------------------------------------------------------------ */
int32_t or_reflections(const double cell[6], double d_min, double d_max, int32_t cap, int32_t *hkl) {
    double A[9], As[9];
    or_basis(cell, A, As);
    int H = (int)ceil(cell[0] / d_min), K = (int)ceil(cell[1] / d_min), Lm = (int)ceil(cell[2] / d_min);
    double s2max = (1.0 + 1e-12) / (d_min * d_min);
    double s2min = d_max > 0.0 ? (1.0 - 1e-12) / (d_max * d_max) : 0.0;
    int32_t n = 0;
    for (int h = -H; h <= H; h++)
        for (int k = -K; k <= K; k++)
            for (int l = -Lm; l <= Lm; l++) {
                if (h == 0 && k == 0 && l == 0) continue;
                double D[3];
                recip_vector(As, h, k, l, D);
                double s2 = dot3(D, D);
                if (s2 > s2max || s2 < s2min) continue;
                if (n < cap) {
                    hkl[3 * n] = h;
                    hkl[3 * n + 1] = k;
                    hkl[3 * n + 2] = l;
                }
                n++;
            }
    return n;
}

/* ------------------------------------------------------------------ */
/* Structure factors, Eq. structure_factor:                              */
/*   F = sum_j occ_j f_e(s) exp(-B_j s^2/4) exp(2 pi i (h x + k y + l z)) */
/* F is written as (re, im) pairs.                                        */
/* ------------------------------------------------------------------ */
static double form_factor(const double *ff, double s2) {
    double f = ff[8];
    for (int i = 0; i < 4; i++) f += ff[i] * exp(-ff[4 + i] * s2 / 4.0);
    return f;
}

void or_structure_factors(const double cell[6], int32_t n_atoms, const double *frac, const double *B,
                          const double *occ, const int32_t *elem, const double *ff, int32_t n_refl,
                          const int32_t *hkl, double *F) {
    double A[9], As[9];
    or_basis(cell, A, As);
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t r = 0; r < n_refl; r++) {
        int h = hkl[3 * r], k = hkl[3 * r + 1], l = hkl[3 * r + 2];
        double D[3];
        recip_vector(As, h, k, l, D);
        double s2 = dot3(D, D);
        double re = 0.0, im = 0.0;
        for (int32_t j = 0; j < n_atoms; j++) {
            double f = form_factor(ff + 9 * elem[j], s2);
            double amp = occ[j] * f * exp(-B[j] * s2 / 4.0);
            double ph = h * frac[3 * j] + k * frac[3 * j + 1] + l * frac[3 * j + 2];
            ph -= nearbyint(ph);
            re += amp * cos(2.0 * OR_PI * ph);
            im += amp * sin(2.0 * OR_PI * ph);
        }
        F[2 * r] = re;
        F[2 * r + 1] = im;
    }
}

/* ------------------------------------------------------------------ */
/* Per-reflection disorder scalars (Eqs. Ah, breadth, Neff, Ipara;       */
/* axis damping D(S) = exp(-1/4 sum B_i (S . a^_i)^2)).                   */
/*   x_i = pi^2 g_i^2 h_i^2;  A_i = exp(-2 x_i);                         */
/*   (1 - A)/(1 + A) = tanh(x_i);   2A/(1 + A^2) = sech(2 x_i)           */
/*   beta_i = min(1, |a_i|/L_i + tanh x_i)            (R4, R5)           */
/* ------------------------------------------------------------------ */
void or_refl_scalars(const or_params *p, int32_t n_refl, const int32_t *hkl, double *beta, double *P,
                     double *DW) {
    double A[9], As[9];
    or_basis(p->cell, A, As);
    double alen[3] = {norm3(A), norm3(A + 3), norm3(A + 6)};
    for (int32_t r = 0; r < n_refl; r++) {
        double Pr = 1.0, dwarg = 0.0;
        for (int i = 0; i < 3; i++) {
            double hi = (double)hkl[3 * r + i];
            double x = OR_PI * OR_PI * p->g[i] * p->g[i] * hi * hi;
            double b = alen[i] / p->L[i] + tanh(x);
            beta[3 * r + i] = b < 1.0 ? b : 1.0;
            if (p->intensity_model == 1) Pr *= 1.0 / cosh(2.0 * x);
            /* S . a^_i at the reflection = h_i / |a_i| */
            double sa = hi / alen[i];
            dwarg += p->B_axis[i] * sa * sa;
        }
        P[r] = Pr;
        DW[r] = exp(-0.25 * dwarg);
    }
}

/* ------------------------------------------------------------------ */
/* Lineshapes K(t; beta) and dK/dbeta (reading R6)                       */
/* ------------------------------------------------------------------ */
static double sinc(double x) {
    if (x == 0.0) return 1.0;
    return sin(OR_PI * x) / (OR_PI * x);
}

double or_lineshape(int32_t lineshape, double t, double beta, double *dK_dbeta) {
    if (lineshape == 0) {
        double N = 1.0 / beta;
        double x = N * t;
        double sx = sinc(x);
        double K = N * sx * sx;
        if (dK_dbeta) {
            /* dK/dN at fixed t = 2 sinc(x) cos(pi x) - sinc(x)^2 ; dN/dbeta = -N^2 */
            double dKdN = 2.0 * sx * cos(OR_PI * x) - sx * sx;
            *dK_dbeta = -N * N * dKdN;
        }
        return K;
    } else if (lineshape == 1) {
        double s = sin(OR_PI * t);
        double s2 = s * s;
        double den = beta * beta + (1.0 - beta * beta) * s2;
        if (dK_dbeta) *dK_dbeta = (s2 * (1.0 + beta * beta) - beta * beta) / (den * den);
        return beta / den;
    } else {
        /* Gaussian of the same integral breadth beta (Sect. "Paracrystalline
         * disorder", the alternative to Eq. Z; reading R20): peak 1/beta, unit
         * integral, K = exp(-pi t^2 / beta^2) / beta. */
        double q = t / beta;
        double K = exp(-OR_PI * q * q) / beta;
        if (dK_dbeta) *dK_dbeta = K * (2.0 * OR_PI * q * q - 1.0) / beta;
        return K;
    }
}

double or_support(int32_t lineshape, double beta, double K_z) {
    if (lineshape == 0 || lineshape == 2) {
        double t = K_z * beta;
        return t < 0.5 ? t : 0.5;
    }
    return 0.5;
}

/* ------------------------------------------------------------------ */
/* Angular shapes g(delta; sigma, gamma), g(0) = 1 (Sect. "Angular peak  */
/* shapes").  Branches: gamma == 0 -> Gaussian; sigma < 1e-12 ->          */
/* Lorentzian; otherwise the Voigt convolution (G * L)(delta)/(G * L)(0)  */
/* evaluated as                                                          */
/*   U(delta) = int_{-pi/2}^{pi/2} exp(-(delta - gamma tan phi)^2/2s^2) dphi */
/* (substituting x = delta - gamma tan phi in int G(x) L(delta - x) dx;  */
/* the constant 1/(pi sigma sqrt(2 pi)) cancels in the ratio).            */
/* ------------------------------------------------------------------ */
typedef struct {
    double delta, sigma, gamma;
    int which; /* 0: U, 1: dU/dsigma, 2: dU/dgamma */
} voigt_ctx;

static double voigt_integrand(const voigt_ctx *c, double phi) {
    double tp = tan(phi);
    double q = c->delta - c->gamma * tp;
    double e = exp(-q * q / (2.0 * c->sigma * c->sigma));
    if (c->which == 0) return e;
    if (c->which == 1) return e * q * q / (c->sigma * c->sigma * c->sigma);
    return e * q * tp / (c->sigma * c->sigma);
}

/* Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n. */
#define GL_N 16
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void) {
    if (gl_ready) return;
    int n = GL_N;
    for (int i = 0; i < n; i++) {
        double x = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(x), p0 = P_{n-1}(x); P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1) */
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

static double gl_panel(const voigt_ctx *c, double a, double b) {
    double m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < GL_N; i++) s += gl_w[i] * voigt_integrand(c, m + h * gl_x[i]);
    return s * h;
}

static double gl_adapt(const voigt_ctx *c, double a, double b, double whole, double tol, int depth) {
    double m = 0.5 * (a + b);
    double l = gl_panel(c, a, m), r = gl_panel(c, m, b);
    if (depth >= 18 || fabs(l + r - whole) <= tol) return l + r;
    return gl_adapt(c, a, m, l, 0.5 * tol, depth + 1) + gl_adapt(c, m, b, r, 0.5 * tol, depth + 1);
}

static double voigt_U(double delta, double sigma, double gamma, int which) {
    voigt_ctx c = {delta, sigma, gamma, which};
    /* Break points at the images of delta + k sigma (k = -12..12), so every
       panel sees the Gaussian bump at a resolvable width. */
    double cuts[27];
    int nc = 0;
    cuts[nc++] = -0.5 * OR_PI;
    for (int k = -12; k <= 12; k++) cuts[nc++] = atan((delta + k * sigma) / gamma);
    cuts[nc++] = 0.5 * OR_PI;
    double coarse[27], scale = 0.0, total = 0.0;
    for (int i = 0; i + 1 < nc; i++) {
        double a = cuts[i], b = cuts[i + 1];
        coarse[i] = b > a ? gl_panel(&c, a, b) : 0.0;
        scale += fabs(coarse[i]);
    }
    for (int i = 0; i + 1 < nc; i++) {
        double a = cuts[i], b = cuts[i + 1];
        if (b <= a) continue;
        total += gl_adapt(&c, a, b, coarse[i], 2e-15 * scale + 1e-300, 0);
    }
    return total;
}

double or_angular(double delta, double sigma, double gamma, double *dg_dsigma, double *dg_dgamma) {
    if (gamma == 0.0) {
        double g = exp(-delta * delta / (2.0 * sigma * sigma));
        if (dg_dsigma) *dg_dsigma = g * delta * delta / (sigma * sigma * sigma);
        if (dg_dgamma) *dg_dgamma = 0.0; /* pure-Gaussian branch: gamma is not a parameter */
        return g;
    }
    if (sigma < 1e-12) {
        double den = delta * delta + gamma * gamma;
        if (dg_dsigma) *dg_dsigma = 0.0;
        if (dg_dgamma) *dg_dgamma = 2.0 * gamma * delta * delta / (den * den);
        return gamma * gamma / den;
    }
    gl_init();
    double U = voigt_U(delta, sigma, gamma, 0), U0 = voigt_U(0.0, sigma, gamma, 0);
    double g = U / U0;
    if (dg_dsigma) {
        double Us = voigt_U(delta, sigma, gamma, 1), U0s = voigt_U(0.0, sigma, gamma, 1);
        *dg_dsigma = (Us * U0 - U * U0s) / (U0 * U0);
    }
    if (dg_dgamma) {
        double Ug = voigt_U(delta, sigma, gamma, 2), U0g = voigt_U(0.0, sigma, gamma, 2);
        *dg_dgamma = (Ug * U0 - U * U0g) / (U0 * U0);
    }
    return g;
}

/* ------------------------------------------------------------------ */
/* Shell nodes, Eqs. gnomonic and node_weight (reading R10):             */
/*   d_j = -T + (j + 1/2) 2T/n,  node k = (j, m) with d1 = d_j, d2 = d_m   */
/*   w = sigma_r sqrt(2 pi) g(Delta) (1 + d1^2 + d2^2)^(-3/2) (2T/n)^2     */
/*   Delta = arccos((1 + d^2)^(-1/2)) = atan(|d|)                          */
/* The r0^2 factor of Eq. node_weight is applied per reflection.          */
/* ------------------------------------------------------------------ */
void or_nodes(const or_params *p, double *d1, double *d2, double *w, double *dw_dsigma, double *dw_dgamma) {
    gl_init();
    int n = p->n_nodes;
    double h = 2.0 * p->T / n;
    double pre = p->sigma_r * sqrt(2.0 * OR_PI) * h * h;
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < n; j++)
        for (int m = 0; m < n; m++) {
            double a1 = -p->T + (j + 0.5) * h, a2 = -p->T + (m + 0.5) * h;
            double rho2 = a1 * a1 + a2 * a2;
            double Delta = atan(sqrt(rho2));
            double gs = 0.0, gg = 0.0;
            double g = or_angular(Delta, p->sigma, p->gamma, &gs, &gg);
            double jac = pow(1.0 + rho2, -1.5);
            int k = j * n + m;
            d1[k] = a1;
            d2[k] = a2;
            w[k] = pre * g * jac;
            if (dw_dsigma) dw_dsigma[k] = pre * gs * jac;
            if (dw_dgamma) dw_dgamma[k] = pre * gg * jac;
        }
}

/* ------------------------------------------------------------------ */
/* Detector pixel -> scattering vector (Ewald construction, Eq. laue):   */
/* u = (i + 1/2 - n_x/2) p along u^ = normalize(n x b),                  */
/* v = (j + 1/2 - n_y/2) p along v^ = b x u^, r = SF b + u u^ + v v^,     */
/* k_out = r / (lambda |r|), k_in = b / lambda, S = k_out - k_in.          */
/* ------------------------------------------------------------------ */
static void detector_frame(const or_params *p, double *bh, double *nh, double *uh, double *vh) {
    double bn = norm3(p->beam), nn = norm3(p->fiber);
    for (int q = 0; q < 3; q++) {
        bh[q] = p->beam[q] / bn;
        nh[q] = p->fiber[q] / nn;
    }
    double t[3];
    cross3(nh, bh, t);
    double tn = norm3(t);
    for (int q = 0; q < 3; q++) uh[q] = t[q] / tn;
    cross3(bh, uh, vh);
}

void or_pixel_S(const or_params *p, int32_t i, int32_t j, double *S, double *R, double *Z) {
    double bh[3], nh[3], uh[3], vh[3];
    detector_frame(p, bh, nh, uh, vh);
    double u = (i + 0.5 - 0.5 * p->n_x) * p->pixel;
    double v = (j + 0.5 - 0.5 * p->n_y) * p->pixel;
    double r[3];
    for (int q = 0; q < 3; q++) r[q] = p->distance * bh[q] + u * uh[q] + v * vh[q];
    double rn = norm3(r);
    for (int q = 0; q < 3; q++) S[q] = r[q] / (p->wavelength * rn) - bh[q] / p->wavelength;
    double z = dot3(S, nh);
    double perp[3];
    for (int q = 0; q < 3; q++) perp[q] = S[q] - z * nh[q];
    *Z = z;
    *R = norm3(perp);
}

/* ------------------------------------------------------------------ */
/* Pattern (Eq. direct_sum + Eq. lorentz at the pixel's query point).     */
/* ------------------------------------------------------------------ */
typedef struct {
    double r0, Sh[3], e1[3], e2[3], eR[3];
    double beta[3], tmax[3];
    double rhoB; /* circumradius of the support box */
} refl_geo;

static void build_refl_geo(const or_params *p, const double *A, const double *As, const double *nh,
                           const double *bh, int32_t n_refl, const int32_t *hkl, const double *beta,
                           refl_geo *G) {
    for (int32_t r = 0; r < n_refl; r++) {
        refl_geo *g = &G[r];
        double D[3];
        recip_vector(As, hkl[3 * r], hkl[3 * r + 1], hkl[3 * r + 2], D);
        g->r0 = norm3(D);
        for (int q = 0; q < 3; q++) g->Sh[q] = D[q] / g->r0;
        double t[3];
        cross3(nh, g->Sh, t);
        double tn = norm3(t);
        if (tn < 1e-12) {
            cross3(bh, g->Sh, t);
            tn = norm3(t);
        }
        for (int q = 0; q < 3; q++) g->e1[q] = t[q] / tn;
        cross3(g->Sh, g->e1, g->e2);
        double ZD = dot3(D, nh);
        double perp[3];
        for (int q = 0; q < 3; q++) perp[q] = D[q] - ZD * nh[q];
        double RD = norm3(perp);
        if (RD < 1e-12 * g->r0) {
            for (int q = 0; q < 3; q++) g->eR[q] = g->e1[q];
        } else {
            for (int q = 0; q < 3; q++) g->eR[q] = perp[q] / RD;
        }
        for (int i = 0; i < 3; i++) {
            g->beta[i] = beta[3 * r + i];
            g->tmax[i] = or_support(p->lineshape, g->beta[i], p->K_z);
        }
        /* box {X : |a_i . X| <= tmax_i} = { sum_i t_i a*_i : |t_i| <= tmax_i } */
        double best = 0.0;
        for (int sb = 0; sb < 4; sb++) {
            double sgn_b = (sb & 1) ? -1.0 : 1.0, sgn_c = (sb & 2) ? -1.0 : 1.0;
            double X[3];
            for (int q = 0; q < 3; q++)
                X[q] = g->tmax[0] * As[q] + sgn_b * g->tmax[1] * As[3 + q] + sgn_c * g->tmax[2] * As[6 + q];
            double xn = norm3(X);
            if (xn > best) best = xn;
        }
        g->rhoB = best;
    }
    (void)A;
}

/*
 * I_out[q] = L(R) sum_r M_r r0^2 sum_{k in supp} w_k prod_i K_i(a_i . (p - s_k))
 * E_out[3q + 0] = number of (reflection, node) terms inside the support
 * E_out[3q + 1] = same count with the support shrunk by eta (strict)
 * E_out[3q + 2] = same count with the support grown by eta (loose)
 * A_out[q] (nullable) = L(R) sum_r M_r r0^2 sum over the nodes counted by the
 * loose count but not by the strict one of |w_k prod_i K_i|: the terms whose
 * inclusion is decided within eta of the support's edge.  The support ends
 * where K is not zero (the Hosemann factor is beta at |t| = 1/2), so these
 * terms are whole jumps of the sum: a computation whose t carries rounding of
 * order eta may include or drop any of them, and A bounds what that changes.
 * cull != 0 skips reflections with | |p| - r0 | > rhoB, which contain no
 * node inside the support (|p - s| <= rhoB and |s| = r0); the result is
 * identical with cull = 0.
 */
void or_pattern(const or_params *p, int32_t n_refl, const int32_t *hkl, const double *M, int32_t n_pix,
                const int32_t *pix, int32_t cull, double eta, double *I_out, int64_t *E_out, double *A_out) {
    double A[9], As[9];
    or_basis(p->cell, A, As);
    double bh[3], nh[3], uh[3], vh[3];
    detector_frame(p, bh, nh, uh, vh);
    int nn = p->n_nodes * p->n_nodes;
    double *d1 = malloc(sizeof(double) * nn), *d2 = malloc(sizeof(double) * nn), *w = malloc(sizeof(double) * nn);
    or_nodes(p, d1, d2, w, NULL, NULL);
    double *beta = malloc(sizeof(double) * 3 * (n_refl > 0 ? n_refl : 1));
    double *Pv = malloc(sizeof(double) * (n_refl > 0 ? n_refl : 1));
    double *DWv = malloc(sizeof(double) * (n_refl > 0 ? n_refl : 1));
    or_refl_scalars(p, n_refl, hkl, beta, Pv, DWv);
    refl_geo *G = malloc(sizeof(refl_geo) * (n_refl > 0 ? n_refl : 1));
    build_refl_geo(p, A, As, nh, bh, n_refl, hkl, beta, G);

#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t q = 0; q < n_pix; q++) {
        double S[3], R, Z;
        or_pixel_S(p, pix[2 * q], pix[2 * q + 1], S, &R, &Z);
        double plen = sqrt(R * R + Z * Z);
        double acc = 0.0, amb = 0.0;
        int64_t e0 = 0, e1c = 0, e2c = 0;
        for (int32_t r = 0; r < n_refl; r++) {
            const refl_geo *g = &G[r];
            if (cull && fabs(plen - g->r0) > g->rhoB * (1.0 + 1e-9) + 1e-12) continue;
            double pq[3];
            for (int c = 0; c < 3; c++) pq[c] = Z * nh[c] + R * g->eR[c];
            double sum = 0.0, edge = 0.0;
            for (int k = 0; k < nn; k++) {
                double inv = 1.0 / sqrt(1.0 + d1[k] * d1[k] + d2[k] * d2[k]);
                double X[3];
                for (int c = 0; c < 3; c++)
                    X[c] = pq[c] - g->r0 * (g->Sh[c] + d1[k] * g->e1[c] + d2[k] * g->e2[c]) * inv;
                double t[3];
                double excess = -1e300;
                for (int i = 0; i < 3; i++) {
                    t[i] = dot3(A + 3 * i, X);
                    double ex = fabs(t[i]) - g->tmax[i];
                    if (ex > excess) excess = ex;
                }
                if (excess <= -eta) e1c++;
                if (excess <= eta) e2c++;
                if (A_out && excess > -eta && excess <= eta) {
                    double Ke = 1.0;
                    for (int i = 0; i < 3; i++) Ke *= or_lineshape(p->lineshape, t[i], g->beta[i], NULL);
                    edge += fabs(w[k] * Ke);
                }
                if (excess > 0.0) continue;
                e0++;
                double Kp = 1.0;
                for (int i = 0; i < 3; i++) Kp *= or_lineshape(p->lineshape, t[i], g->beta[i], NULL);
                sum += w[k] * Kp;
            }
            acc += M[r] * g->r0 * g->r0 * sum;
            amb += fabs(M[r]) * g->r0 * g->r0 * edge;
        }
        double Lf = p->delta_L / (R + p->delta_L);
        I_out[q] = Lf * acc;
        if (A_out) A_out[q] = Lf * amb;
        if (E_out) {
            E_out[3 * q] = e0;
            E_out[3 * q + 1] = e1c;
            E_out[3 * q + 2] = e2c;
        }
    }
    free(d1); free(d2); free(w); free(beta); free(Pv); free(DWv); free(G);
}

/*
 * Ring-integrated cylindrical average (Eq. cyl-average; reading R21): the
 * pixel value is the average of the reciprocal-space intensity over the ring
 * of the pixel's (R, Z) about the fiber axis, with no Lorentz factor:
 *   I = sum_r M_r r0^2 (1/2pi) int dphi sum_k w_k prod_i K_i(a_i . (p(phi) - s_k)),
 *   p(phi) = Z n + R (cos(phi) e_R + sin(phi) e_P),  e_P = n x e_R,
 * phi measured from the reflection's meridional half-plane.  Quadrature per
 * reflection (or_ring_grid): the midpoint rule with N_r points on
 * [-Phi_r, Phi_r], outside which the ring cannot come within
 * rho_tot = rho_B + sqrt(2) r0 T of D (no node is in the support there), and
 * N_r = clamp(ceil(2 Phi_r / dphi), 4, max_n) with the step dphi =
 * w_min / (4 (R_D + rho_tot)), w_min = min_i beta_i / |a_i| (a quarter of the
 * narrowest lattice breadth along the ring at its largest radius).  `over`
 * multiplies N_r (1 for the definition; larger values refine the rule, for
 * convergence checks).
 */
void or_ring_grid_over(double r0, double RD, double rhoB, double T, double w_min, int32_t max_n, int32_t over,
                       double *Phi, int32_t *N) {
    const double rt = rhoB + sqrt(2.0) * r0 * T;
    double ph = OR_PI;
    const double inner = RD - rt;
    if (inner > 0.0) {
        const double x = rt / (2.0 * sqrt(inner * RD));
        if (x < 1.0) ph = 2.0 * asin(x);
    }
    const double dphi = w_min / (4.0 * (RD + rt));
    double n = ceil(2.0 * ph / dphi) * over;
    if (!(n >= 4.0)) n = 4.0;
    if (n > (double)max_n) n = (double)max_n;
    *Phi = ph;
    *N = (int32_t)n;
}

void or_ring_grid(double r0, double RD, double rhoB, double T, double w_min, int32_t max_n, double *Phi, int32_t *N) {
    or_ring_grid_over(r0, RD, rhoB, T, w_min, max_n, 1, Phi, N);
}

/* sum_k w_k prod_i K_i(a_i . (pq - s_k)) over the nodes in the support of pq;
 * *E (nullable) counts them. */
static double node_sum(const or_params *p, const double *A, const refl_geo *g, const double *d1, const double *d2,
                       const double *w, int nn, const double *pq, int64_t *E) {
    double sum = 0.0;
    for (int k = 0; k < nn; k++) {
        double inv = 1.0 / sqrt(1.0 + d1[k] * d1[k] + d2[k] * d2[k]);
        double X[3];
        for (int c = 0; c < 3; c++) X[c] = pq[c] - g->r0 * (g->Sh[c] + d1[k] * g->e1[c] + d2[k] * g->e2[c]) * inv;
        double t[3];
        int in = 1;
        for (int i = 0; i < 3; i++) {
            t[i] = dot3(A + 3 * i, X);
            if (fabs(t[i]) > g->tmax[i]) in = 0;
        }
        if (!in) continue;
        if (E) (*E)++;
        double Kp = 1.0;
        for (int i = 0; i < 3; i++) Kp *= or_lineshape(p->lineshape, t[i], g->beta[i], NULL);
        sum += w[k] * Kp;
    }
    return sum;
}

void or_ring(const or_params *p, int32_t n_refl, const int32_t *hkl, const double *M, int32_t n_pix,
             const int32_t *pix, int32_t max_n, int32_t over, double *I_out, int64_t *E_out) {
    double A[9], As[9];
    or_basis(p->cell, A, As);
    double bh[3], nh[3], uh[3], vh[3];
    detector_frame(p, bh, nh, uh, vh);
    int nn = p->n_nodes * p->n_nodes;
    double *d1 = malloc(sizeof(double) * nn), *d2 = malloc(sizeof(double) * nn), *w = malloc(sizeof(double) * nn);
    or_nodes(p, d1, d2, w, NULL, NULL);
    double *beta = malloc(sizeof(double) * 3 * (n_refl > 0 ? n_refl : 1));
    double *Pv = malloc(sizeof(double) * (n_refl > 0 ? n_refl : 1));
    double *DWv = malloc(sizeof(double) * (n_refl > 0 ? n_refl : 1));
    or_refl_scalars(p, n_refl, hkl, beta, Pv, DWv);
    refl_geo *G = malloc(sizeof(refl_geo) * (n_refl > 0 ? n_refl : 1));
    build_refl_geo(p, A, As, nh, bh, n_refl, hkl, beta, G);
    double alen[3];
    for (int i = 0; i < 3; i++) alen[i] = norm3(A + 3 * i);

#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t q = 0; q < n_pix; q++) {
        double S[3], R, Z;
        or_pixel_S(p, pix[2 * q], pix[2 * q + 1], S, &R, &Z);
        const double plen = sqrt(R * R + Z * Z);
        double acc = 0.0;
        int64_t e0 = 0;
        for (int32_t r = 0; r < n_refl; r++) {
            const refl_geo *g = &G[r];
            if (fabs(plen - g->r0) > g->rhoB * (1.0 + 1e-9) + 1e-12) continue;
            double D[3];
            for (int c = 0; c < 3; c++) D[c] = g->r0 * g->Sh[c];
            const double RD = dot3(D, g->eR);
            double eP[3];
            cross3(nh, g->eR, eP);
            double w_min = 1e300;
            for (int i = 0; i < 3; i++) {
                const double wi = g->beta[i] / alen[i];
                if (wi < w_min) w_min = wi;
            }
            double Phi;
            int32_t N;
            or_ring_grid_over(g->r0, RD, g->rhoB, p->T, w_min, max_n, over, &Phi, &N);
            const double rt = g->rhoB + sqrt(2.0) * g->r0 * p->T;
            const double h = 2.0 * Phi / N;
            double ring = 0.0;
            for (int32_t j = 0; j < N; j++) {
                const double phi = -Phi + (j + 0.5) * h;
                double pq[3], dd[3];
                for (int c = 0; c < 3; c++) pq[c] = Z * nh[c] + R * (cos(phi) * g->eR[c] + sin(phi) * eP[c]);
                for (int c = 0; c < 3; c++) dd[c] = pq[c] - D[c];
                if (norm3(dd) > rt) continue; /* no node can be in the support */
                ring += node_sum(p, A, g, d1, d2, w, nn, pq, &e0);
            }
            acc += M[r] * g->r0 * g->r0 * ring * h / (2.0 * OR_PI);
        }
        I_out[q] = acc;
        if (E_out) E_out[q] = e0;
    }
    free(d1); free(d2); free(w); free(beta); free(Pv); free(DWv); free(G);
}

/* Reciprocal-space intensity at arbitrary points (no Lorentz factor):
 *   I(S) = sum_r M_r r0^2 sum_k w_k prod_i K_i(a_i . (S - s_k)). */
void or_point(const or_params *p, int32_t n_refl, const int32_t *hkl, const double *M, int32_t n_pt,
              const double *pts, double *I_out) {
    double A[9], As[9];
    or_basis(p->cell, A, As);
    double bh[3], nh[3], uh[3], vh[3];
    detector_frame(p, bh, nh, uh, vh);
    int nn = p->n_nodes * p->n_nodes;
    double *d1 = malloc(sizeof(double) * nn), *d2 = malloc(sizeof(double) * nn), *w = malloc(sizeof(double) * nn);
    or_nodes(p, d1, d2, w, NULL, NULL);
    double *beta = malloc(sizeof(double) * 3 * (n_refl > 0 ? n_refl : 1));
    double *Pv = malloc(sizeof(double) * (n_refl > 0 ? n_refl : 1));
    double *DWv = malloc(sizeof(double) * (n_refl > 0 ? n_refl : 1));
    or_refl_scalars(p, n_refl, hkl, beta, Pv, DWv);
    refl_geo *G = malloc(sizeof(refl_geo) * (n_refl > 0 ? n_refl : 1));
    build_refl_geo(p, A, As, nh, bh, n_refl, hkl, beta, G);
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t q = 0; q < n_pt; q++) {
        double acc = 0.0;
        for (int32_t r = 0; r < n_refl; r++)
            acc += M[r] * G[r].r0 * G[r].r0 * node_sum(p, A, &G[r], d1, d2, w, nn, pts + 3 * (size_t)q, NULL);
        I_out[q] = acc;
    }
    free(d1); free(d2); free(w); free(beta); free(Pv); free(DWv); free(G);
}

/*
 * Scatter form of the projection (the paper's own pipeline; Sects. "Numerical
 * evaluation: per-reflection shell quadrature", "Lorentz correction on a
 * sampled reciprocal lattice", "Analytical Solution of the Ewald Diffraction
 * Condition"; reading R22).  For every reflection and every sample m with
 * normalised coordinates (xr, x1, x2) in [-1, 1]^3 and quadrature weight q:
 *   h_r = rho_B (support circumradius), d_i = x_i T, c = (1 + d^2)^(-1/2),
 *   S = (r0 + xr h_r) c (Sh + d1 e1 + d2 e2)                    (Eq. gnomonic)
 *   dV = q h_r T^2 (r0 + xr h_r)^2 c^3                         (r^2 dr dOmega)
 *   I = M r0^2 sum_k w_k prod_i K_i(a_i . (S - s_k))           (Eq. direct_sum)
 *   L = delta_L / (R + delta_L), R = |S - (S.n) n|             (Eq. lorentz)
 * S is rotated about the fiber axis into the diffraction condition with the
 * closed form of Eqs. harmonic and solutions (two solutions, none when
 * |R/sqrt(P^2+Q^2)| > 1, Eq. valid); each k_out = k_in + S_phi with
 * k_out . b > 0 is followed to the flat detector at distance SF, and the
 * hit is rendered as a spot (the paper's detector spot size, reading R25):
 * the spot x spot block of pixels centred on the pixel containing the hit
 * (spot odd) each receives dV L I / spot^2; parts of the block off the
 * detector are lost, as a hit off the detector is.  spot = 1 is the pixel
 * containing the hit.  img[ny][nx] is accumulated (not cleared).  samp (nullable) receives per
 * (reflection, sample) 8 values: I, dV, L, the two hits' continuous pixel
 * coordinates x = u/p + n_x/2, y = v/p + n_y/2 (NaN when there is no hit),
 * and the smallest distance of any node from the edge of the support,
 * min_k |max_i (|t_i| - t_max,i)| (how close the sample is to a node entering
 * or leaving the sum).
 * E (nullable) receives the number of in-support (sample, node) terms.
 */
void or_scatter(const or_params *p, int32_t n_refl, const int32_t *hkl, const double *M, int32_t n_s,
                const double *xs, int32_t spot, double *img, double *samp, int64_t *E) {
    double A[9], As[9];
    or_basis(p->cell, A, As);
    double bh[3], nh[3], uh[3], vh[3];
    detector_frame(p, bh, nh, uh, vh);
    int nn = p->n_nodes * p->n_nodes;
    double *d1 = malloc(sizeof(double) * nn), *d2 = malloc(sizeof(double) * nn), *w = malloc(sizeof(double) * nn);
    or_nodes(p, d1, d2, w, NULL, NULL);
    double *beta = malloc(sizeof(double) * 3 * (n_refl > 0 ? n_refl : 1));
    double *Pv = malloc(sizeof(double) * (n_refl > 0 ? n_refl : 1));
    double *DWv = malloc(sizeof(double) * (n_refl > 0 ? n_refl : 1));
    or_refl_scalars(p, n_refl, hkl, beta, Pv, DWv);
    refl_geo *G = malloc(sizeof(refl_geo) * (n_refl > 0 ? n_refl : 1));
    build_refl_geo(p, A, As, nh, bh, n_refl, hkl, beta, G);
    const double lam = p->wavelength, T = p->T;
    double kin[3];
    for (int q = 0; q < 3; q++) kin[q] = bh[q] / lam;
    const int npx = p->n_x * p->n_y;
    int64_t etot = 0;
#pragma omp parallel
    {
        double *loc = calloc((size_t)npx, sizeof(double));
        int64_t eloc = 0;
#pragma omp for schedule(dynamic, 1)
        for (int32_t r = 0; r < n_refl; r++) {
            const refl_geo *g = &G[r];
            const double hr = g->rhoB;
            for (int32_t m = 0; m < n_s; m++) {
                const double *x = xs + 4 * (size_t)m;
                const double rr = g->r0 + x[0] * hr, dd1 = x[1] * T, dd2 = x[2] * T;
                const double c = 1.0 / sqrt(1.0 + dd1 * dd1 + dd2 * dd2);
                double S[3];
                for (int q = 0; q < 3; q++) S[q] = rr * c * (g->Sh[q] + dd1 * g->e1[q] + dd2 * g->e2[q]);
                const double dV = x[3] * hr * T * T * rr * rr * c * c * c;
                double sum = 0.0, edge = 1e300;
                for (int k = 0; k < nn; k++) {
                    double inv = 1.0 / sqrt(1.0 + d1[k] * d1[k] + d2[k] * d2[k]);
                    double X[3];
                    for (int q = 0; q < 3; q++)
                        X[q] = S[q] - g->r0 * (g->Sh[q] + d1[k] * g->e1[q] + d2[k] * g->e2[q]) * inv;
                    double t[3];
                    double excess = -1e300;
                    for (int i = 0; i < 3; i++) {
                        t[i] = dot3(A + 3 * i, X);
                        double ex = fabs(t[i]) - g->tmax[i];
                        if (ex > excess) excess = ex;
                    }
                    if (fabs(excess) < edge) edge = fabs(excess);
                    if (excess > 0.0) continue;
                    eloc++;
                    double Kp = 1.0;
                    for (int i = 0; i < 3; i++) Kp *= or_lineshape(p->lineshape, t[i], g->beta[i], NULL);
                    sum += w[k] * Kp;
                }
                const double I = M[r] * g->r0 * g->r0 * sum;
                const double Z = dot3(S, nh);
                double perp[3];
                for (int q = 0; q < 3; q++) perp[q] = S[q] - Z * nh[q];
                const double R = norm3(perp);
                const double L = p->delta_L / (R + p->delta_L);
                double *o = samp ? samp + 8 * ((size_t)r * n_s + m) : NULL;
                if (o) o[0] = I, o[1] = dV, o[2] = L, o[3] = o[4] = o[5] = o[6] = NAN, o[7] = edge;
                /* Eqs. harmonic / solutions: P cos(phi) + Q sin(phi) = R_ */
                double nxS[3];
                cross3(nh, S, nxS);
                const double Aq = dot3(kin, S), Bq = dot3(kin, nxS), Dq = dot3(kin, nh) * dot3(nh, S);
                const double Cq = dot3(kin, kin) + dot3(S, S);
                const double Eq = (1.0 / (lam * lam) - Cq) / 2.0 - Dq;
                const double Pp = Aq - Dq, Qp = Bq, Rp = Eq;
                const double ratio = Rp / sqrt(Pp * Pp + Qp * Qp);
                if (!(fabs(ratio) <= 1.0)) continue;
                const double phi0 = atan2(Qp, Pp), dphi = acos(ratio);
                for (int br = 0; br < 2; br++) {
                    const double phi = br == 0 ? phi0 + dphi : phi0 - dphi;
                    const double cp = cos(phi), sp = sin(phi), nS = dot3(nh, S);
                    double ko[3];
                    for (int q = 0; q < 3; q++) ko[q] = kin[q] + S[q] * cp + nxS[q] * sp + nh[q] * nS * (1.0 - cp);
                    const double kb = dot3(ko, bh);
                    if (!(kb > 0.0)) continue;
                    const double xp = p->distance * dot3(ko, uh) / kb / p->pixel + 0.5 * p->n_x;
                    const double yp = p->distance * dot3(ko, vh) / kb / p->pixel + 0.5 * p->n_y;
                    if (o) o[3 + 2 * br] = xp, o[4 + 2 * br] = yp;
                    const double fi = floor(xp), fj = floor(yp);
                    const int half = (spot - 1) / 2;
                    const double share = dV * L * I / ((double)spot * spot);
                    for (int dj = -half; dj <= half; dj++)
                        for (int di = -half; di <= half; di++) {
                            const double qi = fi + di, qj = fj + dj;
                            if (qi < 0.0 || qj < 0.0 || qi >= p->n_x || qj >= p->n_y) continue;
                            loc[(size_t)qj * p->n_x + (size_t)qi] += share;
                        }
                }
            }
        }
#pragma omp critical
        {
            for (int q = 0; q < npx; q++) img[q] += loc[q];
            etot += eloc;
        }
        free(loc);
    }
    if (E) *E = etot;
    free(d1); free(d2); free(w); free(beta); free(Pv); free(DWv); free(G);
}

/*
 * Adjoint of or_pattern for an upstream gradient gI[q] = dLoss/dI_q over the
 * listed pixels.  Outputs (all accumulated over the pixels):
 *   G_refl[r]      = dLoss/dM_r
 *   dbeta[3r + i]  = dLoss/dbeta_{r,i}   (at fixed M)
 *   *dsigma, *dgamma = dLoss/dsigma, dLoss/dgamma through the node weights
 *                      (T held fixed, reading R11)
 */
void or_pattern_adjoint(const or_params *p, int32_t n_refl, const int32_t *hkl, const double *M,
                        int32_t n_pix, const int32_t *pix, const double *gI, double *G_refl, double *dbeta,
                        double *dsigma, double *dgamma) {
    double A[9], As[9];
    or_basis(p->cell, A, As);
    double bh[3], nh[3], uh[3], vh[3];
    detector_frame(p, bh, nh, uh, vh);
    int nn = p->n_nodes * p->n_nodes;
    double *d1 = malloc(sizeof(double) * nn), *d2 = malloc(sizeof(double) * nn), *w = malloc(sizeof(double) * nn);
    double *ws = malloc(sizeof(double) * nn), *wg = malloc(sizeof(double) * nn);
    or_nodes(p, d1, d2, w, ws, wg);
    int32_t nr = n_refl > 0 ? n_refl : 1;
    double *beta = malloc(sizeof(double) * 3 * nr), *Pv = malloc(sizeof(double) * nr), *DWv = malloc(sizeof(double) * nr);
    or_refl_scalars(p, n_refl, hkl, beta, Pv, DWv);
    refl_geo *G = malloc(sizeof(refl_geo) * nr);
    build_refl_geo(p, A, As, nh, bh, n_refl, hkl, beta, G);

    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *accG = calloc((size_t)nthreads * nr, sizeof(double));
    double *accB = calloc((size_t)nthreads * 3 * nr, sizeof(double));
    double *accS = calloc((size_t)nthreads * 2, sizeof(double));

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *myG = accG + (size_t)tid * nr, *myB = accB + (size_t)tid * 3 * nr, *myS = accS + 2 * tid;
#pragma omp for schedule(dynamic, 1)
        for (int32_t q = 0; q < n_pix; q++) {
            if (gI[q] == 0.0) continue;
            double S[3], R, Z;
            or_pixel_S(p, pix[2 * q], pix[2 * q + 1], S, &R, &Z);
            double plen = sqrt(R * R + Z * Z);
            double c = gI[q] * p->delta_L / (R + p->delta_L);
            for (int32_t r = 0; r < n_refl; r++) {
                const refl_geo *g = &G[r];
                if (fabs(plen - g->r0) > g->rhoB * (1.0 + 1e-9) + 1e-12) continue;
                double pq[3];
                for (int cc = 0; cc < 3; cc++) pq[cc] = Z * nh[cc] + R * g->eR[cc];
                double sK = 0.0, sB[3] = {0, 0, 0}, sS = 0.0, sGm = 0.0;
                for (int k = 0; k < nn; k++) {
                    double inv = 1.0 / sqrt(1.0 + d1[k] * d1[k] + d2[k] * d2[k]);
                    double X[3];
                    for (int cc = 0; cc < 3; cc++)
                        X[cc] = pq[cc] - g->r0 * (g->Sh[cc] + d1[k] * g->e1[cc] + d2[k] * g->e2[cc]) * inv;
                    double t[3];
                    int in = 1;
                    for (int i = 0; i < 3; i++) {
                        t[i] = dot3(A + 3 * i, X);
                        if (fabs(t[i]) > g->tmax[i]) in = 0;
                    }
                    if (!in) continue;
                    double K[3], dK[3];
                    for (int i = 0; i < 3; i++) K[i] = or_lineshape(p->lineshape, t[i], g->beta[i], &dK[i]);
                    double Kp = K[0] * K[1] * K[2];
                    sK += w[k] * Kp;
                    sB[0] += w[k] * dK[0] * K[1] * K[2];
                    sB[1] += w[k] * K[0] * dK[1] * K[2];
                    sB[2] += w[k] * K[0] * K[1] * dK[2];
                    sS += ws[k] * Kp;
                    sGm += wg[k] * Kp;
                }
                double f = c * g->r0 * g->r0;
                myG[r] += f * sK;
                for (int i = 0; i < 3; i++) myB[3 * r + i] += f * M[r] * sB[i];
                myS[0] += f * M[r] * sS;
                myS[1] += f * M[r] * sGm;
            }
        }
    }
    for (int32_t r = 0; r < n_refl; r++) {
        double s = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0;
        for (int t = 0; t < nthreads; t++) {
            s += accG[(size_t)t * nr + r];
            b0 += accB[(size_t)t * 3 * nr + 3 * r];
            b1 += accB[(size_t)t * 3 * nr + 3 * r + 1];
            b2 += accB[(size_t)t * 3 * nr + 3 * r + 2];
        }
        G_refl[r] = s;
        dbeta[3 * r] = b0;
        dbeta[3 * r + 1] = b1;
        dbeta[3 * r + 2] = b2;
    }
    double ss = 0.0, sg = 0.0;
    for (int t = 0; t < nthreads; t++) {
        ss += accS[2 * t];
        sg += accS[2 * t + 1];
    }
    *dsigma = ss;
    *dgamma = sg;
    free(d1); free(d2); free(w); free(ws); free(wg); free(beta); free(Pv); free(DWv); free(G);
    free(accG); free(accB); free(accS);
}

/*
 * Chain rule from per-reflection adjoints to the global disorder parameters:
 *   dLoss/dL_i = sum_r dbeta_{r,i} dbeta_{r,i}/dL_i
 *   dLoss/dg_i = sum_r dbeta_{r,i} dbeta_{r,i}/dg_i + G_r dM_r/dg_i
 * with beta = min(1, |a_i|/L_i + tanh x), x = pi^2 g^2 h^2, and
 * M = |F|^2 P DW, P = prod sech(2 x_i) (intensity model Hosemann).
 */
void or_chain_globals(const or_params *p, int32_t n_refl, const int32_t *hkl, const double *F2,
                      const double *G_refl, const double *dbeta, double *dL, double *dg) {
    double A[9], As[9];
    or_basis(p->cell, A, As);
    double alen[3] = {norm3(A), norm3(A + 3), norm3(A + 6)};
    int32_t nr = n_refl > 0 ? n_refl : 1;
    double *beta = malloc(sizeof(double) * 3 * nr), *Pv = malloc(sizeof(double) * nr), *DWv = malloc(sizeof(double) * nr);
    or_refl_scalars(p, n_refl, hkl, beta, Pv, DWv);
    for (int i = 0; i < 3; i++) {
        dL[i] = 0.0;
        dg[i] = 0.0;
    }
    for (int32_t r = 0; r < n_refl; r++) {
        for (int i = 0; i < 3; i++) {
            double hi = (double)hkl[3 * r + i];
            double x = OR_PI * OR_PI * p->g[i] * p->g[i] * hi * hi;
            double braw = alen[i] / p->L[i] + tanh(x);
            int clamped = braw >= 1.0;
            if (!clamped) {
                dL[i] += dbeta[3 * r + i] * (-alen[i] / (p->L[i] * p->L[i]));
                double sech = 1.0 / cosh(x);
                dg[i] += dbeta[3 * r + i] * sech * sech * 2.0 * OR_PI * OR_PI * p->g[i] * hi * hi;
            }
            if (p->intensity_model == 1) {
                double dP = -Pv[r] * tanh(2.0 * x) * 4.0 * OR_PI * OR_PI * p->g[i] * hi * hi;
                dg[i] += G_refl[r] * F2[r] * DWv[r] * dP;
            }
        }
    }
    free(beta); free(Pv); free(DWv);
}

/*
 * Structure-factor adjoint: given Gw[r] = dLoss/dM_r * P_r * DW_r and F,
 * dLoss/dx_{j,c} = sum_r Gw_r 2 Re(conj(F_r) dF_r/dx_{j,c}),
 *   dF/dx_{j,c} = 2 pi i h_c occ_j f_j(s) exp(-B_j s^2/4) exp(2 pi i h.x_j)
 * dLoss/dB_j = sum_r Gw_r 2 Re(conj(F_r) (-s^2/4) T_j).
 * Coordinates are fractional.
 */
void or_sf_adjoint(const double cell[6], int32_t n_atoms, const double *frac, const double *B, const double *occ,
                   const int32_t *elem, const double *ff, int32_t n_refl, const int32_t *hkl, const double *F,
                   const double *Gw, double *dfrac, double *dB) {
    double A[9], As[9];
    or_basis(cell, A, As);
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t j = 0; j < n_atoms; j++) {
        double gx = 0.0, gy = 0.0, gz = 0.0, gb = 0.0;
        for (int32_t r = 0; r < n_refl; r++) {
            if (Gw[r] == 0.0) continue;
            int h = hkl[3 * r], k = hkl[3 * r + 1], l = hkl[3 * r + 2];
            double D[3];
            recip_vector(As, h, k, l, D);
            double s2 = dot3(D, D);
            double amp = occ[j] * form_factor(ff + 9 * elem[j], s2) * exp(-B[j] * s2 / 4.0);
            double ph = h * frac[3 * j] + k * frac[3 * j + 1] + l * frac[3 * j + 2];
            ph -= nearbyint(ph);
            double tr = amp * cos(2.0 * OR_PI * ph), ti = amp * sin(2.0 * OR_PI * ph);
            /* conj(F) * T */
            double cr = F[2 * r] * tr + F[2 * r + 1] * ti;
            double ci = F[2 * r] * ti - F[2 * r + 1] * tr;
            /* 2 Re(conj(F) * 2 pi i h_c T) = -4 pi h_c Im(conj(F) T) */
            double base = -4.0 * OR_PI * ci * Gw[r];
            gx += base * h;
            gy += base * k;
            gz += base * l;
            gb += Gw[r] * 2.0 * cr * (-s2 / 4.0);
        }
        dfrac[3 * j] = gx;
        dfrac[3 * j + 1] = gy;
        dfrac[3 * j + 2] = gz;
        dB[j] = gb;
    }
}

int32_t or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int32_t n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
