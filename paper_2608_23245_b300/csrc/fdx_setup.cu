// Set-up kernels of the pattern path: detector pixel geometry, shell-node
// table with angular weights, and per-reflection records.  All three run in
// FP64 once per problem and round their results to float or float-float
// pairs, so the hot loop can stay in FP32.
#include <math.h>
#include <mutex>

#include "fdx_internal.cuh"

namespace fdx {

// ---------------------------------------------------------------------------
// Cell -> real and reciprocal basis (Eq. recip_basis), in the frame of Sect.
// "Unit cell and reciprocal-space frame": c along z, b in the yz-plane.
// ---------------------------------------------------------------------------
void cell_basis(const fdx_cell &c, double A[9], double As[9]) {
    const double ca = cos(c.alpha), cb = cos(c.beta), cg = cos(c.gamma), sa = sin(c.alpha);
    double a[3], b[3], cc[3];
    cc[0] = 0.0, cc[1] = 0.0, cc[2] = c.c;
    b[0] = 0.0, b[1] = c.b * sa, b[2] = c.b * ca;
    a[2] = c.a * cb;
    a[1] = c.a * (cg - ca * cb) / sa;
    a[0] = sqrt(fmax(0.0, c.a * c.a - a[1] * a[1] - a[2] * a[2]));
    auto cross = [](const double *x, const double *y, double *z) {
        z[0] = x[1] * y[2] - x[2] * y[1];
        z[1] = x[2] * y[0] - x[0] * y[2];
        z[2] = x[0] * y[1] - x[1] * y[0];
    };
    double bc[3], ca_[3], ab[3];
    cross(b, cc, bc);
    cross(cc, a, ca_);
    cross(a, b, ab);
    const double V = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
    for (int k = 0; k < 3; ++k) {
        A[k] = a[k], A[3 + k] = b[k], A[6 + k] = cc[k];
        As[k] = bc[k] / V, As[3 + k] = ca_[k] / V, As[6 + k] = ab[k] / V;
    }
}

// ---------------------------------------------------------------------------
// Weideman (1994, SIAM J. Numer. Anal. 31, 1497) coefficients:
//   a_n = (1/2M) sum_{k=-M}^{M-1} f(theta_k) cos(n theta_k),
//   theta_k = k pi / M, f(theta) = exp(-t^2) (L^2 + t^2), t = L tan(theta/2),
//   M = 2N, L = sqrt(N / sqrt 2).   (f(-pi) = 0.)
// ---------------------------------------------------------------------------
const WeidemanCoeffs &weideman_coeffs() {
    static WeidemanCoeffs wc;
    static std::once_flag once;
    std::call_once(once, [] {
        const int N = FDX_WEIDEMAN_N, M = 2 * N;
        const double L = sqrt(N / sqrt(2.0));
        wc.L = L;
        for (int n = 1; n <= N; ++n) {
            double s = 0.0;
            for (int k = -M + 1; k <= M - 1; ++k) {
                const double th = k * FDX_PI / M;
                const double t = L * tan(0.5 * th);
                s += exp(-t * t) * (L * L + t * t) * cos(n * th);
            }
            wc.a[n - 1] = s / (2.0 * M);
        }
    });
    return wc;
}

// w(z) for z = x + i y, y >= 0, as (re, im).  L - i z = (L + y) - i x ;
// L + i z = (L - y) + i x.
__device__ void faddeeva(double x, double y, const WeidemanCoeffs &wc, double &wr, double &wi) {
    const double L = wc.L;
    const double dr = L + y, di = -x;  // den = L - i z
    const double nr = L - y, ni = x;   // num = L + i z
    const double dd = dr * dr + di * di;
    const double Zr = (nr * dr + ni * di) / dd, Zi = (ni * dr - nr * di) / dd;
    double pr = wc.a[FDX_WEIDEMAN_N - 1], pi = 0.0;
    for (int k = FDX_WEIDEMAN_N - 2; k >= 0; --k) {
        const double tr = pr * Zr - pi * Zi + wc.a[k];
        pi = pr * Zi + pi * Zr;
        pr = tr;
    }
    // 2 p / den^2 + 1 / (sqrt(pi) den)
    const double d2r = dr * dr - di * di, d2i = 2.0 * dr * di;
    const double d2d = d2r * d2r + d2i * d2i;
    const double t1r = 2.0 * (pr * d2r + pi * d2i) / d2d, t1i = 2.0 * (pi * d2r - pr * d2i) / d2d;
    const double isp = 1.0 / sqrt(FDX_PI);
    wr = t1r + isp * dr / dd;
    wi = t1i - isp * di / dd;
}

// Angular shape g(Delta; sigma, gamma), g(0) = 1 (Sect. "Angular peak shapes"),
// and its derivatives.  Voigt: g = Re w(z)/Re w(z0), z = (Delta + i gamma)/(sigma sqrt 2),
// z0 = i gamma/(sigma sqrt 2); w'(z) = -2 z w(z) + 2i/sqrt(pi), dz/dsigma = -z/sigma,
// dz/dgamma = i/(sigma sqrt 2).  The pure-Gaussian branch has no gamma derivative.
__device__ double angular_shape(double D, double sigma, double gamma, const WeidemanCoeffs &wc, double &dgs,
                                double &dgg) {
    if (gamma == 0.0) {
        const double g = exp(-D * D / (2.0 * sigma * sigma));
        dgs = g * D * D / (sigma * sigma * sigma);
        dgg = 0.0;
        return g;
    }
    if (sigma < 1e-12) {
        const double den = D * D + gamma * gamma;
        dgs = 0.0;
        dgg = 2.0 * gamma * D * D / (den * den);
        return gamma * gamma / den;
    }
    const double s = 1.0 / (sigma * sqrt(2.0));
    double w1r, w1i, w0r, w0i;
    const double x1 = D * s, y = gamma * s;
    faddeeva(x1, y, wc, w1r, w1i);
    faddeeva(0.0, y, wc, w0r, w0i);
    const double c2 = 2.0 / sqrt(FDX_PI);
    // w' = -2 z w + 2i/sqrt(pi)
    const double d1r = -2.0 * (x1 * w1r - y * w1i), d1i = -2.0 * (x1 * w1i + y * w1r) + c2;
    const double d0r = -2.0 * (0.0 * w0r - y * w0i), d0i = -2.0 * (0.0 * w0i + y * w0r) + c2;
    // d Re w / dsigma = Re(w' * (-z/sigma)); d Re w / dgamma = Re(w' * i s) = -s Im w'
    const double a1s = -(d1r * x1 - d1i * y) / sigma, a0s = -(d0r * 0.0 - d0i * y) / sigma;
    const double a1g = -s * d1i, a0g = -s * d0i;
    dgs = (a1s * w0r - w1r * a0s) / (w0r * w0r);
    dgg = (a1g * w0r - w1r * a0g) / (w0r * w0r);
    return w1r / w0r;
}

// ---------------------------------------------------------------------------
// Pixel geometry: pixel -> S on the Ewald sphere (Eq. laue) -> (R, Z).
// S = r/(lambda |r|) - b/lambda with r = SF b + u u^ + v v^.  SF/|r| - 1 is
// written as -(u^2+v^2)/(|r|(|r|+SF)) to avoid cancellation near the beam.
// ---------------------------------------------------------------------------
__global__ void pixel_geometry_kernel(PixelParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const double u = (i + 0.5 - 0.5 * p.nx) * p.pix;
    const double v = (j + 0.5 - 0.5 * p.ny) * p.pix;
    const double rho2 = u * u + v * v;
    const double rn = sqrt(p.dist * p.dist + rho2);
    const double fb = -rho2 / (rn * (rn + p.dist));
    double S[3];
    for (int q = 0; q < 3; ++q) S[q] = (fb * p.bh[q] + (u * p.uh[q] + v * p.vh[q]) / rn) / p.lambda;
    const double Z = S[0] * p.nh[0] + S[1] * p.nh[1] + S[2] * p.nh[2];
    double pr[3];
    for (int q = 0; q < 3; ++q) pr[q] = S[q] - Z * p.nh[q];
    const double R = sqrt(pr[0] * pr[0] + pr[1] * pr[1] + pr[2] * pr[2]);
    float4 o;
    split_double(R, o.x, o.y);
    split_double(Z, o.z, o.w);
    p.pixgeo[(size_t)j * p.nx + i] = o;
}

// ---------------------------------------------------------------------------
// Shell nodes (Eq. gnomonic) on the n x n midpoint grid d = -T + (j + 1/2) h
// and weights (Eq. node_weight):
//   w = sigma_r sqrt(2 pi) g(Delta) (1 + d1^2 + d2^2)^(-3/2) h^2,
//   Delta = arccos((1 + d^2)^(-1/2)) = atan |d|.
// Stored: c - 1, c d1, c d2 as float-float (c = (1 + d^2)^(-1/2)) and w.
// c - 1 = -rho^2 / (q (1 + q)), q = sqrt(1 + rho^2), without cancellation.
// ---------------------------------------------------------------------------
__global__ void nodes_kernel(NodeParams p, WeidemanCoeffs wc) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (m >= p.n) return;
    const double d1 = -p.T + (j + 0.5) * p.h, d2 = -p.T + (m + 0.5) * p.h;
    const double rho2 = d1 * d1 + d2 * d2;
    const double q = sqrt(1.0 + rho2), c = 1.0 / q;
    const double cm1 = -rho2 / (q * (1.0 + q));
    const double Delta = atan(sqrt(rho2));
    double dgs, dgg;
    const double g = angular_shape(Delta, p.sigma, p.gamma, wc, dgs, dgg);
    const double pre = p.sigma_r * sqrt(2.0 * FDX_PI) * c * c * c * p.h * p.h;
    const double w = pre * g;
    float4 a, b;
    split_double(cm1, a.x, a.y);
    split_double(d1 * c, a.z, a.w);
    split_double(d2 * c, b.x, b.y);
    b.z = (float)w;
    b.w = 0.0f;
    const size_t k = (size_t)j * p.n + m;
    p.nodes[2 * k] = a;
    p.nodes[2 * k + 1] = b;
    if (p.dnodes) p.dnodes[k] = make_float2((float)(pre * dgs), (float)(pre * dgg));
    if (p.nodes64) {
        p.nodes64[4 * k] = w, p.nodes64[4 * k + 1] = c;
        p.nodes64[4 * k + 2] = pre * dgs, p.nodes64[4 * k + 3] = pre * dgg;
    }
}

// ---------------------------------------------------------------------------
// Per-reflection record (FP64 -> rounded once), see RecField.
// Disorder scalars (Eqs. Ah, breadth, Neff):  x_i = pi^2 g_i^2 h_i^2,
//   (1 - A)/(1 + A) = tanh x_i,  beta_i = min(1, |a_i|/L_i + tanh x_i).
// Reach (for the candidate test): a pixel can see reflection D only if
// | |p| - r0 | <= rho_B and its polar angle is within
//   dpsi = atan(T sqrt 2) + asin(rho_B / r0)
// of D's, rho_B being the circumradius of the support box.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dot3(const double *x, const double *y) {
    return x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
}

__global__ void refl_setup_kernel(ReflSetupParams p) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.n_refl) return;
    const int hk[3] = {p.hkl[3 * r], p.hkl[3 * r + 1], p.hkl[3 * r + 2]};
    double D[3];
    for (int q = 0; q < 3; ++q) D[q] = hk[0] * p.As[q] + hk[1] * p.As[3 + q] + hk[2] * p.As[6 + q];
    const double r0 = sqrt(dot3(D, D));
    double Sh[3] = {D[0] / r0, D[1] / r0, D[2] / r0};
    double t[3] = {p.nh[1] * Sh[2] - p.nh[2] * Sh[1], p.nh[2] * Sh[0] - p.nh[0] * Sh[2],
                   p.nh[0] * Sh[1] - p.nh[1] * Sh[0]};
    double tn = sqrt(dot3(t, t));
    if (tn < 1e-12) {
        t[0] = p.bh[1] * Sh[2] - p.bh[2] * Sh[1];
        t[1] = p.bh[2] * Sh[0] - p.bh[0] * Sh[2];
        t[2] = p.bh[0] * Sh[1] - p.bh[1] * Sh[0];
        tn = sqrt(dot3(t, t));
    }
    const double e1[3] = {t[0] / tn, t[1] / tn, t[2] / tn};
    const double e2[3] = {Sh[1] * e1[2] - Sh[2] * e1[1], Sh[2] * e1[0] - Sh[0] * e1[2],
                          Sh[0] * e1[1] - Sh[1] * e1[0]};
    const double ZD = dot3(D, p.nh);
    double perp[3] = {D[0] - ZD * p.nh[0], D[1] - ZD * p.nh[1], D[2] - ZD * p.nh[2]};
    const double RD = sqrt(dot3(perp, perp));
    double eR[3];
    if (RD < 1e-12 * r0) {
        for (int q = 0; q < 3; ++q) eR[q] = e1[q];
    } else {
        for (int q = 0; q < 3; ++q) eR[q] = perp[q] / RD;
    }
    float *o = p.recs + (size_t)r * REC_SIZE;
    split_double(RD, o[REC_RD], o[REC_RD + 1]);
    split_double(ZD, o[REC_ZD], o[REC_ZD + 1]);
    const double *frame[3] = {Sh, e1, e2};
    for (int q = 0; q < 3; ++q) {
        split_double(dot3(p.nh, frame[q]) / r0, o[REC_NFR + q], o[REC_NFR + 3 + q]);
        split_double(dot3(eR, frame[q]) / r0, o[REC_EFR + q], o[REC_EFR + 3 + q]);
    }
    double beta[3], tm[3];
    for (int i = 0; i < 3; ++i) {
        const double *ai = p.A + 3 * i;
        o[REC_AR + i] = (float)dot3(ai, eR);
        o[REC_H + i] = (float)hk[i];
        o[REC_E1 + i] = (float)(r0 * dot3(ai, e1));
        o[REC_E2 + i] = (float)(r0 * dot3(ai, e2));
        const double x = FDX_PI * FDX_PI * p.g[i] * p.g[i] * (double)hk[i] * hk[i];
        const double b = p.alen[i] / p.L[i] + tanh(x);
        beta[i] = b < 1.0 ? b : 1.0;
        if (p.lineshape == FDX_LINESHAPE_HOSEMANN) {
            tm[i] = 0.5;
            o[REC_LA + i] = (float)(beta[i] * beta[i]);
            o[REC_LB + i] = (float)(1.0 - beta[i] * beta[i]);
        } else if (p.lineshape == FDX_LINESHAPE_GAUSS) {
            // K = exp(-pi t^2 / beta^2) / beta = 2^(-LA t^2) / beta
            tm[i] = fmin(p.K_z * beta[i], 0.5);
            o[REC_LA + i] = (float)(FDX_PI * 1.4426950408889634 / (beta[i] * beta[i]));
            o[REC_LB + i] = 0.0f;
        } else {
            tm[i] = fmin(p.K_z * beta[i], 0.5);
            o[REC_LA + i] = (float)(1.0 / beta[i]);
            o[REC_LB + i] = 0.0f;
        }
        o[REC_TM + i] = (float)tm[i];
    }
    double rhoB = 0.0;
    for (int v = 0; v < 4; ++v) {
        const double sb = (v & 1) ? -1.0 : 1.0, sc = (v & 2) ? -1.0 : 1.0;
        double C[3];
        for (int q = 0; q < 3; ++q) C[q] = tm[0] * p.As[q] + sb * tm[1] * p.As[3 + q] + sc * tm[2] * p.As[6 + q];
        rhoB = fmax(rhoB, sqrt(dot3(C, C)));
        for (int q = 0; q < 3; ++q) o[REC_CR + 3 * v + q] = (float)(dot3(C, frame[q]) / r0);
    }
    const double M = p.M ? (double)p.M[r] : 1.0;
    double fr = M * r0 * r0;
    if (p.lineshape == FDX_LINESHAPE_HOSEMANN) {
        fr *= beta[0] * beta[1] * beta[2];
    } else if (p.lineshape == FDX_LINESHAPE_GAUSS) {
        fr /= beta[0] * beta[1] * beta[2];
    } else {
        const double pi2 = FDX_PI * FDX_PI;
        fr *= (1.0 / beta[0]) * (1.0 / beta[1]) * (1.0 / beta[2]) / (pi2 * pi2 * pi2);
    }
    o[REC_FR] = (float)fr;
    for (int k = REC_FR + 1; k < REC_SIZE; ++k) o[k] = 0.0f;
    o[REC_R2B] = (float)(r0 * r0 * beta[0] * beta[1] * beta[2]);
    for (int i = 0; i < 3; ++i) {
        o[REC_AR0 + i] = (float)(p.alen[i] * r0);
        o[REC_SLB + i] = p.lineshape == FDX_LINESHAPE_HOSEMANN ? (float)sqrt(fmax(0.0, 1.0 - beta[i] * beta[i])) : 0.0f;
        o[REC_BETA + i] = (float)beta[i];
        o[REC_DBF + i] = beta[i] < 1.0 ? (float)(2.0 * beta[i] / (1.0 - beta[i] * beta[i])) : 0.0f;
    }
    o[REC_M] = (float)M;
    if (p.ring) {
        // ring-average record (Eq. cyl-average; azimuth rule of reading R21)
        float *g = p.ring + (size_t)r * RING_REC;
        const double eP[3] = {p.nh[1] * eR[2] - p.nh[2] * eR[1], p.nh[2] * eR[0] - p.nh[0] * eR[2],
                              p.nh[0] * eR[1] - p.nh[1] * eR[0]};
        for (int q = 0; q < 3; ++q) split_double(dot3(eP, frame[q]) / r0, g[RING_TFR + q], g[RING_TFR + 3 + q]);
        double w_min = 1e300;
        for (int i = 0; i < 3; ++i) {
            g[RING_AT + i] = (float)dot3(p.A + 3 * i, eP);
            w_min = fmin(w_min, beta[i] / p.alen3[i]);
        }
        const double rt = rhoB + sqrt(2.0) * r0 * p.T;
        double ph = FDX_PI;
        const double inner = RD - rt;
        if (inner > 0.0) {
            const double x = rt / (2.0 * sqrt(inner * RD));
            if (x < 1.0) ph = 2.0 * asin(x);
        }
        double nr = ceil(2.0 * ph / (w_min / (4.0 * (RD + rt))));
        if (!(nr >= 4.0)) nr = 4.0;
        if (nr > (double)p.ring_max_n) nr = (double)p.ring_max_n;
        split_double(ph, g[RING_PHI], g[RING_PHI + 1]);
        g[RING_N] = (float)nr;
        g[RING_HW] = (float)(2.0 * ph / nr / (2.0 * FDX_PI));
        g[RING_RT] = (float)rt;
        g[14] = g[15] = 0.0f;
    }
    if (p.frames) {
        double *fr64 = p.frames + (size_t)r * 12;
        for (int q = 0; q < 3; ++q) fr64[q] = Sh[q], fr64[3 + q] = e1[q], fr64[6 + q] = e2[q];
        fr64[9] = r0, fr64[10] = rhoB, fr64[11] = 0.0;
    }
    // Polar-angle window of the pixels this reflection can reach.  A pixel's
    // query point p lies in the reflection's meridional plane (spanned by S^
    // and e2, reading R12); a node s = r0 (S^ + d1 e1 + d2 e2)/sqrt(1 + d^2)
    // contributes only if |p - s| <= rho_B, and so does its projection onto
    // that plane, which sits at the in-plane angle atan(d2) from S^ (|d2| <= T)
    // and at radius >= r0 / sqrt(1 + T^2).  Hence |psi_p - psi_D| <= atan(T)
    // + asin(rho_B sqrt(1 + T^2) / r0).  (The ring average, whose query points
    // leave the plane, widens this by atan(T sqrt 2) - atan(T).)
    const double psiD = atan2(RD, ZD);
    const double rho_in = rhoB * sqrt(1.0 + p.T * p.T);
    const double dpsi = atan(p.T) + (rho_in < r0 ? asin(rho_in / r0) : FDX_PI);
    p.reach[r] = make_float4((float)r0, (float)(rhoB * (1.0 + 1e-4) + 1e-6), (float)psiD,
                             (float)(dpsi * (1.0 + 1e-4) + 1e-6));
}

cudaError_t launch_pixel_geometry(const PixelParams &p, cudaStream_t s) {
    dim3 grid((p.nx + 127) / 128, p.ny);
    pixel_geometry_kernel<<<grid, 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_nodes(const NodeParams &p, const WeidemanCoeffs &wc, cudaStream_t s) {
    dim3 grid((p.n + 63) / 64, p.n);
    nodes_kernel<<<grid, 64, 0, s>>>(p, wc);
    return cudaGetLastError();
}

cudaError_t launch_refl_setup(const ReflSetupParams &p, cudaStream_t s) {
    if (p.n_refl <= 0) return cudaSuccess;
    refl_setup_kernel<<<(p.n_refl + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fdx
