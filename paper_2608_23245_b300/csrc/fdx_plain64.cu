// Plain FP64 form of the same method on the GPU: the comparison the
// refinement-throughput metric is quoted against.  Same work decomposition as
// the FP32 path (pixel-major gather for the pattern, reflection-major adjoint
// over detector bands, one thread per reflection or atom for the structure
// factors), but straightforward FP64 arithmetic: every (pixel, node) term in
// each pixel's projected-box node range is evaluated directly,
//   s_k = r0 (S^ + d1 e1 + d2 e2) / sqrt(1 + d1^2 + d2^2),  t_i = a_i . (p - s_k),
//   K_i = beta_i / (beta_i^2 + (1 - beta_i^2) sin^2(pi t_i)),
// with CUDA's FP64 sinpi/sincospi/exp, FP64 sums, and no staging, culling or
// float-float rewrites.  Hosemann lineshape only.
#include "fdx_adjoint.cuh"
#include "fdx_pair.cuh"

namespace fdx {

// Per-reflection FP64 record.
enum Rec64 {
    R64_D = 0, R64_R0 = 3, R64_SH = 4, R64_E1 = 7, R64_E2 = 10, R64_ER = 13,
    R64_LA = 16, R64_LB = 19, R64_TM = 22, R64_CR = 25 /* 4 x 3 corners, local frame / r0 */,
    R64_R2B = 37, R64_M = 38, R64_BETA = 39, R64_DBF = 42, R64_ZD = 45, R64_RD = 46, R64_SIZE = 48
};

__global__ void plain64_refl_kernel(Plain64Params p) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.n_refl) return;
    const int hk[3] = {p.hkl[3 * r], p.hkl[3 * r + 1], p.hkl[3 * r + 2]};
    double *o = p.recs64 + (size_t)r * R64_SIZE;
    double D[3];
    for (int q = 0; q < 3; ++q) D[q] = hk[0] * p.As[q] + hk[1] * p.As[3 + q] + hk[2] * p.As[6 + q];
    const double r0 = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    double Sh[3] = {D[0] / r0, D[1] / r0, D[2] / r0};
    double t[3] = {p.nh[1] * Sh[2] - p.nh[2] * Sh[1], p.nh[2] * Sh[0] - p.nh[0] * Sh[2], p.nh[0] * Sh[1] - p.nh[1] * Sh[0]};
    double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    if (tn < 1e-12) {
        t[0] = p.bh[1] * Sh[2] - p.bh[2] * Sh[1];
        t[1] = p.bh[2] * Sh[0] - p.bh[0] * Sh[2];
        t[2] = p.bh[0] * Sh[1] - p.bh[1] * Sh[0];
        tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    }
    const double e1[3] = {t[0] / tn, t[1] / tn, t[2] / tn};
    const double e2[3] = {Sh[1] * e1[2] - Sh[2] * e1[1], Sh[2] * e1[0] - Sh[0] * e1[2], Sh[0] * e1[1] - Sh[1] * e1[0]};
    const double ZD = D[0] * p.nh[0] + D[1] * p.nh[1] + D[2] * p.nh[2];
    double pr[3] = {D[0] - ZD * p.nh[0], D[1] - ZD * p.nh[1], D[2] - ZD * p.nh[2]};
    const double RD = sqrt(pr[0] * pr[0] + pr[1] * pr[1] + pr[2] * pr[2]);
    for (int q = 0; q < 3; ++q) {
        o[R64_D + q] = D[q], o[R64_SH + q] = Sh[q], o[R64_E1 + q] = e1[q], o[R64_E2 + q] = e2[q];
        o[R64_ER + q] = RD < 1e-12 * r0 ? e1[q] : pr[q] / RD;
    }
    o[R64_R0] = r0, o[R64_ZD] = ZD, o[R64_RD] = RD;
    double beta[3];
    for (int i = 0; i < 3; ++i) {
        const double x = FDX_PI * FDX_PI * p.g[i] * p.g[i] * (double)hk[i] * hk[i];
        const double b = p.alen[i] / p.L[i] + tanh(x);
        beta[i] = b < 1.0 ? b : 1.0;
        o[R64_LA + i] = beta[i] * beta[i], o[R64_LB + i] = 1.0 - beta[i] * beta[i], o[R64_TM + i] = 0.5;
        o[R64_BETA + i] = beta[i];
        o[R64_DBF + i] = beta[i] < 1.0 ? 2.0 * beta[i] / (1.0 - beta[i] * beta[i]) : 0.0;
    }
    const double *frame[3] = {Sh, e1, e2};
    for (int v = 0; v < 4; ++v) {
        const double sb = (v & 1) ? -1.0 : 1.0, sc = (v & 2) ? -1.0 : 1.0;
        double C[3];
        for (int q = 0; q < 3; ++q) C[q] = 0.5 * p.As[q] + sb * 0.5 * p.As[3 + q] + sc * 0.5 * p.As[6 + q];
        for (int q = 0; q < 3; ++q)
            o[R64_CR + 3 * v + q] = (C[0] * frame[q][0] + C[1] * frame[q][1] + C[2] * frame[q][2]) / r0;
    }
    o[R64_R2B] = r0 * r0 * beta[0] * beta[1] * beta[2];
    o[R64_M] = p.M64 ? p.M64[r] : 1.0;
}

// Node range of one pixel (projected support-box corners, as the FP32 path).
__device__ __forceinline__ void plain64_range(const Plain64Params &p, const double *rec, double R, double Z,
                                              bool valid, int &j0, int &j1, int &m0, int &m1) {
    const int n = p.n;
    j0 = n, j1 = -1, m0 = n, m1 = -1;
    if (!valid) return;
    double P[3];
    const double ZD = rec[R64_ZD], RD = rec[R64_RD];
    // p - D = (Z - Z_D) n + (R - R_D) e_R, in the local frame / r0
    for (int q = 0; q < 3; ++q) {
        const double *f = rec + (q == 0 ? R64_SH : (q == 1 ? R64_E1 : R64_E2));
        const double nf = p.nh[0] * f[0] + p.nh[1] * f[1] + p.nh[2] * f[2];
        const double ef = rec[R64_ER] * f[0] + rec[R64_ER + 1] * f[1] + rec[R64_ER + 2] * f[2];
        P[q] = ((Z - ZD) * nf + (R - RD) * ef) / rec[R64_R0];
    }
    double d1lo = 1e300, d1hi = -1e300, d2lo = 1e300, d2hi = -1e300;
    bool degenerate = false;
    for (int v = 0; v < 4; ++v)
        for (int s = 0; s < 2; ++s) {
            const double sg = s ? -1.0 : 1.0;
            const double X0 = 1.0 + P[0] + sg * rec[R64_CR + 3 * v];
            const double X1 = P[1] + sg * rec[R64_CR + 3 * v + 1], X2 = P[2] + sg * rec[R64_CR + 3 * v + 2];
            degenerate |= !(X0 > 0.05);
            d1lo = fmin(d1lo, X1 / X0), d1hi = fmax(d1hi, X1 / X0);
            d2lo = fmin(d2lo, X2 / X0), d2hi = fmax(d2hi, X2 / X0);
        }
    if (degenerate) {
        j0 = 0, j1 = n - 1, m0 = 0, m1 = n - 1;
        return;
    }
    j0 = max(0, (int)ceil((d1lo + p.T) / p.h - 0.5) - 1);
    j1 = min(n - 1, (int)floor((d1hi + p.T) / p.h - 0.5) + 1);
    m0 = max(0, (int)ceil((d2lo + p.T) / p.h - 0.5) - 1);
    m1 = min(n - 1, (int)floor((d2hi + p.T) / p.h - 0.5) + 1);
}

// Direct FP64 evaluation of one (pixel, node) term.  Returns false outside the
// support; K and dK products for the adjoint through the outputs.
struct Term64 {
    double kp;            // w prod K / prod beta = w / prod den
    double den;           // prod den
    double inv_den[3];
};

__device__ __forceinline__ bool plain64_term(const Plain64Params &p, const double *rec, const double *pq, int j, int m,
                                             Term64 &out) {
    const double d1 = -p.T + (j + 0.5) * p.h, d2 = -p.T + (m + 0.5) * p.h;
    const double c = 1.0 / sqrt(1.0 + d1 * d1 + d2 * d2);
    const double r0 = rec[R64_R0];
    double X[3];
    for (int q = 0; q < 3; ++q)
        X[q] = pq[q] - r0 * c * (rec[R64_SH + q] + d1 * rec[R64_E1 + q] + d2 * rec[R64_E2 + q]);
    double den = 1.0;
    for (int i = 0; i < 3; ++i) {
        const double ti = p.A[3 * i] * X[0] + p.A[3 * i + 1] * X[1] + p.A[3 * i + 2] * X[2];
        if (fabs(ti) > rec[R64_TM + i]) return false;
        const double s = sinpi(ti);
        const double di = rec[R64_LA + i] + rec[R64_LB + i] * s * s;
        out.inv_den[i] = 1.0 / di;
        den *= di;
    }
    out.den = den;
    out.kp = p.nodes64[4 * ((size_t)j * p.n + m)] / den;
    return true;
}

__global__ void __launch_bounds__(128) plain64_fwd_kernel(Plain64Params p) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px0 = blockIdx.x * 16 + (warp & 1) * 8, py0 = blockIdx.y * 8 + (warp >> 1) * 4;
    if (px0 >= p.nx || py0 >= p.ny) return;
    const int px = px0 + (lane & 7), py = py0 + (lane >> 3);
    const bool valid = px < p.nx && py < p.ny;
    const float4 g = p.pixgeo[valid ? (size_t)py * p.nx + px : (size_t)py0 * p.nx + px0];
    const double R = (double)g.x + (double)g.y, Z = (double)g.z + (double)g.w;
    const float rlen = sqrtf(g.x * g.x + g.z * g.z), psi = atan2f(g.x, g.z);
    const float rmin = warp_min(valid ? rlen : 3e38f), rmax = warp_max(valid ? rlen : -3e38f);
    const float pmin = warp_min(valid ? psi : 3e38f), pmax = warp_max(valid ? psi : -3e38f);
    double acc = 0.0;
    for (int base = 0; base < p.n_refl; base += 32) {
        bool cand = false;
        if (base + lane < p.n_refl) {
            const float4 q = p.reach[base + lane];
            cand = (q.x - q.y <= rmax) && (q.x + q.y >= rmin) && (q.z - q.w <= pmax) && (q.z + q.w >= pmin);
        }
        unsigned mask = __ballot_sync(FDX_FULL_MASK, cand);
        while (mask) {
            const int r = base + __ffs(mask) - 1;
            mask &= mask - 1;
            const double *rec = p.recs64 + (size_t)r * R64_SIZE;
            int j0, j1, m0, m1;
            plain64_range(p, rec, R, Z, valid, j0, j1, m0, m1);
            const int J0 = __reduce_min_sync(FDX_FULL_MASK, j0), J1 = __reduce_max_sync(FDX_FULL_MASK, j1);
            const int M0 = __reduce_min_sync(FDX_FULL_MASK, m0), M1 = __reduce_max_sync(FDX_FULL_MASK, m1);
            if (J0 > J1 || M0 > M1) continue;
            double pq[3];
            for (int q = 0; q < 3; ++q) pq[q] = Z * p.nh[q] + R * rec[R64_ER + q];
            double sum = 0.0;
            for (int j = J0; j <= J1; ++j)
                for (int m = M0; m <= M1; ++m) {
                    Term64 tt;
                    if (valid && plain64_term(p, rec, pq, j, m, tt)) sum += tt.kp;
                }
            acc += rec[R64_M] * rec[R64_R2B] * sum;
        }
    }
    if (valid) p.image64[(size_t)py * p.nx + px] = p.delta_L / (R + p.delta_L) * acc;
}

// Reflection-major adjoint: six sums per (reflection, band) item (layout of the FP32 path).
__global__ void __launch_bounds__(128) plain64_adj_kernel(Plain64Params p) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * 4 + warp;
    if (item >= (long long)p.n_refl * p.n_bands) return;
    const int r = (int)(item / p.n_bands), b = (int)(item % p.n_bands);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const float4 q = p.reach[r];
    const float4 bb = p.band_bounds[b];
    if ((q.x - q.y <= bb.y) && (q.x + q.y >= bb.x) && (q.z - q.w <= bb.w) && (q.z + q.w >= bb.z)) {
        const double *rec = p.recs64 + (size_t)r * R64_SIZE;
        const int pj0 = b * p.rows_per_band, pj1 = min(p.npy, pj0 + p.rows_per_band);
        const int np = (pj1 - pj0) * p.npx;
        for (int base = 0; base < np; base += 32) {
            bool cand = false;
            if (base + lane < np) {
                const float4 pb = p.patch_bounds[(size_t)pj0 * p.npx + base + lane];
                cand = (q.x - q.y <= pb.y) && (q.x + q.y >= pb.x) && (q.z - q.w <= pb.w) && (q.z + q.w >= pb.z);
            }
            unsigned mask = __ballot_sync(FDX_FULL_MASK, cand);
            while (mask) {
                const int pidx = pj0 * p.npx + base + __ffs(mask) - 1;
                mask &= mask - 1;
                const int px = 8 * (pidx % p.npx) + (lane & 7), py = 4 * (pidx / p.npx) + (lane >> 3);
                const bool valid = px < p.nx && py < p.ny;
                double R = 0.0, Z = 0.0, c = 0.0;
                if (valid) {
                    const float4 g = p.pixgeo[(size_t)py * p.nx + px];
                    R = (double)g.x + (double)g.y, Z = (double)g.z + (double)g.w;
                    c = (double)p.gI[(size_t)py * p.nx + px] * p.delta_L / (R + p.delta_L);
                }
                int j0, j1, m0, m1;
                plain64_range(p, rec, R, Z, valid && c != 0.0, j0, j1, m0, m1);
                const int J0 = __reduce_min_sync(FDX_FULL_MASK, j0), J1 = __reduce_max_sync(FDX_FULL_MASK, j1);
                const int M0 = __reduce_min_sync(FDX_FULL_MASK, m0), M1 = __reduce_max_sync(FDX_FULL_MASK, m1);
                if (J0 > J1 || M0 > M1) continue;
                double pq[3];
                for (int k = 0; k < 3; ++k) pq[k] = Z * p.nh[k] + R * rec[R64_ER + k];
                double s[6] = {0, 0, 0, 0, 0, 0};
                for (int j = J0; j <= J1; ++j)
                    for (int m = M0; m <= M1; ++m) {
                        Term64 tt;
                        if (!(valid && c != 0.0 && plain64_term(p, rec, pq, j, m, tt))) continue;
                        const double *nd = p.nodes64 + 4 * ((size_t)j * p.n + m);  // w, -, dw/dsigma, dw/dgamma
                        s[0] += tt.kp;
                        for (int i = 0; i < 3; ++i) s[1 + i] += tt.kp * (tt.inv_den[i] - 1.0);
                        s[4] += nd[2] / tt.den;
                        s[5] += nd[3] / tt.den;
                    }
                for (int k = 0; k < 6; ++k) acc[k] += warp_sum_d(c * s[k]);
            }
        }
    }
    if (lane == 0)
        for (int k = 0; k < 6; ++k) p.item_out[item * 6 + k] = acc[k];
}

// Per reflection: bands -> dL/dM, dbeta, dsigma, dgamma; chain to L, g; SF adjoint coefficient.
__global__ void plain64_refl_adj_kernel(Plain64Params p) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.n_refl) return;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < p.n_bands; ++b)
        for (int k = 0; k < 6; ++k) s[k] += p.item_out[((size_t)r * p.n_bands + b) * 6 + k];
    const double *rec = p.recs64 + (size_t)r * R64_SIZE;
    const double r2b = rec[R64_R2B], M = rec[R64_M];
    const double G = r2b * s[0];
    double P = 1.0, dw = 0.0, x[3];
    int hk[3];
    for (int i = 0; i < 3; ++i) {
        hk[i] = p.hkl[3 * r + i];
        x[i] = FDX_PI * FDX_PI * p.g[i] * p.g[i] * (double)hk[i] * hk[i];
        if (p.intensity_model == FDX_INTENSITY_HOSEMANN) P *= 1.0 / cosh(2.0 * x[i]);
        const double sa = hk[i] / p.alen[i];
        dw += p.Bax[i] * sa * sa;
    }
    const double DW = exp(-0.25 * dw);
    const double Fr = p.F64[2 * r], Fi = p.F64[2 * r + 1];
    double *o = p.refl_out + (size_t)r * 8;
    for (int i = 0; i < 3; ++i) {
        const double dbeta = M * r2b * (s[0] / rec[R64_BETA + i] - rec[R64_DBF + i] * s[1 + i]);
        const double braw = p.alen[i] / p.L[i] + tanh(x[i]);
        double dLi = 0.0, dgi = 0.0;
        if (braw < 1.0) {
            dLi = dbeta * (-p.alen[i] / (p.L[i] * p.L[i]));
            const double sh = 1.0 / cosh(x[i]);
            dgi = dbeta * sh * sh * 2.0 * FDX_PI * FDX_PI * p.g[i] * (double)hk[i] * hk[i];
        }
        if (p.intensity_model == FDX_INTENSITY_HOSEMANN)
            dgi += G * (Fr * Fr + Fi * Fi) * DW * (-P * tanh(2.0 * x[i]) * 4.0 * FDX_PI * FDX_PI * p.g[i] * (double)hk[i] * hk[i]);
        o[i] = dLi, o[3 + i] = dgi;
    }
    o[6] = M * r2b * s[4];
    o[7] = M * r2b * s[5];
    p.Gw64[r] = G * P * DW;
}

// FP64 structure factors: one thread per reflection, all atoms.
__global__ void plain64_sf_kernel(Plain64Params p) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.n_refl) return;
    const int h = p.hkl[3 * r], k = p.hkl[3 * r + 1], l = p.hkl[3 * r + 2];
    double D[3];
    for (int q = 0; q < 3; ++q) D[q] = h * p.As[q] + k * p.As[3 + q] + l * p.As[6 + q];
    const double s2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    double fe[64];
    for (int e = 0; e < p.n_elem; ++e) {
        const float *f = p.ff + 9 * e;
        double v = f[8];
        for (int i = 0; i < 4; ++i) v += (double)f[i] * exp(-(double)f[4 + i] * s2 * 0.25);
        fe[e] = v;
    }
    double re = 0.0, im = 0.0;
    for (int j = 0; j < p.n_atoms; ++j) {
        const double occ = p.occ ? (double)p.occ[j] : 1.0;
        const double amp = occ * fe[p.elem[j] < p.n_elem ? p.elem[j] : 0] * exp(-(double)p.B[j] * s2 * 0.25);
        const double ph = h * p.frac[3 * j] + k * p.frac[3 * j + 1] + l * p.frac[3 * j + 2];
        double sn, cs;
        sincospi(2.0 * (ph - rint(ph)), &sn, &cs);
        re += amp * cs, im += amp * sn;
    }
    p.F64[2 * r] = re, p.F64[2 * r + 1] = im;
    double P = 1.0, dw = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double hi = (double)p.hkl[3 * r + i];
        const double x = FDX_PI * FDX_PI * p.g[i] * p.g[i] * hi * hi;
        if (p.intensity_model == FDX_INTENSITY_HOSEMANN) P *= 1.0 / cosh(2.0 * x);
        const double sa = hi / p.alen[i];
        dw += p.Bax[i] * sa * sa;
    }
    p.M64[r] = (re * re + im * im) * P * exp(-0.25 * dw);
}

// FP64 structure-factor adjoint: one thread per atom, all reflections.
__global__ void plain64_sf_adj_kernel(Plain64Params p) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.n_atoms) return;
    const double occ = p.occ ? (double)p.occ[j] : 1.0;
    const int e = p.elem[j] < p.n_elem ? p.elem[j] : 0;
    double gx = 0, gy = 0, gz = 0, gb = 0;
    for (int r = 0; r < p.n_refl; ++r) {
        const double Gw = p.Gw64[r];
        if (Gw == 0.0) continue;
        const int h = p.hkl[3 * r], k = p.hkl[3 * r + 1], l = p.hkl[3 * r + 2];
        double D[3];
        for (int q = 0; q < 3; ++q) D[q] = h * p.As[q] + k * p.As[3 + q] + l * p.As[6 + q];
        const double s2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
        const float *f = p.ff + 9 * e;
        double fv = f[8];
        for (int i = 0; i < 4; ++i) fv += (double)f[i] * exp(-(double)f[4 + i] * s2 * 0.25);
        const double amp = occ * fv * exp(-(double)p.B[j] * s2 * 0.25);
        const double ph = h * p.frac[3 * j] + k * p.frac[3 * j + 1] + l * p.frac[3 * j + 2];
        double sn, cs;
        sincospi(2.0 * (ph - rint(ph)), &sn, &cs);
        const double tr = amp * cs, ti = amp * sn;
        const double Fr = p.F64[2 * r], Fi = p.F64[2 * r + 1];
        const double cr = Fr * tr + Fi * ti, ci = Fr * ti - Fi * tr;  // conj(F) T
        const double base = -4.0 * FDX_PI * ci * Gw;
        gx += base * h, gy += base * k, gz += base * l;
        gb += Gw * 2.0 * cr * (-s2 / 4.0);
    }
    if (p.dfrac) p.dfrac[3 * j] = gx, p.dfrac[3 * j + 1] = gy, p.dfrac[3 * j + 2] = gz;
    if (p.dB) p.dB[j] = gb;
}

// FP64 loss L = sum m (I - I_t)^2 / (I_t + 1) and dL/dI (fixed-order reduction).
__global__ void plain64_loss_kernel(Plain64Params p) {
    __shared__ double red[256];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)p.nx * p.ny;
    double v = 0.0;
    if (i < n) {
        const double It = p.It64[i], m = p.mask ? (double)p.mask[i] : 1.0;
        const double w = m / (It + 1.0), d = p.image64[i] - It;
        v = w * d * d;
        p.gI[i] = 2.0 * w * d;
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) p.loss_partial[blockIdx.x] = red[0];
}

__global__ void plain64_loss_final_kernel(Plain64Params p, int nb) {
    __shared__ double red[256];
    double v = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) v += p.loss_partial[k];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *p.loss = red[0];
}

cudaError_t launch_plain64_loss(Plain64Params &p, cudaStream_t s) {
    const long long n = (long long)p.nx * p.ny;
    const int nb = (int)((n + 255) / 256);
    plain64_loss_kernel<<<nb, 256, 0, s>>>(p);
    plain64_loss_final_kernel<<<1, 256, 0, s>>>(p, nb);
    return cudaGetLastError();
}

cudaError_t launch_plain64_forward(Plain64Params &p, cudaStream_t s) {
    if (p.n_refl > 0) {
        plain64_sf_kernel<<<(p.n_refl + 127) / 128, 128, 0, s>>>(p);
        plain64_refl_kernel<<<(p.n_refl + 127) / 128, 128, 0, s>>>(p);
    }
    dim3 grid((p.nx + 15) / 16, (p.ny + 7) / 8);
    plain64_fwd_kernel<<<grid, 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_plain64_backward(Plain64Params &p, AdjParams &A, cudaStream_t s) {
    // patch and band bounds and the global reduction are shared with the FP32 path
    launch_bounds_only(A, s);
    if (p.n_refl > 0) {
        const long long items = (long long)p.n_refl * p.n_bands;
        plain64_adj_kernel<<<(unsigned)((items + 3) / 4), 128, 0, s>>>(p);
        plain64_refl_adj_kernel<<<(p.n_refl + 127) / 128, 128, 0, s>>>(p);
    }
    launch_globals_only(A, s);
    if (p.n_refl > 0 && (p.dfrac || p.dB)) plain64_sf_adj_kernel<<<(p.n_atoms + 127) / 128, 128, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fdx
