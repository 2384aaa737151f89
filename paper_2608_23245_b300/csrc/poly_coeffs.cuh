/* Generated by fit_poly.py (weighted least squares + Lawson iterations). */
#pragma once
/* sin(2 pi r) = r * S(r^2), |r| <= 1/8; max rel err 3.24e-09 */
#define FDX_SIN2PI_C {6.283185287e+00f, -4.134166145e+01f, 8.159235355e+01f, -7.539356270e+01f}
/* cos(2 pi r) = C(r^2), |r| <= 1/8; max abs err 4.74e-11 */
#define FDX_COS2PI_C {1.000000000e+00f, -1.973920865e+01f, 6.493931621e+01f, -8.544285212e+01f, 5.922040724e+01f}
/* sin(2 pi r) = r * SH(r^2), |r| <= 1/4; max rel err 5.31e-09 */
#define FDX_SIN2PI_H_C {6.283185274e+00f, -4.134167748e+01f, 8.160223124e+01f, -7.657499212e+01f, 3.971091765e+01f}
/* cos(2 pi r) = CH(r^2), |r| <= 1/4; max abs err 2.19e-10 */
#define FDX_COS2PI_H_C {9.999999998e-01f, -1.973920855e+01f, 6.493934663e+01f, -8.545357162e+01f, 6.014401505e+01f, -2.498223756e+01f}
/* sin^2(pi t) = t^2 * Q(t^2), |t| <= 1/2; max rel err 1.39e-08 */
#define FDX_SINPI2_C {9.869604264e+00f, -3.246966236e+01f, 4.272692743e+01f, -3.009855317e+01f, 1.303711163e+01f, -3.336210712e+00f}
