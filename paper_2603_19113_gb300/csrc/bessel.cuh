// Device evaluation of the fundamental solution phi_kappa (Sec. 3.1, eq. FundamentalSol).
//
// 2D: phi = (i/4) H0^(1)(x), x = kappa r.  For x >= XA the Hankel function is
// written in modulus/phase form H0 = M exp(i theta) with
//     M(x) = sqrt(2 / (pi x)) f(x),   theta(x) = x - pi/4 + g(x)
// (Hankel's asymptotic form, DLMF 10.17.1 / 10.18), where f and g are smooth
// in t = XA / x and are evaluated from fitted polynomials (bessel_coeffs.h,
// written by gen_bessel_coeffs.py from high-precision J0 and Y0).  Then
//     phi = (M / 4) exp(i (theta + pi/2)) = (M / 4) exp(i (x + pi/4 + g)).
// For small x the power series of J0 and Y0 (DLMF 10.2.2, 10.8.2) are summed.
// 3D: phi = exp(i kappa r) / (4 pi r).
#pragma once

#include "bessel_coeffs.h"
#include "common.cuh"

__device__ __constant__ float c_f32_64F[MBS_F32_X64_DEG + 1] = MBS_F32_X64_F;
__device__ __constant__ float c_f32_64G[MBS_F32_X64_DEG + 1] = MBS_F32_X64_G;
__device__ __constant__ float c_f32_8F[MBS_F32_X8_DEG + 1] = MBS_F32_X8_F;
__device__ __constant__ float c_f32_8G[MBS_F32_X8_DEG + 1] = MBS_F32_X8_G;
__device__ __constant__ float c_f32_F[MBS_F32_X3_DEG + 1] = MBS_F32_X3_F;
__device__ __constant__ float c_f32_G[MBS_F32_X3_DEG + 1] = MBS_F32_X3_G;
__device__ __constant__ double c_f64_4F[MBS_F64_X4_DEG + 1] = MBS_F64_X4_F;
__device__ __constant__ double c_f64_4G[MBS_F64_X4_DEG + 1] = MBS_F64_X4_G;
__device__ __constant__ double c_f64_16F[MBS_F64_X16_DEG + 1] = MBS_F64_X16_F;
__device__ __constant__ double c_f64_16G[MBS_F64_X16_DEG + 1] = MBS_F64_X16_G;
__device__ __constant__ double c_f64_64F[MBS_F64_X64_DEG + 1] = MBS_F64_X64_F;
__device__ __constant__ double c_f64_64G[MBS_F64_X64_DEG + 1] = MBS_F64_X64_G;

template <int DEG>
__device__ __forceinline__ float horner_f32(const float* c, float u) {
    float r = c[0];
#pragma unroll
    for (int i = 1; i <= DEG; ++i) r = fmaf(r, u, c[i]);
    return r;
}

template <int DEG>
__device__ __forceinline__ double horner_f64(const double* c, double u) {
    double r = c[0];
#pragma unroll
    for (int i = 1; i <= DEG; ++i) r = fma(r, u, c[i]);
    return r;
}

// (i/4) H0(x) for 0 < x < 3 in FP32: power series of J0 and Y0.
//   J0 = sum_k (-y)^k / (k!)^2,  y = x^2 / 4
//   Y0 = (2/pi) [ (ln(x/2) + gamma) J0 - sum_{k>=1} H_k (-y)^k / (k!)^2 ]
__device__ __forceinline__ float2 phi2d_small_f32(float x) {
    const float y = 0.25f * x * x;
    float term = 1.f, J = 1.f, S = 0.f, H = 0.f;
#pragma unroll
    for (int k = 1; k <= 11; ++k) {
        term *= -y / (float)(k * k);
        H += 1.f / (float)k;
        J += term;
        S = fmaf(H, term, S);
    }
    const float Y = 0.63661977236758134f * ((logf(0.5f * x) + 0.57721566490153286f) * J - S);
    return make_float2(-0.25f * Y, 0.25f * J);
}

// (i/4) H0(x) for x > 0 in FP64.
__device__ __forceinline__ double2 phi2d_f64(double x) {
    double f, g;
    if (x >= MBS_F64_X16_XA) {
        const double u = 2.0 * MBS_F64_X16_XA / x - 1.0;
        f = horner_f64<MBS_F64_X16_DEG>(c_f64_16F, u);
        g = horner_f64<MBS_F64_X16_DEG>(c_f64_16G, u);
    } else if (x >= MBS_F64_X4_XA) {
        const double u = 2.0 * MBS_F64_X4_XA / x - 1.0;
        f = horner_f64<MBS_F64_X4_DEG>(c_f64_4F, u);
        g = horner_f64<MBS_F64_X4_DEG>(c_f64_4G, u);
    } else {
        const double y = 0.25 * x * x;
        double term = 1.0, J = 1.0, S = 0.0, H = 0.0;
#pragma unroll
        for (int k = 1; k <= 20; ++k) {
            term *= -y / (double)(k * k);
            H += 1.0 / (double)k;
            J += term;
            S = fma(H, term, S);
        }
        const double Y = (2.0 / MBS_PI) * ((log(0.5 * x) + MBS_EULER_GAMMA) * J - S);
        return make_double2(-0.25 * Y, 0.25 * J);
    }
    // 0.25 * sqrt(2/pi) = 0.19947114020071633
    const double amp = 0.19947114020071633 * f * rsqrt(x);
    double s, c;
    sincos(x + 0.25 * MBS_PI + g, &s, &c);
    return make_double2(amp * c, amp * s);
}

// (i/4) H0(kappa r) in FP64 from the squared distance r2 (the form the G_hat
// and field kernels use): one reciprocal square root gives 1/r for the fit
// variable u = 2 XA / x - 1 = (2 XA / kappa) / r, and r itself after one
// Newton step (r <- r + (r2 - r^2) / (2 r)), so the phase kappa r keeps the
// accuracy of a rounded square root without a division.  Fits: degree 6 for
// x >= 64, 10 for x >= 16, 20 for x >= 4, power series below.
__device__ __forceinline__ double2 phi2d_f64_r2(double kappa, double r2) {
    const double rinv = rsqrt(r2);
    double r = r2 * rinv;
    r = fma(0.5 * rinv, fma(-r, r, r2), r);
    const double x = kappa * r;
    double f, g;
    if (x >= MBS_F64_X64_XA) {
        const double u = (2.0 * MBS_F64_X64_XA / kappa) * rinv - 1.0;
        f = horner_f64<MBS_F64_X64_DEG>(c_f64_64F, u);
        g = horner_f64<MBS_F64_X64_DEG>(c_f64_64G, u);
    } else if (x >= MBS_F64_X16_XA) {
        const double u = (2.0 * MBS_F64_X16_XA / kappa) * rinv - 1.0;
        f = horner_f64<MBS_F64_X16_DEG>(c_f64_16F, u);
        g = horner_f64<MBS_F64_X16_DEG>(c_f64_16G, u);
    } else if (x >= MBS_F64_X4_XA) {
        const double u = (2.0 * MBS_F64_X4_XA / kappa) * rinv - 1.0;
        f = horner_f64<MBS_F64_X4_DEG>(c_f64_4F, u);
        g = horner_f64<MBS_F64_X4_DEG>(c_f64_4G, u);
    } else {
        return phi2d_f64(x);
    }
    // 0.25 * sqrt(2/pi) = 0.19947114020071633
    const double amp = 0.19947114020071633 * f * rsqrt(x);
    double s, c;
    sincos(x + 0.25 * MBS_PI + g, &s, &c);
    return make_double2(amp * c, amp * s);
}

// e^{i kappa r} / (4 pi r) from r2: 1/r by one reciprocal square root, r by
// one Newton step.
__device__ __forceinline__ double2 phi3d_f64_r2(double kappa, double r2) {
    const double rinv = rsqrt(r2);
    double r = r2 * rinv;
    r = fma(0.5 * rinv, fma(-r, r, r2), r);
    double s, c;
    sincos(kappa * r, &s, &c);
    const double a = rinv * (1.0 / (4.0 * MBS_PI));
    return make_double2(a * c, a * s);
}

template <int DIM>
__device__ __forceinline__ double2 phi_f64_r2(double kappa, double r2) {
    if (DIM == 2) return phi2d_f64_r2(kappa, r2);
    return phi3d_f64_r2(kappa, r2);
}

// phi in 3D at distance r, FP64.
__device__ __forceinline__ double2 phi3d_f64(double kappa, double r) {
    double s, c;
    sincos(kappa * r, &s, &c);
    const double a = 1.0 / (4.0 * MBS_PI * r);
    return make_double2(a * c, a * s);
}

template <int DIM>
__device__ __forceinline__ double2 phi_f64(double kappa, double r) {
    if (DIM == 2) return phi2d_f64(kappa * r);
    return phi3d_f64(kappa, r);
}
