// FP32 evaluation of phi_kappa for one point pair with the body-pair phase
// split (shared by the FP32 G_hat kernels).
//
// Coordinates are x_hat = c_tau + delta with small local offsets delta.  Per
// body pair (tau, sigma) a table holds D = c_tau - c_sigma, R = |D| and the
// phase (kappa R + const) mod 2 pi, computed once in FP64.  Per point pair,
// with d = delta_i - delta_j,
//     s = 2 D.d + |d|^2,  r^2 = R^2 + s,  r - R = s / (r + R),
// so the phase kappa r = kappa R + kappa (r - R) keeps FP32 accuracy even when
// kappa r is in the thousands.
#pragma once

#include "bessel.cuh"
#include "common.cuh"

struct F32Const {
    float kappa;  // wavenumber
    float ampc;   // (1/4) sqrt(2 / (pi kappa))
    float c8;     // 2 * 8 / kappa  (u = c8 / r - 1 for the x >= 8 fit)
    float c3;     // 2 * 3 / kappa
    float c64;    // 2 * 64 / kappa (the x >= 64 fit)
    // modulus fits with the amplitude constant ampc folded in; a kernel takes
    // F32Const by value, so these sit in its parameter space (constant bank)
    // and multiply-adds read them without registers
    float f8a[MBS_F32_X8_DEG + 1];
    float f64a[MBS_F32_X64_DEG + 1];
};

inline F32Const make_f32const(double kappa) {
    F32Const K;
    K.kappa = (float)kappa;
    K.ampc = (float)(0.25 * sqrt(2.0 / (MBS_PI * kappa)));
    K.c8 = (float)(2.0 * MBS_F32_X8_XA / kappa);
    K.c3 = (float)(2.0 * MBS_F32_X3_XA / kappa);
    K.c64 = (float)(2.0 * MBS_F32_X64_XA / kappa);
    const float f8[] = MBS_F32_X8_F, f64[] = MBS_F32_X64_F;
    for (int k = 0; k <= MBS_F32_X8_DEG; ++k) K.f8a[k] = f8[k] * K.ampc;
    for (int k = 0; k <= MBS_F32_X64_DEG; ++k) K.f64a[k] = f64[k] * K.ampc;
    return K;
}

// exp(i ph) reduced to [-pi, pi] by one Cody-Waite step with the FP32 value
// of 2 pi.  The constant's error, 1.7e-7, times n = ph / 2 pi adds at most
// 2.8e-8 |ph| to the reduced phase: below the FP32 rounding of ph itself
// (up to 6e-8 |ph|), so a second, exact-split constant buys no accuracy.
__device__ __forceinline__ float2 expi_f32(float ph) {
    // n = nearest integer to ph / (2 pi), by adding and removing 1.5 * 2^23
    // (exact for |ph / 2 pi| < 2^22; keeps the rounding off the XU pipe)
    const float n = fmaf(ph, 0.159154943091895336f, 12582912.f) - 12582912.f;
    ph = fmaf(-n, 6.28318530717958648f, ph);
    float sn, cs;
    __sincosf(ph, &sn, &cs);
    return make_float2(cs, sn);
}

// (i/4) H0(kappa r) for kappa r >= XA from the modulus/phase fit, with the
// phase kappa r + pi/4 + g split as phi0 + kappa (r - R) + g.
template <int DEG>
__device__ __forceinline__ float2 far_phi_f32(const float* cf, const float* cg, float c2xa,
                                              float rinv, float r, float s, float R, float phi0,
                                              const F32Const& K) {
    const float dr = __fdividef(s, r + R);
    const float u = fmaf(c2xa, rinv, -1.f);
    const float f = horner_f32<DEG>(cf, u);
    const float g = horner_f32<DEG>(cg, u);
    const float2 e = expi_f32(phi0 + fmaf(K.kappa, dr, g));
    const float amp = K.ampc * f * rsqrtf(r);
    return make_float2(amp * e.x, amp * e.y);
}

// phi for one point pair in FP32 with the body-pair phase split.
// P = (Dx, Dy, R, phi0) in 2D, (Dx, Dy, Dz, R) in 3D (phi0 passed separately);
// R2 = R * R.  The caller never passes a pair of the same body.
template <int DIM, bool FAR>
__device__ __forceinline__ float2 pair_phi_f32(const float* di, const float* dj, const float4 P,
                                               const float R2, const float phi0,
                                               const F32Const& K) {
    const float dx = di[0] - dj[0];
    const float dy = di[1] - dj[1];
    float s, R;
    if (DIM == 2) {
        s = fmaf(fmaf(2.f, P.x, dx), dx, fmaf(2.f, P.y, dy) * dy);
        R = P.z;
    } else {
        const float dz = di[2] - dj[2];
        s = fmaf(fmaf(2.f, P.x, dx), dx, fmaf(fmaf(2.f, P.y, dy), dy, fmaf(2.f, P.z, dz) * dz));
        R = P.w;
    }
    const float r2 = R2 + s;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    if (DIM == 2) {
        if (FAR)  // every pair of this body pair has kappa r >= 8
            return far_phi_f32<MBS_F32_X8_DEG>(c_f32_8F, c_f32_8G, K.c8, rinv, r, s, R, P.w, K);
        const float x = K.kappa * r;
        if (x >= MBS_F32_X8_XA)
            return far_phi_f32<MBS_F32_X8_DEG>(c_f32_8F, c_f32_8G, K.c8, rinv, r, s, R, P.w, K);
        if (x >= MBS_F32_X3_XA)
            return far_phi_f32<MBS_F32_X3_DEG>(c_f32_F, c_f32_G, K.c3, rinv, r, s, R, P.w, K);
        return phi2d_small_f32(x);
    } else {
        const float dr = __fdividef(s, r + R);
        const float2 e = expi_f32(fmaf(K.kappa, dr, phi0));
        const float amp = 0.0795774715459476679f * rinv;  // 1 / (4 pi r)
        return make_float2(amp * e.x, amp * e.y);
    }
}

