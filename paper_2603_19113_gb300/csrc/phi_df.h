// The fundamental solution phi_kappa (Sec. 3.1, eq. FundamentalSol) in
// double-float arithmetic (dfloat.h) on the FP32 pipe, for FP64-accurate
// residuals without the FP64 pipe.  Host and device code.
//
// Phase accuracy: a double-float carries ~48 bits, so kappa r itself would
// lose 2e-11 rad at kappa r ~ 6000.  The phase is therefore split per body
// pair as for the FP32 kernels: with D = c_tau - c_sigma, R = |D| and the
// point-pair offset delta, s = r^2 - R^2 = 2 D.delta + |delta|^2 is small,
// r - R = s / (r + R), and the phase is phi0 + kappa (r - R) with phi0 =
// kappa R (3D) or kappa R + pi/4 (2D) reduced mod 2 pi on the host; every term
// then carries double-float accuracy relative to a small number.
#pragma once

#include "dfloat.h"

// pi / 2 as P1 + P2 + P3 + P4: the first three carry 12 significant bits, so
// n * Pk is exact for integers |n| < 2^12 (phases below 6434 rad); the sum
// is within 2e-21 of pi / 2.
#define DF_PIO2_1 0x1.922p+0f
#define DF_PIO2_2 -0x1.2aep-18f
#define DF_PIO2_3 -0x1.deap-31f
#define DF_PIO2_4 0x1.184698p-44f

DF_HD constexpr dfl df_const(double d) { return df_from_double(d); }

// sin and cos of a double-float angle |th| < 6434: Cody-Waite reduction by
// pi / 2 to |t| <= pi / 4, then the Taylor series of sin t = t + t^3 c(t^2)
// and cos t = 1 + t^2 d(t^2), their leading terms in double-float and the
// terms below 4e-8 in FP32 (truncation error below 2e-16).
DF_HD void df_sincos(dfl th, dfl& sn, dfl& cs) {
    const float nf = rintf(th.hi * 0.636619772367581343f);
    dfl t = df_add_f(th, -nf * DF_PIO2_1);
    t = df_add_f(t, -nf * DF_PIO2_2);
    t = df_add_f(t, -nf * DF_PIO2_3);
    t = df_add_f(t, -nf * DF_PIO2_4);
    const dfl t2 = df_mul(t, t);
    const float z = t2.hi;
    // c(z) = -1/3! + z/5! - z^2/7! + z^3/9! - z^4/11! + z^5/13! - z^6/15!
    float ts = fmaf(z, -1.0f / 1307674368000.0f, 1.0f / 6227020800.0f);
    ts = fmaf(z, ts, -1.0f / 39916800.0f);
    dfl c = df_add_f(df_const(1.0 / 362880.0), z * ts);
    c = df_fma(t2, c, df_const(-1.0 / 5040.0));
    c = df_fma(t2, c, df_const(1.0 / 120.0));
    c = df_fma(t2, c, df_const(-1.0 / 6.0));
    const dfl s = df_add(t, df_mul(df_mul(t2, t), c));
    // d(z) = -1/2! + z/4! - z^2/6! + z^3/8! - z^4/10! + z^5/12! - z^6/14! + z^7/16!
    float tc = fmaf(z, 1.0f / 20922789888000.0f, -1.0f / 87178291200.0f);
    tc = fmaf(z, tc, 1.0f / 479001600.0f);
    tc = fmaf(z, tc, -1.0f / 3628800.0f);
    dfl d = df_add_f(df_const(1.0 / 40320.0), z * tc);
    d = df_fma(t2, d, df_const(-1.0 / 720.0));
    d = df_fma(t2, d, df_const(1.0 / 24.0));
    d = df_fma(t2, d, df_const(-0.5));
    const dfl c0 = df_add_f(df_mul(t2, d), 1.0f);
    switch (((int)nf) & 3) {
        case 0: sn = s; cs = c0; break;
        case 1: sn = c0; cs = df_neg(s); break;
        case 2: sn = df_neg(s); cs = df_neg(c0); break;
        default: sn = df_neg(c0); cs = s; break;
    }
}

// 1 / sqrt(a), a > 0: FP32 estimate and one Newton step y (3 - a y^2) / 2
DF_HD dfl df_rsqrt(dfl a) {
    const float y = 1.0f / sqrtf(a.hi);
    const dfl e = df_add_f(df_neg(df_mul_f(df_mul_f(a, y), y)), 1.0f);  // 1 - a y^2
    return df_add_f(df_mul_f(e, 0.5f * y), y);
}

// r, 1/r and r - R from R and s = r^2 - R^2 (R > 0, r > 0)
DF_HD void df_split_r(dfl R, dfl s, dfl& r, dfl& rinv, dfl& dr) {
    const dfl r2 = df_add(df_mul(R, R), s);
    rinv = df_rsqrt(r2);
    r = df_mul(r2, rinv);
    r = df_add(r, df_mul(df_mul_f(rinv, 0.5f), df_sub(r2, df_mul(r, r))));  // one Newton step
    dr = df_div(s, df_add(r, R));
}

// e^{i kappa r} / (4 pi r), phase phi0 + kappa (r - R) with phi0 = kappa R mod 2 pi
DF_HD void phi3d_df(dfl kappa, dfl R, dfl s, dfl phi0, dfl& re, dfl& im) {
    dfl r, rinv, dr;
    df_split_r(R, s, r, rinv, dr);
    dfl sn, cs;
    df_sincos(df_add(phi0, df_mul(kappa, dr)), sn, cs);
    const dfl a = df_mul(rinv, df_const(0.079577471545947667884));  // 1 / (4 pi)
    re = df_mul(a, cs);
    im = df_mul(a, sn);
}

// Polynomial of degree deg, coefficients highest first as (hi, lo) pairs.
DF_HD dfl df_horner(const float* hi, const float* lo, int deg, dfl u) {
    dfl p = {hi[0], lo[0]};
    for (int k = 1; k <= deg; ++k) p = df_fma(p, u, dfl{hi[k], lo[k]});
    return p;
}

// One modulus/phase fit of H0 on x >= xa (the FP64 fits of bessel_coeffs.h):
// (i/4) H0(x) = amp e^{i phase} with u = 2 xa / x - 1,
// amp = (1/4) sqrt(2/pi) f(u) / sqrt(x) and phase = x + pi/4 + g(u).
struct DfFit {
    float xa;
    int deg;
    const float *fhi, *flo, *ghi, *glo;
};

// (i/4) H0(kappa r) for kappa r >= the smallest fit's xa; phase phi0 + kappa
// (r - R) + g with phi0 = kappa R + pi / 4 mod 2 pi.  fits: nfit <= 3 fits
// ordered by decreasing xa (selected with constant indices, so that a device
// caller's fit table stays in registers).  Returns false below the last fit
// (the caller evaluates those rare pairs otherwise).
DF_HD bool phi2d_df(dfl kappa, dfl R, dfl s, dfl phi0, const DfFit* fits, int nfit, dfl& re, dfl& im) {
    dfl r, rinv, dr;
    df_split_r(R, s, r, rinv, dr);
    const dfl x = df_mul(kappa, r);
    DfFit F = fits[0];
    bool found = false;
#if defined(__CUDACC__)
#pragma unroll
#endif
    for (int k = 0; k < 3; ++k)
        if (k < nfit && !found && x.hi >= fits[k].xa) {
            F = fits[k];
            found = true;
        }
    if (!found) return false;
    // u = (2 xa / kappa) / r - 1
    const dfl u = df_add_f(df_mul(df_div(df_make(2.0f * F.xa), kappa), rinv), -1.0f);
    const dfl f = df_horner(F.fhi, F.flo, F.deg, u);
    const dfl g = df_horner(F.ghi, F.glo, F.deg, u);
    const dfl amp = df_mul(df_mul(df_const(0.19947114020071633897), f), df_rsqrt(x));  // sqrt(2/pi) / 4
    dfl sn, cs;
    df_sincos(df_add(df_add(phi0, df_mul(kappa, dr)), g), sn, cs);
    re = df_mul(amp, cs);
    im = df_mul(amp, sn);
    return true;
}
