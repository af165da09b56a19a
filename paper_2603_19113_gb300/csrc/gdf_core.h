// Building blocks of an FP64-accurate G_hat matvec in double-float arithmetic
// (Sec. 1 eq. Gmtx-entries; Sec. 2.2): y_i = sum over sources j of other
// bodies of phi(x_i - x_j) q_j.  Host and device code, shared by the kernel
// and its host-side check.
//
// Points are x = c_body + delta with delta the rotated local offset.  For a
// target i (body tau, offset delta_i) and a source body sigma, with
// D = c_tau - c_sigma and R = |D|:
//   r^2 = R^2 + s,  s = A + B . delta_j + |delta_j|^2,
//   A = 2 D . delta_i + |delta_i|^2,  B = -2 (D + delta_i),
// so per source only B . delta_j + |delta_j|^2 is formed, and the phase is
// split as phi0 + kappa (r - R) (phi_df.h).
#pragma once

#include "phi_df.h"

// phi0 = kappa |D| (+ pi/4 in 2D) mod 2 pi for one body pair, from the FP64
// centre difference D (once per body pair, so FP64 is affordable): |D| and
// the product in double-double (exact squares and product by fma), then a
// two-part reduction; accurate to ~1e-16 rad.  A double-float phi0 would
// carry kappa R ~ 5000 at 48 bits, ~2e-11 rad, the same for every pair of the
// two bodies.
DF_HD double phi0_pair(double kappa, const double* D, int dim, bool pio4) {
    double s = 0.0, e = 0.0;  // D . D as s + e
    for (int a = 0; a < dim; ++a) {
        const double p = D[a] * D[a];
        const double pe = fma(D[a], D[a], -p);
        const double t = s + p;
        const double bb = t - s;
        e += ((s - (t - bb)) + (p - bb)) + pe;
        s = t;
    }
    const double r = sqrt(s);
    const double rr = r * r;
    const double rl = ((s - rr) - fma(r, r, -rr) + e) / (2.0 * r);  // |D| = r + rl
    double ph = kappa * r;
    double pl = fma(kappa, r, -ph) + kappa * rl;
    if (pio4) {
        const double t = ph + 0.78539816339744830962;
        pl += (0.78539816339744830962 - (t - ph)) + 3.061616997868383e-17;
        ph = t;
    }
    const double n = rint(ph * 0.15915494309189533577);
    double t = fma(-n, 6.283185307179586232, ph);  // 2 pi = hi + lo
    t = fma(-n, 2.4492935982947064e-16, t);
    return t + pl;
}

struct DfTarget {  // per (target, source body)
    dfl A, B[3], R, phi0;
};

// D: double-float centre difference c_tau - c_sigma (from the FP64 difference,
// so it keeps 48 bits relative to |D|); di: target offset; phi0 from phi0_pair
DF_HD DfTarget df_target_const(int dim, const dfl* D, const dfl* di, dfl phi0) {
    DfTarget t;
    dfl DD = df_make(0.f), Dd = df_make(0.f), dd = df_make(0.f);
    for (int a = 0; a < dim; ++a) {
        DD = df_fma(D[a], D[a], DD);
        Dd = df_fma(D[a], di[a], Dd);
        dd = df_fma(di[a], di[a], dd);
        t.B[a] = df_mul_f(df_add(D[a], di[a]), -2.0f);
    }
    for (int a = dim; a < 3; ++a) t.B[a] = df_make(0.f);
    t.R = df_sqrt(DD);
    t.A = df_add(df_mul_f(Dd, 2.0f), dd);
    t.phi0 = phi0;
    return t;
}

// s = A + B . delta_j + |delta_j|^2 (dj2 = |delta_j|^2 precomputed per source)
DF_HD dfl df_pair_s(int dim, const DfTarget& t, const dfl* dj, dfl dj2) {
    dfl s = df_add(t.A, dj2);
    for (int a = 0; a < dim; ++a) s = df_fma(t.B[a], dj[a], s);
    return s;
}

// Compensated accumulator: the high part takes each addend through a two-sum,
// the rounding errors and the addends' low parts collect in the low part;
// df_acc_norm (every few terms and at the end) keeps |lo| <= ulp(hi).
struct DfAcc {
    float hi, lo;
};

DF_HD void df_acc_add(DfAcc& a, dfl p) {
    const dfl s = two_sum(a.hi, p.hi);
    a.hi = s.hi;
    a.lo += s.lo + p.lo;
}

DF_HD void df_acc_norm(DfAcc& a) {
    const dfl s = fast_two_sum(a.hi, a.lo);
    a.hi = s.hi;
    a.lo = s.lo;
}

// a * b as an unnormalised double-float: the high parts' product exactly
// (fma), the cross terms added to its error; the accumulator's two-sum takes
// the normalisation, so the product skips its own (4 operations, not 7)
DF_HD dfl df_mul_acc(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    return {p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)))};
}

// (re, im) += phi * q for one right-hand side
DF_HD void df_cmac(DfAcc& re, DfAcc& im, dfl pr, dfl pi, dfl qr, dfl qi) {
    df_acc_add(re, df_mul_acc(pr, qr));
    df_acc_add(re, df_neg(df_mul_acc(pi, qi)));
    df_acc_add(im, df_mul_acc(pr, qi));
    df_acc_add(im, df_mul_acc(pi, qr));
}
