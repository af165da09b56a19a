// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  It runs on the
// FP32 pipe, which on GB300 issues 64 times as many operations as the FP64
// pipe.  Error-free transformations: Knuth's two-sum, the fast two-sum for
// |a| >= |b| (Dekker 1971), and the exact product via one fused multiply-add.
// The compound operations follow the standard double-word algorithms (Dekker
// 1971; Joldes, Muller & Popescu 2017 give their error bounds): add within
// 3 u^2, multiply within 4 u^2 relative (u = 2^-24), divide and square root by
// one Newton correction of the FP32 estimate.
//
// Host and device code: plain IEEE FP32 operations and fmaf only, so results
// are the same on any IEEE machine with single-precision arithmetic and no
// reassociation (no fast-math); flush-to-zero only loses the lo part of
// values below 2^-102.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

struct dfl {
    float hi, lo;
};

// s + e = a + b exactly
DF_HD dfl two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// s + e = a + b exactly, valid when |a| >= |b| (or a = 0)
DF_HD dfl fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return {s, e};
}

// p + e = a * b exactly (barring underflow)
DF_HD dfl two_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    return {p, e};
}

DF_HD dfl df_make(float hi) { return {hi, 0.f}; }

// nearest double-float to a double
DF_HD constexpr dfl df_from_double(double d) {
    return {(float)d, (float)(d - (double)(float)d)};
}

DF_HD double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

DF_HD dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

// accurate sum (both parts of both operands through two-sums)
DF_HD dfl df_add(dfl a, dfl b) {
    dfl s = two_sum(a.hi, b.hi);
    const dfl t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

DF_HD dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

DF_HD dfl df_add_f(dfl a, float b) {
    dfl s = two_sum(a.hi, b);
    s.lo += a.lo;
    return fast_two_sum(s.hi, s.lo);
}

DF_HD dfl df_mul(dfl a, dfl b) {
    dfl p = two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

DF_HD dfl df_mul_f(dfl a, float b) {
    dfl p = two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// a * b + c
DF_HD dfl df_fma(dfl a, dfl b, dfl c) { return df_add(df_mul(a, b), c); }

// a / b: FP32 quotient, then one correction from the exact remainder
DF_HD dfl df_div(dfl a, dfl b) {
    const float q1 = a.hi / b.hi;
    const dfl r = df_sub(a, df_mul_f(b, q1));
    const float q2 = r.hi / b.hi;
    return fast_two_sum(q1, q2);
}

// sqrt(a), a >= 0: y = FP32 root, corrected by (a - y^2) / (2 y)
DF_HD dfl df_sqrt(dfl a) {
    if (!(a.hi > 0.f)) return {0.f, 0.f};
    const float y = sqrtf(a.hi);
    const dfl y2 = two_prod(y, y);
    const float r = ((a.hi - y2.hi) - y2.lo) + a.lo;
    return fast_two_sum(y, r / (2.f * y));
}
