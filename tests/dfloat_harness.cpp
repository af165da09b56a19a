// Test harness (C linkage for ctypes) for the double-float arithmetic.
#include <math.h>

#include "../paper_2603_19113_gb300/csrc/dfloat.h"

// error-free transformations: out[4i..4i+3] = two_sum(a, b), two_prod(a, b)
extern "C" void df_eft(int n, const float* a, const float* b, float* out) {
    for (int i = 0; i < n; ++i) {
        const dfl s = two_sum(a[i], b[i]), p = two_prod(a[i], b[i]);
        out[4 * i] = s.hi;
        out[4 * i + 1] = s.lo;
        out[4 * i + 2] = p.hi;
        out[4 * i + 3] = p.lo;
    }
}

// x = df(a), y = df(b); out[12i + 2k], out[12i + 2k + 1] = hi, lo of
// k = 0 add, 1 sub, 2 mul, 3 div, 4 sqrt(|x|), 5 x * y.hi
extern "C" void df_ops(int n, const double* a, const double* b, float* out) {
    for (int i = 0; i < n; ++i) {
        const dfl x = df_from_double(a[i]), y = df_from_double(b[i]);
        const dfl ax = x.hi < 0.f ? df_neg(x) : x;
        const dfl r[6] = {df_add(x, y), df_sub(x, y), df_mul(x, y), df_div(x, y), df_sqrt(ax),
                          df_mul_f(x, y.hi)};
        for (int k = 0; k < 6; ++k) {
            out[12 * i + 2 * k] = r[k].hi;
            out[12 * i + 2 * k + 1] = r[k].lo;
        }
    }
}
