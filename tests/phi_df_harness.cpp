// Test harness (C linkage for ctypes) for the double-float fundamental solution.
#include <math.h>

#include "df_fits.h"

// in: 4 df values per point (kappa, R, s, phi0) as (hi, lo) float pairs;
// out: 4 floats per point (re hi, re lo, im hi, im lo); ok: 1 if evaluated
extern "C" void phi_df_batch(int dim, int n, const float* in, float* out, int* ok) {
    const DfFit* fits = df_fits();
    for (int i = 0; i < n; ++i) {
        const float* q = in + 8 * i;
        const dfl kappa{q[0], q[1]}, R{q[2], q[3]}, s{q[4], q[5]}, phi0{q[6], q[7]};
        dfl re{0.f, 0.f}, im{0.f, 0.f};
        ok[i] = 1;
        if (dim == 3)
            phi3d_df(kappa, R, s, phi0, re, im);
        else
            ok[i] = phi2d_df(kappa, R, s, phi0, fits, 3, re, im) ? 1 : 0;
        out[4 * i] = re.hi;
        out[4 * i + 1] = re.lo;
        out[4 * i + 2] = im.hi;
        out[4 * i + 3] = im.lo;
    }
}

// out: 4 floats per angle (sin hi, lo, cos hi, lo)
extern "C" void sincos_df_batch(int n, const float* in, float* out) {
    for (int i = 0; i < n; ++i) {
        dfl s, c;
        df_sincos(dfl{in[2 * i], in[2 * i + 1]}, s, c);
        out[4 * i] = s.hi;
        out[4 * i + 1] = s.lo;
        out[4 * i + 2] = c.hi;
        out[4 * i + 3] = c.lo;
    }
}
