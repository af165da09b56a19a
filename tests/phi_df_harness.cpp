// Test harness (C linkage for ctypes) for the double-float fundamental solution.
#include <math.h>

#include "../paper_2603_19113_gb300/csrc/bessel_coeffs.h"
#include "../paper_2603_19113_gb300/csrc/phi_df.h"

namespace {
const double kF64[] = MBS_F64_X64_F, kG64[] = MBS_F64_X64_G;
const double kF16[] = MBS_F64_X16_F, kG16[] = MBS_F64_X16_G;
const double kF4[] = MBS_F64_X4_F, kG4[] = MBS_F64_X4_G;
float fh[3][32], fl[3][32], gh[3][32], gl[3][32];
DfFit fits[3];

void split(const double* c, int n, float* hi, float* lo) {
    for (int k = 0; k < n; ++k) {
        const dfl d = df_from_double(c[k]);
        hi[k] = d.hi;
        lo[k] = d.lo;
    }
}

void init() {
    static bool done = false;
    if (done) return;
    const double* F[3] = {kF64, kF16, kF4};
    const double* G[3] = {kG64, kG16, kG4};
    const int deg[3] = {MBS_F64_X64_DEG, MBS_F64_X16_DEG, MBS_F64_X4_DEG};
    const float xa[3] = {(float)MBS_F64_X64_XA, (float)MBS_F64_X16_XA, (float)MBS_F64_X4_XA};
    for (int i = 0; i < 3; ++i) {
        split(F[i], deg[i] + 1, fh[i], fl[i]);
        split(G[i], deg[i] + 1, gh[i], gl[i]);
        fits[i] = DfFit{xa[i], deg[i], fh[i], fl[i], gh[i], gl[i]};
    }
    done = true;
}
}  // namespace

// in: 4 df values per point (kappa, R, s, phi0) as (hi, lo) float pairs;
// out: 4 floats per point (re hi, re lo, im hi, im lo); ok: 1 if evaluated
extern "C" void phi_df_batch(int dim, int n, const float* in, float* out, int* ok) {
    init();
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
