// Test support: the FP64 modulus/phase fits of H0 (bessel_coeffs.h) split into
// double-float coefficient tables, for the host-side checks.
#pragma once

#include "../paper_2603_19113_gb300/csrc/bessel_coeffs.h"
#include "../paper_2603_19113_gb300/csrc/phi_df.h"

inline const DfFit* df_fits() {
    static const double F64[] = MBS_F64_X64_F, G64[] = MBS_F64_X64_G;
    static const double F16[] = MBS_F64_X16_F, G16[] = MBS_F64_X16_G;
    static const double F4[] = MBS_F64_X4_F, G4[] = MBS_F64_X4_G;
    static float fh[3][32], fl[3][32], gh[3][32], gl[3][32];
    static DfFit fits[3];
    static bool done = false;
    if (!done) {
        const double* F[3] = {F64, F16, F4};
        const double* G[3] = {G64, G16, G4};
        const int deg[3] = {MBS_F64_X64_DEG, MBS_F64_X16_DEG, MBS_F64_X4_DEG};
        const float xa[3] = {(float)MBS_F64_X64_XA, (float)MBS_F64_X16_XA, (float)MBS_F64_X4_XA};
        for (int i = 0; i < 3; ++i) {
            for (int k = 0; k <= deg[i]; ++k) {
                const dfl f = df_from_double(F[i][k]), g = df_from_double(G[i][k]);
                fh[i][k] = f.hi;
                fl[i][k] = f.lo;
                gh[i][k] = g.hi;
                gl[i][k] = g.lo;
            }
            fits[i] = DfFit{xa[i], deg[i], fh[i], fl[i], gh[i], gl[i]};
        }
        done = true;
    }
    return fits;
}
