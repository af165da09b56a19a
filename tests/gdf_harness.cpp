// Test harness (C linkage for ctypes): the double-float G_hat matvec of
// csrc/gdf_core.h as a plain host loop, in the order a kernel takes it
// (per target, per source body, per source), for comparison with the oracle.
#include <cmath>
#include <cstdint>
#include <vector>

#include "../paper_2603_19113_gb300/csrc/gdf_core.h"
#include "df_fits.h"

// centres: T x 3; delta: N x 3 (row-major, offsets from the body centre);
// off: T + 1 body offsets; q, y: [nrhs][N] complex interleaved (FP64)
extern "C" int64_t gdf_matvec(int dim, double kappa, int T, const int64_t* off, const double* centres,
                              const double* delta, int nrhs, const double* q, double* y) {
    const DfFit* fits = df_fits();
    const int64_t N = off[T];
    const dfl kd = df_from_double(kappa);
    std::vector<dfl> d(3 * (size_t)N), d2((size_t)N), qd(2 * (size_t)N * nrhs);
    for (int64_t j = 0; j < N; ++j) {
        dfl s = df_make(0.f);
        for (int a = 0; a < 3; ++a) {
            d[3 * j + a] = df_from_double(delta[3 * j + a]);
            if (a < dim) s = df_fma(d[3 * j + a], d[3 * j + a], s);
        }
        d2[j] = s;
    }
    for (size_t e = 0; e < qd.size(); ++e) qd[e] = df_from_double(q[e]);
    int64_t fallback = 0;
    std::vector<DfAcc> re(nrhs), im(nrhs);
    for (int tau = 0; tau < T; ++tau)
        for (int64_t i = off[tau]; i < off[tau + 1]; ++i) {
            for (int r = 0; r < nrhs; ++r) re[r] = im[r] = DfAcc{0.f, 0.f};
            for (int sg = 0; sg < T; ++sg) {
                if (sg == tau) continue;  // zero diagonal block
                double D64[3];
                dfl D[3];
                for (int a = 0; a < 3; ++a) {
                    D64[a] = centres[3 * tau + a] - centres[3 * sg + a];
                    D[a] = df_from_double(D64[a]);
                }
                const dfl ph0 = df_from_double(phi0_pair(kappa, D64, dim, dim == 2));
                const DfTarget t = df_target_const(dim, D, &d[3 * i], ph0);
                int cnt = 0;
                for (int64_t j = off[sg]; j < off[sg + 1]; ++j) {
                    const dfl s = df_pair_s(dim, t, &d[3 * j], d2[j]);
                    dfl pr, pi;
                    if (dim == 3) {
                        phi3d_df(kd, t.R, s, t.phi0, pr, pi);
                    } else if (!phi2d_df(kd, t.R, s, t.phi0, fits, 3, pr, pi)) {
                        // kappa r below the fits: FP64 Bessel functions
                        double r2 = 0;
                        for (int a = 0; a < dim; ++a) {
                            const double e = (centres[3 * tau + a] + delta[3 * i + a]) -
                                             (centres[3 * sg + a] + delta[3 * j + a]);
                            r2 += e * e;
                        }
                        const double x = kappa * std::sqrt(r2);
                        pr = df_from_double(-0.25 * std::cyl_neumann(0.0, x));
                        pi = df_from_double(0.25 * std::cyl_bessel_j(0.0, x));
                        ++fallback;
                    }
                    for (int r = 0; r < nrhs; ++r) {
                        const size_t k = 2 * ((size_t)r * N + j);
                        df_cmac(re[r], im[r], pr, pi, qd[k], qd[k + 1]);
                    }
                    if (++cnt % 16 == 0)
                        for (int r = 0; r < nrhs; ++r) {
                            df_acc_norm(re[r]);
                            df_acc_norm(im[r]);
                        }
                }
            }
            for (int r = 0; r < nrhs; ++r) {
                df_acc_norm(re[r]);
                df_acc_norm(im[r]);
                const size_t k = 2 * ((size_t)r * N + i);
                y[k] = (double)re[r].hi + (double)re[r].lo;
                y[k + 1] = (double)im[r].hi + (double)im[r].lo;
            }
        }
    return fallback;
}
