// Test harness (C linkage for ctypes): runs the block-GMRES least-squares
// reduction over a given sequence of block columns and returns the residual
// norms after every step and the final solution.
#include <complex>
#include <vector>

#include "../paper_2603_19113_gb300/csrc/blsq.h"

extern "C" int blsq_run(int s, int restart, int nsteps, const double* R0, const double* beta,
                        const double* Hcols, const double* Rks, double* resid, double* Y) {
    using cd = std::complex<double>;
    try {
        BlockLsq L;
        L.start(s, restart, reinterpret_cast<const cd*>(R0), beta);
        size_t off = 0;
        for (int j = 0; j < nsteps; ++j) {
            const int K = (j + 1) * s;
            L.add(j, reinterpret_cast<const cd*>(Hcols) + off,
                  reinterpret_cast<const cd*>(Rks) + (size_t)j * s * s);
            off += (size_t)K * s;
            for (int q = 0; q < s; ++q) resid[(size_t)j * s + q] = L.residual(q);
        }
        std::vector<cd> Yv;
        L.solve(nsteps, Yv);
        for (size_t e = 0; e < Yv.size(); ++e) {
            Y[2 * e] = Yv[e].real();
            Y[2 * e + 1] = Yv[e].imag();
        }
        return 0;
    } catch (...) {
        return 1;
    }
}
