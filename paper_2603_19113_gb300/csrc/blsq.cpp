// Least-squares part of block GMRES: incremental Givens reduction of the block
// Hessenberg matrix and the back substitution (host code, no CUDA).
#include "blsq.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

void BlockLsq::start(int s, int restart, const cd* R0, const double* beta) {
    if (s < 1 || s > 16 || restart < 1) throw std::invalid_argument("BlockLsq: 1 <= s <= 16, restart >= 1");
    s_ = s;
    restart_ = restart;
    M_ = restart * s;          // columns of the block Hessenberg matrix
    ldH_ = (restart + 1) * s;  // its rows
    last_ = -1;
    // every entry of H read later (rows < (j+2)s of block column j) is written
    // in this cycle first: no clearing between cycles
    if (H_.size() < (size_t)ldH_ * M_) H_.resize((size_t)ldH_ * M_);
    G_.assign((size_t)ldH_ * s, cd(0.0));  // right-hand side of the small problem, column-major ldH
    for (int q = 0; q < s; ++q)
        for (int i = 0; i <= q; ++i) G_[(size_t)q * ldH_ + i] = R0[(size_t)q * s + i] * beta[q];
    cs_.assign((size_t)M_ * s, cd(1.0));
    sn_.assign((size_t)M_ * s, cd(0.0));
}

void BlockLsq::add(int j, const cd* Hcol, const cd* Rk) {
    const int s = s_;
    if (j != last_ + 1 || j >= restart_) throw std::invalid_argument("BlockLsq::add: steps out of order");
    last_ = j;
    const int K = (j + 1) * s;
    const int ldH = ldH_;
    // Rows 0..K-1 of the new columns from Hcol, rows K..K+s-1 from Rk.  The
    // rotations of earlier steps act on the s new columns alike: they are
    // applied to all s together (column index fastest, real arithmetic, so
    // the s chains are independent).
    const int nrow = K + s;
    Tre_.assign((size_t)nrow * s, 0.0);
    Tim_.assign((size_t)nrow * s, 0.0);
    for (int a = 0; a < s; ++a) {
        for (int i = 0; i < K; ++i) {
            Tre_[(size_t)i * s + a] = Hcol[(size_t)a * K + i].real();
            Tim_[(size_t)i * s + a] = Hcol[(size_t)a * K + i].imag();
        }
        for (int i = 0; i <= a; ++i) {
            Tre_[(size_t)(K + i) * s + a] = Rk[(size_t)a * s + i].real();
            Tim_[(size_t)(K + i) * s + a] = Rk[(size_t)a * s + i].imag();
        }
    }
    for (int pc = 0; pc < j * s; ++pc)
        for (int t = 0; t < s; ++t) {
            const int row = pc + s - t;  // rotation on rows (row-1, row)
            const cd cc = cs_[(size_t)pc * s + t], ss = sn_[(size_t)pc * s + t];
            const double cr = cc.real(), ci = cc.imag(), sr = ss.real(), si = ss.imag();
            double* __restrict__ ur = &Tre_[(size_t)(row - 1) * s];
            double* __restrict__ ui = &Tim_[(size_t)(row - 1) * s];
            double* __restrict__ vr = &Tre_[(size_t)row * s];
            double* __restrict__ vi = &Tim_[(size_t)row * s];
            for (int a = 0; a < s; ++a) {
                const double xr = ur[a], xi = ui[a], yr = vr[a], yi = vi[a];
                ur[a] = (cr * xr + ci * xi) + (sr * yr + si * yi);
                ui[a] = (cr * xi - ci * xr) + (sr * yi - si * yr);
                vr[a] = (cr * yr - ci * yi) - (sr * xr - si * xi);
                vi[a] = (cr * yi + ci * yr) - (sr * xi + si * xr);
            }
        }
    for (int a = 0; a < s; ++a) {
        const int col = j * s + a;
        cd* hc = &H_[(size_t)col * ldH];
        for (int i = 0; i < nrow; ++i) hc[i] = cd(Tre_[(size_t)i * s + a], Tim_[(size_t)i * s + a]);
        // rotations of this step's earlier columns (in generation order)
        for (int pc = j * s; pc < col; ++pc)
            for (int t = 0; t < s; ++t) {
                const int row = pc + s - t;
                const cd cc = cs_[(size_t)pc * s + t], ss = sn_[(size_t)pc * s + t];
                const cd u = hc[row - 1], v = hc[row];
                hc[row - 1] = std::conj(cc) * u + std::conj(ss) * v;
                hc[row] = -ss * u + cc * v;
            }
        // new rotations: zero rows col+s .. col+1 (bottom up)
        for (int t = 0; t < s; ++t) {
            const int row = col + s - t;
            const cd u = hc[row - 1], v = hc[row];
            const double den = std::sqrt(std::norm(u) + std::norm(v));
            const cd cc = den > 0 ? u / den : cd(1.0), ss = den > 0 ? v / den : cd(0.0);
            cs_[(size_t)col * s + t] = cc;
            sn_[(size_t)col * s + t] = ss;
            hc[row - 1] = den;
            hc[row] = 0.0;
            for (int q = 0; q < s; ++q) {
                cd* gq = &G_[(size_t)q * ldH];
                const cd gu = gq[row - 1], gv = gq[row];
                gq[row - 1] = std::conj(cc) * gu + std::conj(ss) * gv;
                gq[row] = -ss * gu + cc * gv;
            }
        }
    }
}

double BlockLsq::residual(int q) const {
    // rows (j+1)s .. (j+2)s-1 of the rotated right-hand side
    const int j = last_;
    double rr = 0.0;
    for (int i = (j + 1) * s_; i < (j + 2) * s_; ++i) rr += std::norm(G_[(size_t)q * ldH_ + i]);
    return std::sqrt(rr);
}

void BlockLsq::solve(int jdone, std::vector<cd>& Y) {
    const int s = s_, ldH = ldH_;
    if (jdone < 0 || jdone > last_ + 1) throw std::invalid_argument("BlockLsq::solve: steps not added");
    // Column-oriented back substitution: once y_i is known, column i of R
    // (contiguous) updates the rows above i.
    const int Mj = jdone * s;
    Y.assign((size_t)Mj * s, cd(0.0));
    Tre_.assign((size_t)Mj * s, 0.0);
    Tim_.assign((size_t)Mj * s, 0.0);
    for (int q = 0; q < s; ++q)
        for (int i = 0; i < Mj; ++i) {
            Tre_[(size_t)i * s + q] = G_[(size_t)q * ldH + i].real();
            Tim_[(size_t)i * s + q] = G_[(size_t)q * ldH + i].imag();
        }
    for (int i = Mj - 1; i >= 0; --i) {
        double yr[16], yi[16];  // s <= 16; local arrays keep the update loop free of aliasing
        const cd* hcol = &H_[(size_t)i * ldH];
        const cd dgl = hcol[i];
        for (int q = 0; q < s; ++q) {
            const cd y = std::abs(dgl) > 0 ? cd(Tre_[(size_t)i * s + q], Tim_[(size_t)i * s + q]) / dgl : cd(0.0);
            Y[(size_t)q * Mj + i] = y;
            yr[q] = y.real();
            yi[q] = y.imag();
        }
        for (int l = 0; l < i; ++l) {
            const double hr = hcol[l].real(), hi = hcol[l].imag();
            double* __restrict__ gr = &Tre_[(size_t)l * s];
            double* __restrict__ gi = &Tim_[(size_t)l * s];
            for (int q = 0; q < s; ++q) {
                gr[q] -= hr * yr[q] - hi * yi[q];
                gi[q] -= hr * yi[q] + hi * yr[q];
            }
        }
    }
}
