// Least-squares part of block GMRES (host code, no CUDA).
//
// Restarted GMRES on the global system (Sec. 2.4) with s right-hand sides
// advanced together: step j appends one block of s Krylov vectors, so the
// Arnoldi relation is A V_j = V_{j+1} H_j with H block upper Hessenberg
// (s sub-diagonals).  Each cycle minimises || G0 - H Y ||_F column by column,
// G0 = [R0 diag(beta); 0] from the QR factor of the initial residual block.
// H is reduced to upper triangular form by Givens rotations as it grows (s
// rotations per new column), so the residual norm of every right-hand side is
// known after every step without solving; Y is solved once per cycle.
#pragma once

#include <complex>
#include <vector>

class BlockLsq {
  public:
    using cd = std::complex<double>;

    // Start a cycle of at most `restart` steps for s right-hand sides.
    // R0: s x s upper triangular, column-major (R0[q * s + i] = R0(i, q));
    // beta: the s scale factors of its columns.
    void start(int s, int restart, const cd* R0, const double* beta);

    // Append block column j (steps in order 0, 1, ...):
    // Hcol = V^H (A v_j), K x s column-major (Hcol[a * K + i]), K = (j + 1) s;
    // Rk: s x s upper triangular factor of the new block (Rk[a * s + i]).
    void add(int j, const cd* Hcol, const cd* Rk);

    // Least-squares residual norm of right-hand side q after the last add.
    double residual(int q) const;

    // Y = R^{-1} G over the first jdone steps: Y[q * Mj + i], Mj = jdone * s.
    void solve(int jdone, std::vector<cd>& Y);

  private:
    int s_ = 0, restart_ = 0, M_ = 0, ldH_ = 0, last_ = -1;
    std::vector<cd> H_, G_, cs_, sn_;
    std::vector<double> Tre_, Tim_;
};
