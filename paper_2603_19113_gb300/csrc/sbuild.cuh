// Job descriptors of the batched S build (one per distinct shape) and of the
// right-hand-side kernel (one per body).
#pragma once

#include "common.cuh"

struct SBuildJob {
    // inputs (device, SoA local coordinates)
    int m, n, p;
    const double* x;
    const double* y;
    const double* z;
    int kfix;       // > 0: fixed skeleton count
    double eps;     // else: relative stopping tolerance
    // randomized ID (0 rows: the ID comes from the pivoted QR of B itself)
    int sketch_d;        // rows of the Gaussian sketch Omega B (k + oversampling)
    unsigned int seed;   // generator key: (seed, shape index)
    int shape_index;
    double2* OM;         // sketch_d x p: Omega
    double2* Y;          // sketch_d x m: Omega B, factored in place
    int* permY;          // m
    double2* diagY;      // min(sketch_d, m)
    // workspace
    double2* BD;    // p x (m + n), ld p: B | D, factored in place
    double2* AU;    // m x (n + kcap), ld m: A | U, factored in place (kept: A's reflectors)
    double2* W1;    // kcap x max(m, n)
    double2* W2;    // min(p, m) x n
    double2* W3;    // m x n
    double2* XB;    // m x min(p, m): reflectors of the RZ reduction of R_B, later G = Z* C F
    double2* XA;    // n x n: R_A^H, rotated by the Jacobi sweeps
    double* sig;    // n singular values of A
    int* keep;      // n: columns kept by the truncation
    double* nrm2;   // max(m, n)
    int* permB;     // m
    double2* diagB; // min(p, m)
    int* permA;     // n
    double2* diagA; // n
    double2* JA;    // n x n (kept): accumulated rotations, kept columns first
    double2* FA;    // n x n (kept): F = P_A V_r Sigma_r^{-1}, first rankS columns
    // outputs
    int k;          // skeleton count
    int rankB;
    int rankA;      // steps of the pivoted QR of A
    int rankS;      // singular values of A kept (> ls_rcond * largest)
    int sweepsA;    // Jacobi sweeps run
    double snorm;   // Frobenius norm of S
    double eps_ach;
    int* skel;      // kcap
    double2* Zs;    // k x m, ld k (kept)
    double2* C;     // m x n, ld m (kept)
    double2* S;     // k x k, ld k (kept)
};

struct RhsBody {
    int m, n, k, rankA, rankS;
    int64_t voff;   // first collocation row of this body in v
    int64_t boff;   // first skeleton row of this body in b
    int64_t moff;   // first MFS source of this body in q_mfs
    const double2* A;      // Householder reflectors of the pivoted QR of A (m x n, ld m)
    const double2* J;      // rotations of the truncated SVD of A (ld n, first rankS columns)
    const double2* F;      // P_A V_r Sigma_r^{-1} (n x rankS, ld n)
    const double2* C;      // m x n
    const double2* Zs;     // k x m
    const double2* W;      // injected k x m, or nullptr
};

// The whole build of njobs shapes: one persistent launch per phase of
// `threads`-thread CTAs (128, 256 or 512) that take the jobs in order from
// d_counter (3 ints, one per phase, zeroed here); rows_max = max over the
// jobs of max(p, m) (shared-memory reflector).
void launch_sbuild(int dim, SBuildJob* d_jobs, int njobs, int* d_counter, int rows_max, int threads,
                   double kappa, double rcond, cudaStream_t st);
void launch_rhs(const RhsBody* d_bodies, int T, int nrhs, int mmax, int nmax, const double2* v,
                int64_t Mtot, double2* b, int64_t N, cudaStream_t st);
// q_mfs_tau = A_tau^+ (v_tau - U_tau w_hat_tau) for every body (Sec. 4.6), with
// w_hat = G_hat q_hat the incoming field at the skeleton points ([nrhs][N]) and
// U = (Z*)^T; q_mfs is [nrhs][Nm] with body tau at rows moff .. moff + n - 1.
void launch_recon(const RhsBody* d_bodies, int T, int nrhs, int mmax, int nmax, const double2* v,
                  int64_t Mtot, const double2* w_hat, int64_t N, double2* qmfs, int64_t Nm,
                  cudaStream_t st);
