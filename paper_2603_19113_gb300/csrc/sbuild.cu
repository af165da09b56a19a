// Batched FP64 construction of the local scattering matrices (Sec. 4.2-4.5).
//
// One CTA per distinct shape does the whole local computation in FP64 on
// matrices kept in global memory (L2-resident for the sizes used here):
//
//  phase 1   B(i,j) = phi(z_i - x_j)  (p x m, eq. B-matrix)
//            D(i,j) = phi(z_i - y_j)  (p x n)         A(i,j) = phi(x_i - y_j)  (m x n)
//            Householder QR of B with column pivoting (largest remaining
//            column norm, recomputed in full after every step; ties within a
//            relative 1e-10 go to the lowest original column index), with the
//            same reflectors applied to D.  The skeleton count k is fixed or
//            the first step at which the largest remaining column norm is at
//            most eps times the largest initial one; the factorisation goes on
//            to the numerical rank r_B (relative ls_rcond) for the
//            least-squares solve below.
//  phase 2   Z* = [I_k | R11^{-1} R12] in pivot order (ID, eq. B_fac),
//            C = basic least-squares solution of B C = D from the same
//            factorisation truncated at r_B (Sec. 4.4),
//            U = (Z*)^T (Sec. 4.2), pivoted QR of A truncated at r_A with the
//            reflectors applied to U, and
//            S = ((Z* C) P_A)(:, 1:r_A) R_A11^{-1} (Q_A^H U)(1:r_A, :),
//            i.e. S = Z* C A^+ U (eq. scattering-matrix) with A^+ applied as a
//            truncated pivoted-QR solve.  The division by the small pivots acts
//            on rows of Z* C before the product with the projections of U, which
//            keeps the rounding of the ill-conditioned MFS solve out of S.
//
// The right-hand side b = Z* C A^+ v (Sec. 4.5) is formed right to left from
// the stored factors (rhs_kernel): Q_A^H v, a triangular solve, C, then Z*.
#include <algorithm>

#include "bessel.cuh"
#include "common.cuh"
#include "sbuild.cuh"

namespace {

constexpr int SBT = 512;  // threads per shape CTA
constexpr int NW = SBT / 32;
constexpr double TIE = 1e-10;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
    return make_double2(warp_sum(v.x), warp_sum(v.y));
}

struct Red {
    double d[NW];
    double d2[NW];
    int i[NW];
    int j[NW];
};

// Block-wide sum of a double (every thread gets the result).
__device__ double block_sum(double v, Red& r) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) r.d[w] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += r.d[k];
    return t;
}

__device__ double block_max(double v, Red& r) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) r.d[w] = v;
    __syncthreads();
    double t = r.d[0];
#pragma unroll
    for (int k = 1; k < NW; ++k) t = fmax(t, r.d[k]);
    return t;
}

// Block-wide argmin of key (ties: smaller idx); returns idx.
__device__ int block_argmin(int key, int idx, Red& r) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int k2 = __shfl_xor_sync(0xffffffffu, key, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (k2 < key || (k2 == key && i2 < idx)) {
            key = k2;
            idx = i2;
        }
    }
    __syncthreads();
    if (lane == 0) {
        r.i[w] = key;
        r.j[w] = idx;
    }
    __syncthreads();
    int bk = r.i[0], bi = r.j[0];
#pragma unroll
    for (int k = 1; k < NW; ++k)
        if (r.i[k] < bk || (r.i[k] == bk && r.j[k] < bi)) {
            bk = r.i[k];
            bi = r.j[k];
        }
    return bi;
}

template <int DIM>
__device__ void fill_kernel_matrix(double2* M, int ld, const double* T, int nt, const double* S,
                                   int ns, double kappa) {
    for (int64_t e = threadIdx.x; e < (int64_t)nt * ns; e += blockDim.x) {
        const int i = (int)(e % nt), j = (int)(e / nt);
        double r2 = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const double d = T[c * nt + i] - S[c * ns + j];
            r2 = fma(d, d, r2);
        }
        M[(int64_t)j * ld + i] = phi_f64<DIM>(kappa, sqrt(r2));
    }
}

// Pivoted Householder QR of the first `cols` columns of A (rows x cols,
// leading dimension ld); `extra` further columns are transformed by the same
// reflectors but never pivoted.  Column j of the result holds the unit
// reflector v_j in rows j..rows-1 (H_j = I - 2 v v^H), diag[j] = R_jj, and
// rows < j of later columns hold R.  Stops at step j when
//   j == min(rows, cols), or
//   the skeleton count is known, j >= it, and the largest remaining column
//   norm is <= rcond * (largest initial norm).
// kfix > 0: skeleton count kfix; else the first j with max norm <= eps * max0.
__device__ void cta_cpqr(double2* A, int ld, int rows, int cols, int extra, int* perm,
                         double2* diag, double* nrm2, double2* s_v, int kfix, double eps,
                         double rcond, Red& red, int* out_rank, int* out_k, double* out_eps) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) perm[c] = c;
    for (int c = w; c < cols; c += NW) {
        double s = 0.0;
        for (int i = lane; i < rows; i += 32) s += cabs2(A[(int64_t)c * ld + i]);
        s = warp_sum(s);
        if (lane == 0) nrm2[c] = s;
    }
    __syncthreads();
    double m0 = 0.0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) m0 = fmax(m0, nrm2[c]);
    const double max0 = block_max(m0, red);
    const int kmax = min(rows, cols);
    int kskel = -1;
    double eps_ach = 0.0;
    int j = 0;
    for (; j < kmax; ++j) {
        double mloc = 0.0;
        for (int c = j + threadIdx.x; c < cols; c += blockDim.x) mloc = fmax(mloc, nrm2[c]);
        const double mx = block_max(mloc, red);
        if (kskel < 0) {
            if (kfix > 0 && j == kfix) {
                kskel = j;
                eps_ach = sqrt(mx / max0);
            } else if (kfix <= 0 && mx <= eps * eps * max0) {
                kskel = j;
                eps_ach = sqrt(mx / max0);
            }
        }
        if (kskel >= 0 && j >= kskel && mx <= rcond * rcond * max0) break;
        if (mx <= 0.0) break;
        // pivot: lowest original index among the columns within TIE of the max
        const double thr = (1.0 - TIE) * (1.0 - TIE) * mx;
        int key = INT_MAX, idx = INT_MAX;
        for (int c = j + threadIdx.x; c < cols; c += blockDim.x)
            if (nrm2[c] >= thr && perm[c] < key) {
                key = perm[c];
                idx = c;
            }
        const int q = block_argmin(key, idx, red);
        if (q != j) {
            for (int i = threadIdx.x; i < rows; i += blockDim.x) {
                const double2 t = A[(int64_t)j * ld + i];
                A[(int64_t)j * ld + i] = A[(int64_t)q * ld + i];
                A[(int64_t)q * ld + i] = t;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const int tp = perm[j];
                perm[j] = perm[q];
                perm[q] = tp;
                const double tn = nrm2[j];
                nrm2[j] = nrm2[q];
                nrm2[q] = tn;
            }
        }
        __syncthreads();
        // Householder reflector of column j, rows j..rows-1
        double2* cj = A + (int64_t)j * ld;
        double sl = 0.0;
        for (int i = j + threadIdx.x; i < rows; i += blockDim.x) sl += cabs2(cj[i]);
        const double nx2 = block_sum(sl, red);
        const double2 x0 = cj[j];
        const double ax0 = sqrt(cabs2(x0));
        const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
        const double nx = sqrt(nx2);
        const double2 alpha = make_double2(-ph.x * nx, -ph.y * nx);
        const double2 v0 = csub(x0, alpha);
        const double nv2 = nx2 - ax0 * ax0 + cabs2(v0);
        const double inv = nv2 > 0.0 ? 1.0 / sqrt(nv2) : 0.0;
        __syncthreads();
        for (int i = j + threadIdx.x; i < rows; i += blockDim.x) {
            const double2 v = (i == j) ? cscale(v0, inv) : cscale(cj[i], inv);
            s_v[i - j] = v;
            cj[i] = v;
        }
        if (threadIdx.x == 0) diag[j] = alpha;
        __syncthreads();
        // apply H_j to the trailing columns (warp per column), refresh norms
        for (int c = j + 1 + w; c < cols + extra; c += NW) {
            double2* cc = A + (int64_t)c * ld;
            double2 d = make_double2(0.0, 0.0);
            for (int i = j + lane; i < rows; i += 32) d = cadd(d, cmulc(s_v[i - j], cc[i]));
            d = warp_sum2(d);
            d = cscale(d, 2.0);
            double s = 0.0;
            for (int i = j + lane; i < rows; i += 32) {
                const double2 nv = csub(cc[i], cmul(s_v[i - j], d));
                cc[i] = nv;
                if (i > j) s += cabs2(nv);
            }
            if (c < cols) {
                s = warp_sum(s);
                if (lane == 0) nrm2[c] = s;
            }
        }
        __syncthreads();
    }
    if (kskel < 0) {
        kskel = (kfix > 0) ? min(kfix, j) : j;
        eps_ach = 0.0;
    }
    if (threadIdx.x == 0) {
        *out_rank = j;
        *out_k = kskel;
        *out_eps = eps_ach;
    }
    __syncthreads();
}

// X(0:n, c) = R(0:n, 0:n)^{-1} Bm(0:n, c) for c < ncols, R upper triangular stored
// above the diagonal of Rm (leading dimension ldr) with its diagonal in diag.
// One thread per right-hand-side column.  X may alias Bm.
__device__ void cta_backsub(const double2* Rm, int ldr, const double2* diag, int n,
                            const double2* Bm, int ldb, int ncols, double2* X, int ldx) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        for (int i = n - 1; i >= 0; --i) {
            double2 s = Bm[(int64_t)c * ldb + i];
            for (int l = i + 1; l < n; ++l)
                s = csub(s, cmul(Rm[(int64_t)l * ldr + i], X[(int64_t)c * ldx + l]));
            const double2 d = diag[i];
            const double id = 1.0 / cabs2(d);
            X[(int64_t)c * ldx + i] = cscale(cmulc(d, s), id);  // s / d
        }
    }
    __syncthreads();
}

}  // namespace

// ----------------------------------------------------------------------------
// phase 1: fill B | D and A, pivoted QR of B (with D)
// ----------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(SBT) sbuild_phase1(SBuildJob* jobs, double kappa, double rcond) {
    __shared__ Red red;
    extern __shared__ double2 s_v[];
    SBuildJob& J = jobs[blockIdx.x];
    fill_kernel_matrix<DIM>(J.BD, J.p, J.z, J.p, J.x, J.m, kappa);
    fill_kernel_matrix<DIM>(J.BD + (int64_t)J.m * J.p, J.p, J.z, J.p, J.y, J.n, kappa);
    fill_kernel_matrix<DIM>(J.AU, J.m, J.x, J.m, J.y, J.n, kappa);
    __syncthreads();
    cta_cpqr(J.BD, J.p, J.p, J.m, J.n, J.permB, J.diagB, J.nrm2, s_v, J.kfix, J.eps, rcond, red,
             &J.rankB, &J.k, &J.eps_ach);
}

// ----------------------------------------------------------------------------
// phase 2: Z*, C, U, pivoted QR of A (with U), S
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(SBT) sbuild_phase2(SBuildJob* jobs, double rcond) {
    __shared__ Red red;
    extern __shared__ double2 s_v[];
    SBuildJob& J = jobs[blockIdx.x];
    const int m = J.m, n = J.n, p = J.p, k = J.k, rB = J.rankB;
    // skeleton indices
    for (int i = threadIdx.x; i < k; i += blockDim.x) J.skel[i] = J.permB[i];
    // Z* (k x m, ld k): identity on the skeleton, T = R11^{-1} R12 elsewhere
    for (int64_t e = threadIdx.x; e < (int64_t)k * m; e += blockDim.x) J.Zs[e] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        J.Zs[(int64_t)J.permB[i] * k + i] = make_double2(1.0, 0.0);
    // T columns: solve into the work area W1 (k x (m-k), ld k)
    cta_backsub(J.BD, p, J.diagB, k, J.BD + (int64_t)k * p, p, m - k, J.W1, k);
    for (int64_t e = threadIdx.x; e < (int64_t)k * (m - k); e += blockDim.x) {
        const int i = (int)(e % k), c = (int)(e / k);
        J.Zs[(int64_t)J.permB[k + c] * k + i] = J.W1[e];
    }
    // C (m x n, ld m): R_B(0:rB,0:rB)^{-1} (Q^H D)(0:rB, :) in pivot order, zeros beyond rB
    cta_backsub(J.BD, p, J.diagB, rB, J.BD + (int64_t)m * p, p, n, J.W2, rB > 0 ? rB : 1);
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) J.C[e] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)rB * n; e += blockDim.x) {
        const int i = (int)(e % rB), c = (int)(e / rB);
        J.C[(int64_t)c * m + J.permB[i]] = J.W2[e];
    }
    // U = (Z*)^T into AU columns n..n+k-1 (m x k, ld m)
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)m * k; e += blockDim.x) {
        const int i = (int)(e % m), c = (int)(e / m);
        J.AU[(int64_t)(n + c) * m + i] = J.Zs[(int64_t)i * k + c];
    }
    __syncthreads();
    // pivoted QR of A (m x n) truncated at rcond, reflectors applied to U
    int kdummy;
    double edummy;
    cta_cpqr(J.AU, m, m, n, k, J.permA, J.diagA, J.nrm2, s_v, -1, rcond, rcond, red, &J.rankA,
             &kdummy, &edummy);
    const int rA = J.rankA;
    // M = Z* C (k x n) with its columns permuted by P_A: MP(:, j) = M(:, permA[j]); into W1
    for (int64_t e = threadIdx.x; e < (int64_t)k * rA; e += blockDim.x) {
        const int i = (int)(e % k), j = (int)(e / k);
        const int col = J.permA[j];
        double2 s = make_double2(0.0, 0.0);
        for (int l = 0; l < m; ++l) s = cadd(s, cmul(J.Zs[(int64_t)l * k + i], J.C[(int64_t)col * m + l]));
        J.W1[e] = s;
    }
    __syncthreads();
    // Gc R_A11 = MP  (row-wise forward substitution), in place in W1 (k x rA, ld k)
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        for (int j = 0; j < rA; ++j) {
            double2 s = J.W1[(int64_t)j * k + i];
            for (int l = 0; l < j; ++l)
                s = csub(s, cmul(J.W1[(int64_t)l * k + i], J.AU[(int64_t)j * m + l]));
            const double2 d = J.diagA[j];
            J.W1[(int64_t)j * k + i] = cscale(cmulc(d, s), 1.0 / cabs2(d));
        }
    }
    __syncthreads();
    // S = Gc (Q_A^H U)(0:rA, :)   (k x k, ld k)
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
        const int i = (int)(e % k), c = (int)(e / k);
        double2 s = make_double2(0.0, 0.0);
        for (int l = 0; l < rA; ++l)
            s = cadd(s, cmul(J.W1[(int64_t)l * k + i], J.AU[(int64_t)(n + c) * m + l]));
        J.S[e] = s;
    }
}

// ----------------------------------------------------------------------------
// right-hand side b_tau = Z* C A^+ v_tau, right to left, one CTA per (body, rhs)
// ----------------------------------------------------------------------------
// qm = A^+ t for one body with the stored pivoted QR of A truncated at rank
// r_A (basic solution): t <- Q_A^H t by the Householder reflectors, back
// substitution with R_A11, and the column permutation.  t (m) and qm (n) are
// in shared memory; every thread of the block takes part.
__device__ void apply_Apinv(const RhsBody& B, double2* t, double2* qm, double* rs, double* rs2) {
    const int m = B.m, n = B.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < B.rankA; ++j) {
        const double2* vj = B.A + (int64_t)j * m;
        double2 d = make_double2(0.0, 0.0);
        for (int i = j + threadIdx.x; i < m; i += blockDim.x) d = cadd(d, cmulc(vj[i], t[i]));
        d = warp_sum2(d);
        __syncthreads();
        if (lane == 0) {
            rs[w] = d.x;
            rs2[w] = d.y;
        }
        __syncthreads();
        double2 tot = make_double2(0.0, 0.0);
        for (int k2 = 0; k2 < nw; ++k2) {
            tot.x += rs[k2];
            tot.y += rs2[k2];
        }
        tot = cscale(tot, 2.0);
        for (int i = j + threadIdx.x; i < m; i += blockDim.x) t[i] = csub(t[i], cmul(vj[i], tot));
        __syncthreads();
    }
    // back substitution with R_A11 (thread 0: rA is small) into qm in pivot order
    for (int i = threadIdx.x; i < n; i += blockDim.x) qm[i] = make_double2(0.0, 0.0);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = B.rankA - 1; i >= 0; --i) {
            double2 s = t[i];
            for (int l = i + 1; l < B.rankA; ++l) s = csub(s, cmul(B.A[(int64_t)l * m + i], t[l]));
            const double2 d = B.diagA[i];
            t[i] = cscale(cmulc(d, s), 1.0 / cabs2(d));
        }
        for (int i = 0; i < B.rankA; ++i) qm[B.permA[i]] = t[i];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) rhs_kernel(const RhsBody* __restrict__ bodies, int T,
                                                  const double2* __restrict__ v, int64_t Mtot,
                                                  double2* __restrict__ b, int64_t N) {
    __shared__ double rs[8], rs2[8];
    extern __shared__ double2 sm[];
    const int tau = blockIdx.x, r = blockIdx.y;
    const RhsBody B = bodies[tau];
    const int m = B.m, n = B.n, k = B.k;
    double2* t = sm;          // m
    double2* qm = sm + m;     // n
    double2* q = sm + m + n;  // m
    const double2* vin = v + (int64_t)r * Mtot + B.voff;
    for (int i = threadIdx.x; i < m; i += blockDim.x) t[i] = vin[i];
    __syncthreads();
    if (B.W) {  // injected W: b = W v
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            double2 s = make_double2(0.0, 0.0);
            for (int l = 0; l < m; ++l) s = cadd(s, cmul(B.W[(int64_t)l * k + i], t[l]));
            b[(int64_t)r * N + B.boff + i] = s;
        }
        return;
    }
    apply_Apinv(B, t, qm, rs, rs2);
    // q = C q_mfs
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int l = 0; l < n; ++l) s = cadd(s, cmul(B.C[(int64_t)l * m + i], qm[l]));
        q[i] = s;
    }
    __syncthreads();
    // b = Z* q
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int l = 0; l < m; ++l) s = cadd(s, cmul(B.Zs[(int64_t)l * k + i], q[l]));
        b[(int64_t)r * N + B.boff + i] = s;
    }
}

// Sec. 4.6: q_mfs = A^+ (v - U w_hat), U(i, a) = Z*(a, i).
__global__ void __launch_bounds__(256) recon_kernel(const RhsBody* __restrict__ bodies, int T,
                                                    const double2* __restrict__ v, int64_t Mtot,
                                                    const double2* __restrict__ w_hat, int64_t N,
                                                    double2* __restrict__ qmfs, int64_t Nm) {
    __shared__ double rs[8], rs2[8];
    extern __shared__ double2 sm[];
    const int tau = blockIdx.x, r = blockIdx.y;
    const RhsBody B = bodies[tau];
    const int m = B.m, n = B.n, k = B.k;
    double2* t = sm;       // m
    double2* qm = sm + m;  // n
    const double2* vin = v + (int64_t)r * Mtot + B.voff;
    const double2* wh = w_hat + (int64_t)r * N + B.boff;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 s = vin[i];
        for (int a = 0; a < k; ++a) s = csub(s, cmul(B.Zs[(int64_t)i * k + a], wh[a]));
        t[i] = s;
    }
    __syncthreads();
    apply_Apinv(B, t, qm, rs, rs2);
    for (int j = threadIdx.x; j < n; j += blockDim.x) qmfs[(int64_t)r * Nm + B.moff + j] = qm[j];
}

void launch_sbuild_phase1(int dim, SBuildJob* d_jobs, int njobs, int pmax, double kappa,
                          double rcond, cudaStream_t st) {
    const size_t sm = (size_t)std::max(pmax, 1) * sizeof(double2);
    if (dim == 2) {
        if (sm > 48 * 1024)
            MBS_CUDA_TRY(cudaFuncSetAttribute(sbuild_phase1<2>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        sbuild_phase1<2><<<njobs, SBT, sm, st>>>(d_jobs, kappa, rcond);
    } else {
        if (sm > 48 * 1024)
            MBS_CUDA_TRY(cudaFuncSetAttribute(sbuild_phase1<3>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        sbuild_phase1<3><<<njobs, SBT, sm, st>>>(d_jobs, kappa, rcond);
    }
    MBS_CHECK_LAUNCH();
}

void launch_sbuild_phase2(SBuildJob* d_jobs, int njobs, int mmax, double rcond, cudaStream_t st) {
    const size_t sm = (size_t)std::max(mmax, 1) * sizeof(double2);
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(sbuild_phase2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm));
    sbuild_phase2<<<njobs, SBT, sm, st>>>(d_jobs, rcond);
    MBS_CHECK_LAUNCH();
}

void launch_rhs(const RhsBody* d_bodies, int T, int nrhs, int mmax, int nmax, const double2* v,
                int64_t Mtot, double2* b, int64_t N, cudaStream_t st) {
    if (T == 0 || nrhs == 0) return;
    const size_t sm = (size_t)(2 * mmax + nmax) * sizeof(double2);
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(rhs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm));
    dim3 g((unsigned)T, (unsigned)nrhs);
    rhs_kernel<<<g, 256, sm, st>>>(d_bodies, T, v, Mtot, b, N);
    MBS_CHECK_LAUNCH();
}

void launch_recon(const RhsBody* d_bodies, int T, int nrhs, int mmax, int nmax, const double2* v,
                  int64_t Mtot, const double2* w_hat, int64_t N, double2* qmfs, int64_t Nm,
                  cudaStream_t st) {
    if (T == 0 || nrhs == 0) return;
    const size_t sm = (size_t)(mmax + nmax) * sizeof(double2);
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(recon_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm));
    dim3 g((unsigned)T, (unsigned)nrhs);
    recon_kernel<<<g, 256, sm, st>>>(d_bodies, T, v, Mtot, w_hat, N, qmfs, Nm);
    MBS_CHECK_LAUNCH();
}
