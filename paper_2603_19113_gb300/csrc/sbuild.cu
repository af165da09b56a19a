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
//            to the numerical rank r_B (largest remaining column norm above
//            10 ls_rcond, see B_QR_CUT) for the least-squares solve below.
//            Randomized ID (option id_sketch): the skeleton and Z* come instead
//            from the pivoted QR of the sketch Y = Omega B (k + oversampling
//            rows, Omega a complex Gaussian test matrix from Philox4x32-10
//            keyed by the seed and the shape index, Box-Muller); B's own
//            pivoted QR then serves the least-squares solve for C only.
//  phase 2   Z* = [I_k | R11^{-1} R12] in pivot order (ID, eq. B_fac);
//            C = minimum-norm least-squares solution of B C = D on the rank r_B
//            of that factorisation (Sec. 4.4): a complete orthogonal
//            decomposition R_B Z^H = [T 0] by reflectors from the right (RZ
//            reduction of the trapezoidal R_B), then
//            C P_B = Z^H [T^{-1} (Q_B^H D)(1:r_B, :); 0];
//            U = (Z*)^T (Sec. 4.2) and the pivoted QR of A with its reflectors
//            applied to U, run to the rounding level (0.01 ls_rcond).
//  phase 3   truncated SVD of A (Sec. 3.1, "truncated SVD"): one-sided Jacobi
//            (Hestenes) on X = R_A^H, the columns of X J mutually orthogonal,
//            so R_A = J Sigma V^H with V = (X J) Sigma^{-1} and
//            A P_A = (Q_A J) Sigma V^H.  Singular values at most ls_rcond times
//            the largest are dropped, as in the oracle, so that
//            A^+ = P_A V_r Sigma_r^{-1} J_r^H Q_A^H, and
//            S = (Z* C P_A V_r Sigma_r^{-1}) (J_r^H (Q_A^H U)(1:r_A, :))
//            (eq. scattering-matrix).  The division by the small singular
//            values acts on the columns of Z* C P_A V_r before the product with
//            the projections of U, which keeps the rounding of the
//            ill-conditioned MFS solve out of S.  Pivoted QR ahead of the
//            Jacobi sweeps (Drmac & Veselic 2008) leaves X with strongly graded
//            columns, so few sweeps converge.
//
// The right-hand side b = Z* C A^+ v (Sec. 4.5) is formed right to left from
// the stored factors (rhs_kernel): Q_A^H v, J_r^H, the scaled right singular
// vectors, C, then Z*.
#include <algorithm>

#include "bessel.cuh"
#include "common.cuh"
#include "sbuild.cuh"

namespace {

constexpr int SBT_MAX = 512;      // largest CTA size (threads per shape CTA: 128, 256 or 512)
constexpr int NW_MAX = SBT_MAX / 32;
constexpr double TIE = 1e-10;
// The rank of B for the least-squares solve of C: the pivoted QR stops where
// its largest remaining column norm falls to B_QR_CUT * ls_rcond.  A pivoted
// QR's diagonal overestimates the singular values it tracks; cut at 10 x
// ls_rcond it keeps the rank of the truncated SVD at ls_rcond to within 0-2
// on the test shapes (2D smooth, corner-refined and 3D), where a cut at
// ls_rcond itself keeps 4-11 more, noise-level directions.
constexpr double B_QR_CUT = 10.0;

// warps of the CTA (the block size is chosen at launch)
__device__ __forceinline__ int nwarps() { return (int)(blockDim.x >> 5); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
    return make_double2(warp_sum(v.x), warp_sum(v.y));
}

struct Red {
    double d[NW_MAX];
    double d2[NW_MAX];
    int i[NW_MAX];
    int j[NW_MAX];
};

// Block-wide sum of a double (every thread gets the result).
__device__ double block_sum(double v, Red& r) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) r.d[w] = v;
    __syncthreads();
    double t = 0.0;
    const int nw = nwarps();
    for (int k = 0; k < nw; ++k) t += r.d[k];
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
    const int nw = nwarps();
    for (int k = 1; k < nw; ++k) t = fmax(t, r.d[k]);
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
    const int nw = nwarps();
    for (int k = 1; k < nw; ++k)
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

// Step j of a Householder QR of A (rows x ncols columns, leading dimension
// ld): the unit reflector v of column j (rows j..rows-1) replaces the column
// there (H = I - 2 v v^H), diag[j] = R_jj, and H is applied to columns
// j+1 .. ntot-1 (one warp per column).  With nrm2 given, the squared norms of
// rows j+1.. of columns j+1 .. ncols-1 are refreshed in full.
__device__ void householder_step(double2* A, int ld, int rows, int j, int ncols, int ntot,
                                 double2* diag, double* nrm2, double2* s_v, Red& red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
    for (int c = j + 1 + w; c < ntot; c += nwarps()) {
        double2* cc = A + (int64_t)c * ld;
        double2 d = make_double2(0.0, 0.0);
        for (int i = j + lane; i < rows; i += 32) d = cfmac(s_v[i - j], cc[i], d);
        d = warp_sum2(d);
        d = cscale(d, 2.0);
        double s = 0.0;
        for (int i = j + lane; i < rows; i += 32) {
            const double2 nv = cfms(s_v[i - j], d, cc[i]);
            cc[i] = nv;
            if (i > j) s = abs2_acc(nv, s);
        }
        if (nrm2 && c < ncols) {
            s = warp_sum(s);
            if (lane == 0) nrm2[c] = s;
        }
    }
    __syncthreads();
}

// One-sided Jacobi (Hestenes 1958) on the r columns of X (rows x r, leading
// dimension ldx): plane rotations from the right until every pair of columns
// is orthogonal to tol relative to the product of their norms; X J = W with
// orthogonal columns, J (r x r, leading dimension ldj, starts as I)
// accumulating the rotations.  Pairs are taken in round-robin tournament
// order, so every round rotates r/2 disjoint pairs, one warp per pair; the
// result does not depend on the warp schedule.  Returns the sweeps run
// (maxsweep + 1 if the last one still rotated).
__device__ int cta_jacobi(double2* X, int ldx, int rows, int r, double2* Jm, int ldj, double tol,
                          int maxsweep, int* s_flag) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int re = r + (r & 1);  // with a dummy column when r is odd
    const int half = re / 2;
    for (int sweep = 0; sweep < maxsweep; ++sweep) {
        if (threadIdx.x == 0) *s_flag = 0;
        __syncthreads();
        for (int rho = 0; rho < re - 1; ++rho) {
            for (int pi = w; pi < half; pi += nwarps()) {
                int i, j;
                if (pi == 0) {
                    i = rho;
                    j = re - 1;
                } else {
                    i = (rho + pi) % (re - 1);
                    j = (rho - pi + re - 1) % (re - 1);
                }
                if (i > j) {
                    const int t = i;
                    i = j;
                    j = t;
                }
                if (j >= r) continue;
                double2* xi = X + (int64_t)i * ldx;
                double2* xj = X + (int64_t)j * ldx;
                double a = 0.0, b = 0.0;
                double2 c = make_double2(0.0, 0.0);
                for (int l = lane; l < rows; l += 32) {
                    const double2 u = xi[l], v = xj[l];
                    a = abs2_acc(u, a);
                    b = abs2_acc(v, b);
                    c = cfmac(u, v, c);
                }
                a = warp_sum(a);
                b = warp_sum(b);
                c = warp_sum2(c);
                const double ac = sqrt(cabs2(c));
                if (!(ac > 0.0) || ac <= tol * sqrt(a) * sqrt(b)) continue;
                if (lane == 0) *s_flag = 1;
                // x_j' = e^{-i arg c} x_j makes the pair's inner product real and
                // positive; then the real rotation with t = tan(theta) the
                // smaller root of t^2 + 2 zeta t - 1 = 0
                const double2 ph = make_double2(c.x / ac, -c.y / ac);
                const double zeta = (b - a) / (2.0 * ac);
                const double t = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
                const double cs = 1.0 / hypot(1.0, t);
                const double sn = cs * t;
                for (int l = lane; l < rows; l += 32) {
                    const double2 u = xi[l], v = cmul(ph, xj[l]);
                    xi[l] = make_double2(cs * u.x - sn * v.x, cs * u.y - sn * v.y);
                    xj[l] = make_double2(sn * u.x + cs * v.x, sn * u.y + cs * v.y);
                }
                double2* ji = Jm + (int64_t)i * ldj;
                double2* jj = Jm + (int64_t)j * ldj;
                for (int l = lane; l < r; l += 32) {
                    const double2 u = ji[l], v = cmul(ph, jj[l]);
                    ji[l] = make_double2(cs * u.x - sn * v.x, cs * u.y - sn * v.y);
                    jj[l] = make_double2(sn * u.x + cs * v.x, sn * u.y + cs * v.y);
                }
            }
            __syncthreads();
        }
        const int more = *s_flag;
        __syncthreads();
        if (!more) return sweep + 1;
    }
    return maxsweep + 1;
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
    for (int c = w; c < cols; c += nwarps()) {
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
        householder_step(A, ld, rows, j, cols, cols + extra, diag, nrm2, s_v, red);
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
                s = cfms(Rm[(int64_t)l * ldr + i], X[(int64_t)c * ldx + l], s);
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
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Entry (i, l) of the complex Gaussian test matrix: counter (l, i, 0, 0), key
// (seed, shape); two 53-bit uniforms in (0, 1) and the Box-Muller transform,
// scaled to unit variance (the same definition as the oracle's).
__device__ __forceinline__ double2 sketch_entry(int i, int l, unsigned seed, int shape) {
    const uint4 w = philox4x32_10(make_uint4((unsigned)l, (unsigned)i, 0u, 0u), make_uint2(seed, (unsigned)shape));
    const double u1 = (double)(((unsigned long long)w.x << 21) + (w.y >> 11)) * 0x1p-53 + 0x1p-54;
    const double u2 = (double)(((unsigned long long)w.z << 21) + (w.w >> 11)) * 0x1p-53 + 0x1p-54;
    const double rad = sqrt(-2.0 * log(u1));
    const double th = 6.283185307179586 * u2;
    const double is2 = 0.70710678118654752440;
    return make_double2(rad * cos(th) * is2, rad * sin(th) * is2);
}

template <int DIM>
__device__ __forceinline__ void sbuild_phase1(SBuildJob& J, double kappa, double rcond, Red& red, double2* s_v) {
    fill_kernel_matrix<DIM>(J.BD, J.p, J.z, J.p, J.x, J.m, kappa);
    fill_kernel_matrix<DIM>(J.BD + (int64_t)J.m * J.p, J.p, J.z, J.p, J.y, J.n, kappa);
    fill_kernel_matrix<DIM>(J.AU, J.m, J.x, J.m, J.y, J.n, kappa);
    __syncthreads();
    if (J.sketch_d > 0) {
        const int d = J.sketch_d, p = J.p, m = J.m;
        for (int64_t e = threadIdx.x; e < (int64_t)d * p; e += blockDim.x)
            J.OM[e] = sketch_entry((int)(e % d), (int)(e / d), J.seed, J.shape_index);
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)d * m; e += blockDim.x) {
            const int i = (int)(e % d), j = (int)(e / d);
            double2 sum = make_double2(0.0, 0.0);
            for (int l = 0; l < p; ++l) sum = cfma(J.OM[(int64_t)l * d + i], J.BD[(int64_t)j * p + l], sum);
            J.Y[e] = sum;
        }
        __syncthreads();
        // the ID from the sketch: halted at k (a cutoff above every column norm)
        int rankY;
        cta_cpqr(J.Y, d, d, m, 0, J.permY, J.diagY, J.nrm2, s_v, J.kfix, 0.0, 2.0, red, &rankY, &J.k,
                 &J.eps_ach);
        // B's own factorisation, for the least-squares solve of C
        int kd;
        double ed;
        cta_cpqr(J.BD, J.p, J.p, J.m, J.n, J.permB, J.diagB, J.nrm2, s_v, J.kfix, J.eps, B_QR_CUT * rcond, red,
                 &J.rankB, &kd, &ed);
        return;
    }
    cta_cpqr(J.BD, J.p, J.p, J.m, J.n, J.permB, J.diagB, J.nrm2, s_v, J.kfix, J.eps, B_QR_CUT * rcond, red,
             &J.rankB, &J.k, &J.eps_ach);
}

// ----------------------------------------------------------------------------
// phase 2: Z*, C (minimum norm), U, pivoted QR of A (with U)
// ----------------------------------------------------------------------------
__device__ __forceinline__ void sbuild_phase2(SBuildJob& J, double rcond, Red& red, double2* s_v) {
    const int m = J.m, n = J.n, p = J.p, k = J.k, rB = J.rankB;
    // the ID's factorisation: B's own pivoted QR, or the sketch's
    const bool sk = J.sketch_d > 0;
    const double2* RI = sk ? J.Y : J.BD;
    const int ldi = sk ? J.sketch_d : p;
    const int* permI = sk ? J.permY : J.permB;
    const double2* diagI = sk ? J.diagY : J.diagB;
    // skeleton indices
    for (int i = threadIdx.x; i < k; i += blockDim.x) J.skel[i] = permI[i];
    // Z* (k x m, ld k): identity on the skeleton, T = R11^{-1} R12 elsewhere
    for (int64_t e = threadIdx.x; e < (int64_t)k * m; e += blockDim.x) J.Zs[e] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        J.Zs[(int64_t)permI[i] * k + i] = make_double2(1.0, 0.0);
    // T columns: solve into the work area W1 (k x (m-k), ld k)
    cta_backsub(RI, ldi, diagI, k, RI + (int64_t)k * ldi, ldi, m - k, J.W1, k);
    for (int64_t e = threadIdx.x; e < (int64_t)k * (m - k); e += blockDim.x) {
        const int i = (int)(e % k), c = (int)(e / k);
        J.Zs[(int64_t)permI[k + c] * k + i] = J.W1[e];
    }
    // C (m x n, ld m): minimum-norm solution of R_B (C P_B) = (Q_B^H D)(0:rB, :) with
    // R_B = [R11 R12] (rB x m, upper trapezoidal, pivot order).  Complete
    // orthogonal decomposition by reflectors from the right (the RZ reduction):
    // for rows i = rB-1 .. 0 a reflector P_i on column i and columns rB..m-1
    // zeroes row i of R12, so R_B P_{rB-1} ... P_0 = [T 0] with T upper
    // triangular; then C P_B = P_{rB-1} ... P_0 [T^{-1} (Q_B^H D)(0:rB, :); 0].
    // A reflector has 1 + m - rB entries (m - rB is small when B is close to
    // full rank), so this costs O(rB^2 (m - rB)), not the O(m rB^2) of a QR of
    // R_B^H.  V (1 + m - rB) x rB in XB holds the unit reflectors.
    {
        const int L = m - rB + 1;
        double2* V = J.XB;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = nwarps();
        // entry l of row r's reduced vector: column r (l = 0) or column rB + l - 1
        auto col_of = [&](int r, int l) { return l == 0 ? r : rB + l - 1; };
        if (L > 1) {
            for (int i = rB - 1; i >= 0; --i) {
                double sl = 0.0;
                for (int l = threadIdx.x; l < L; l += blockDim.x)
                    sl += cabs2(l == 0 ? J.diagB[i] : J.BD[(int64_t)col_of(i, l) * p + i]);
                const double nx2 = block_sum(sl, red);
                // a = conj(u) with u = row i's vector; P a = alpha e1, so u P = conj(alpha) e1
                const double2 u0 = J.diagB[i];
                const double2 a0 = make_double2(u0.x, -u0.y);
                const double ax0 = sqrt(cabs2(a0));
                const double2 ph = ax0 > 0.0 ? make_double2(a0.x / ax0, a0.y / ax0) : make_double2(1.0, 0.0);
                const double nx = sqrt(nx2);
                const double2 alpha = make_double2(-ph.x * nx, -ph.y * nx);
                const double2 v0 = csub(a0, alpha);
                const double nv2 = nx2 - ax0 * ax0 + cabs2(v0);
                const double inv = nv2 > 0.0 ? 1.0 / sqrt(nv2) : 0.0;
                for (int l = threadIdx.x; l < L; l += blockDim.x) {
                    double2 v;
                    if (l == 0) {
                        v = cscale(v0, inv);
                    } else {
                        const double2 u = J.BD[(int64_t)col_of(i, l) * p + i];
                        v = cscale(make_double2(u.x, -u.y), inv);
                        J.BD[(int64_t)col_of(i, l) * p + i] = make_double2(0.0, 0.0);
                    }
                    V[(int64_t)i * L + l] = v;
                }
                __syncthreads();  // every thread has read R(i, i) before it is replaced
                if (threadIdx.x == 0) J.diagB[i] = make_double2(alpha.x, -alpha.y);
                // rows r < i: w <- w P_i = w - 2 (w . v) v^H
                for (int r = w; r < i; r += nw) {
                    double2 d = make_double2(0.0, 0.0);
                    for (int l = lane; l < L; l += 32)
                        d = cfma(J.BD[(int64_t)col_of(i, l) * p + r], V[(int64_t)i * L + l], d);
                    d = cscale(warp_sum2(d), 2.0);
                    for (int l = lane; l < L; l += 32) {
                        double2& x = J.BD[(int64_t)col_of(i, l) * p + r];
                        x = cfmsc(V[(int64_t)i * L + l], d, x);  // x - conj(v_l) d
                    }
                }
                __syncthreads();
            }
        }
        // Y = T^{-1} (Q_B^H D)(0:rB, :) into W2 (rB x n, ld rB), T now in R_B's place
        const int ldy = rB > 0 ? rB : 1;
        cta_backsub(J.BD, p, J.diagB, rB, J.BD + (int64_t)m * p, p, n, J.W2, ldy);
        for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
            const int i = (int)(e % m), c = (int)(e / m);
            J.W3[e] = i < rB ? J.W2[(int64_t)c * ldy + i] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        // W3 <- P_{rB-1} ... P_0 W3 (P_0 first), P_i x = x - 2 v (v^H x)
        if (L > 1) {
            for (int i = 0; i < rB; ++i) {
                for (int c = w; c < n; c += nw) {
                    double2* x = J.W3 + (int64_t)c * m;
                    double2 d = make_double2(0.0, 0.0);
                    for (int l = lane; l < L; l += 32) d = cfmac(V[(int64_t)i * L + l], x[col_of(i, l)], d);
                    d = cscale(warp_sum2(d), 2.0);
                    for (int l = lane; l < L; l += 32)
                        x[col_of(i, l)] = cfms(V[(int64_t)i * L + l], d, x[col_of(i, l)]);
                }
                __syncthreads();
            }
        }
    }
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += blockDim.x) {
        const int i = (int)(e % m), c = (int)(e / m);
        J.C[(int64_t)c * m + J.permB[i]] = J.W3[e];
    }
    // U = (Z*)^T into AU columns n..n+k-1 (m x k, ld m)
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)m * k; e += blockDim.x) {
        const int i = (int)(e % m), c = (int)(e / m);
        J.AU[(int64_t)(n + c) * m + i] = J.Zs[(int64_t)i * k + c];
    }
    __syncthreads();
    // pivoted QR of A (m x n), reflectors applied to U, run down to the
    // rounding level: the truncation itself is done on the singular values
    const double rq = 0.01 * rcond;
    int kdummy;
    double edummy;
    cta_cpqr(J.AU, m, m, n, k, J.permA, J.diagA, J.nrm2, s_v, -1, rq, rq, red, &J.rankA, &kdummy,
             &edummy);
}

// ----------------------------------------------------------------------------
// phase 3: truncated SVD of A from its pivoted QR (one-sided Jacobi on
// R_A^H), the factors of A^+, and S
// ----------------------------------------------------------------------------
__device__ __forceinline__ void sbuild_phase3(SBuildJob& J, double rcond, Red& red, int& s_flag, int& s_r) {
    const int m = J.m, n = J.n, k = J.k, rA = J.rankA;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // X = R_A^H (n x rA, ld n) and J = I (rA x rA, ld n)
    for (int64_t e = threadIdx.x; e < (int64_t)n * rA; e += blockDim.x) {
        const int c = (int)(e % n), i = (int)(e / n);
        double2 v = make_double2(0.0, 0.0);
        if (c == i)
            v = J.diagA[i];
        else if (c > i)
            v = J.AU[(int64_t)c * m + i];
        J.XA[e] = make_double2(v.x, -v.y);
    }
    for (int64_t e = threadIdx.x; e < (int64_t)rA * rA; e += blockDim.x) {
        const int l = (int)(e % rA), i = (int)(e / rA);
        J.JA[(int64_t)i * n + l] = make_double2(l == i ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    const double tol = 2.220446049250313e-16 * sqrt((double)max(n, 1));
    const int sweeps = cta_jacobi(J.XA, n, n, rA, J.JA, n, tol, 60, &s_flag);
    // singular values = column norms of X J
    for (int i = w; i < rA; i += nwarps()) {
        double sum = 0.0;
        for (int l = lane; l < n; l += 32) sum = abs2_acc(J.XA[(int64_t)i * n + l], sum);
        sum = warp_sum(sum);
        if (lane == 0) J.sig[i] = sqrt(sum);
    }
    __syncthreads();
    double mloc = 0.0;
    for (int i = threadIdx.x; i < rA; i += blockDim.x) mloc = fmax(mloc, J.sig[i]);
    const double smax = block_max(mloc, red);
    if (threadIdx.x == 0) {
        int r = 0;
        for (int i = 0; i < rA; ++i)
            if (J.sig[i] > rcond * smax) J.keep[r++] = i;
        s_r = r;
        J.rankS = r;
        J.sweepsA = sweeps;
    }
    __syncthreads();
    const int r = s_r;
    // F = P_A V_r Sigma_r^{-1} = P_A (X J)(:, kept) Sigma_r^{-2}  (n x r, ld n, rows in
    // the original column order of A)
    for (int64_t e = threadIdx.x; e < (int64_t)n * r; e += blockDim.x) {
        const int row = (int)(e % n), slot = (int)(e / n);
        const int i = J.keep[slot];
        const double sg = J.sig[i];
        J.FA[(int64_t)slot * n + J.permA[row]] = cscale(J.XA[(int64_t)i * n + row], 1.0 / (sg * sg));
    }
    // kept columns of J moved to the front, in order (a source column is never
    // the destination of an earlier one)
    for (int slot = 0; slot < r; ++slot) {
        const int i = J.keep[slot];
        if (i != slot)
            for (int l = threadIdx.x; l < rA; l += blockDim.x)
                J.JA[(int64_t)slot * n + l] = J.JA[(int64_t)i * n + l];
        __syncthreads();
    }
    // M = Z* C (k x n, ld k) into W1
    for (int64_t e = threadIdx.x; e < (int64_t)k * n; e += blockDim.x) {
        const int i = (int)(e % k), c = (int)(e / k);
        double2 sum = make_double2(0.0, 0.0);
        for (int l = 0; l < m; ++l) sum = cfma(J.Zs[(int64_t)l * k + i], J.C[(int64_t)c * m + l], sum);
        J.W1[e] = sum;
    }
    // H = J_r^H (Q_A^H U)(0:rA, :)  (r x k, ld r) into W3
    const int ldh = r > 0 ? r : 1;
    for (int64_t e = threadIdx.x; e < (int64_t)r * k; e += blockDim.x) {
        const int i = (int)(e % ldh), c = (int)(e / ldh);
        double2 sum = make_double2(0.0, 0.0);
        for (int l = 0; l < rA; ++l)
            sum = cfmac(J.JA[(int64_t)i * n + l], J.AU[(int64_t)(n + c) * m + l], sum);
        J.W3[e] = sum;
    }
    __syncthreads();
    // G = M F  (k x r, ld k) into XB
    for (int64_t e = threadIdx.x; e < (int64_t)k * r; e += blockDim.x) {
        const int i = (int)(e % k), c = (int)(e / k);
        double2 sum = make_double2(0.0, 0.0);
        for (int l = 0; l < n; ++l) sum = cfma(J.W1[(int64_t)l * k + i], J.FA[(int64_t)c * n + l], sum);
        J.XB[e] = sum;
    }
    __syncthreads();
    // S = G H  (k x k, ld k), and its Frobenius norm
    double sq = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
        const int i = (int)(e % k), c = (int)(e / k);
        double2 sum = make_double2(0.0, 0.0);
        for (int l = 0; l < r; ++l) sum = cfma(J.XB[(int64_t)l * k + i], J.W3[(int64_t)c * ldh + l], sum);
        J.S[e] = sum;
        sq += cabs2(sum);
    }
    sq = block_sum(sq, red);
    if (threadIdx.x == 0) J.snorm = sqrt(sq);
}

// ----------------------------------------------------------------------------
// persistent launches: every CTA takes the next shape from an atomic counter.
// The host orders the shapes by decreasing work, so this is longest-
// processing-time-first scheduling over uneven sizes, and a launch covers the
// whole batch with a grid sized to the GPU.  The three phases stay separate
// kernels (one register allocation each; a fused kernel spilled).
// ----------------------------------------------------------------------------
__device__ __forceinline__ int next_job(int* counter, int* s_job) {
    if (threadIdx.x == 0) *s_job = atomicAdd(counter, 1);
    __syncthreads();
    const int j = *s_job;
    __syncthreads();  // every thread holds j before thread 0 fetches the next one
    return j;
}

template <int DIM>
__global__ void __launch_bounds__(SBT_MAX) sbuild_phase1_kernel(SBuildJob* jobs, int njobs, int* counter,
                                                                double kappa, double rcond) {
    __shared__ Red red;
    __shared__ int s_job;
    extern __shared__ double2 s_v[];
    for (int j = next_job(counter, &s_job); j < njobs; j = next_job(counter, &s_job))
        sbuild_phase1<DIM>(jobs[j], kappa, rcond, red, s_v);
}

__global__ void __launch_bounds__(SBT_MAX) sbuild_phase2_kernel(SBuildJob* jobs, int njobs, int* counter,
                                                                double rcond) {
    __shared__ Red red;
    __shared__ int s_job;
    extern __shared__ double2 s_v[];
    for (int j = next_job(counter, &s_job); j < njobs; j = next_job(counter, &s_job))
        sbuild_phase2(jobs[j], rcond, red, s_v);
}

__global__ void __launch_bounds__(SBT_MAX) sbuild_phase3_kernel(SBuildJob* jobs, int njobs, int* counter,
                                                                double rcond) {
    __shared__ Red red;
    __shared__ int s_job, s_flag, s_r;
    for (int j = next_job(counter, &s_job); j < njobs; j = next_job(counter, &s_job))
        sbuild_phase3(jobs[j], rcond, red, s_flag, s_r);
}

// ----------------------------------------------------------------------------
// right-hand side b_tau = Z* C A^+ v_tau, right to left, one CTA per (body, rhs)
// ----------------------------------------------------------------------------
// qm = A^+ t for one body from the stored factors of the truncated SVD:
// t <- Q_A^H t by the Householder reflectors, z = J_r^H t(0:rA) (r values),
// qm = F z with F = P_A V_r Sigma_r^{-1}.  t (m), z (n) and qm (n) are in
// shared memory; every thread of the block takes part.
__device__ void apply_Apinv(const RhsBody& B, double2* t, double2* z, double2* qm, double* rs,
                            double* rs2) {
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
    for (int s = threadIdx.x; s < B.rankS; s += blockDim.x) {
        double2 sum = make_double2(0.0, 0.0);
        for (int l = 0; l < B.rankA; ++l) sum = cadd(sum, cmulc(B.J[(int64_t)s * n + l], t[l]));
        z[s] = sum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double2 sum = make_double2(0.0, 0.0);
        for (int s = 0; s < B.rankS; ++s) sum = cadd(sum, cmul(B.F[(int64_t)s * n + i], z[s]));
        qm[i] = sum;
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
    double2* t = sm;              // m
    double2* qm = sm + m;         // n
    double2* q = sm + m + n;      // m
    double2* z = sm + 2 * m + n;  // n
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
    apply_Apinv(B, t, z, qm, rs, rs2);
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
    double2* t = sm;           // m
    double2* qm = sm + m;      // n
    double2* z = sm + m + n;   // n
    const double2* vin = v + (int64_t)r * Mtot + B.voff;
    const double2* wh = w_hat + (int64_t)r * N + B.boff;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 s = vin[i];
        for (int a = 0; a < k; ++a) s = csub(s, cmul(B.Zs[(int64_t)i * k + a], wh[a]));
        t[i] = s;
    }
    __syncthreads();
    apply_Apinv(B, t, z, qm, rs, rs2);
    for (int j = threadIdx.x; j < n; j += blockDim.x) qmfs[(int64_t)r * Nm + B.moff + j] = qm[j];
}

template <typename K>
static int blocks_per_sm(K kern, int threads, size_t sm) {
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int nb = 0;
    MBS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, sm));
    return std::max(nb, 1);
}

void launch_sbuild(int dim, SBuildJob* d_jobs, int njobs, int* d_counter, int rows_max, int threads,
                   double kappa, double rcond, cudaStream_t st) {
    if (njobs == 0) return;
    if (threads != 128 && threads != 256 && threads != 512)
        throw MbsError{MBS_ERR_ARG, "S build: threads per CTA must be 128, 256 or 512"};
    const size_t sm = (size_t)std::max(rows_max, 1) * sizeof(double2);
    const int nsm = mbs_num_sms();
    MBS_CUDA_TRY(cudaMemsetAsync(d_counter, 0, 3 * sizeof(int), st));
    if (dim == 2) {
        const int g = std::min(njobs, nsm * blocks_per_sm(sbuild_phase1_kernel<2>, threads, sm));
        sbuild_phase1_kernel<2><<<g, threads, sm, st>>>(d_jobs, njobs, d_counter, kappa, rcond);
    } else {
        const int g = std::min(njobs, nsm * blocks_per_sm(sbuild_phase1_kernel<3>, threads, sm));
        sbuild_phase1_kernel<3><<<g, threads, sm, st>>>(d_jobs, njobs, d_counter, kappa, rcond);
    }
    MBS_CHECK_LAUNCH();
    int g = std::min(njobs, nsm * blocks_per_sm(sbuild_phase2_kernel, threads, sm));
    sbuild_phase2_kernel<<<g, threads, sm, st>>>(d_jobs, njobs, d_counter + 1, rcond);
    MBS_CHECK_LAUNCH();
    g = std::min(njobs, nsm * blocks_per_sm(sbuild_phase3_kernel, threads, 0));
    sbuild_phase3_kernel<<<g, threads, 0, st>>>(d_jobs, njobs, d_counter + 2, rcond);
    MBS_CHECK_LAUNCH();
}

void launch_rhs(const RhsBody* d_bodies, int T, int nrhs, int mmax, int nmax, const double2* v,
                int64_t Mtot, double2* b, int64_t N, cudaStream_t st) {
    if (T == 0 || nrhs == 0) return;
    const size_t sm = (size_t)(2 * mmax + 2 * nmax) * sizeof(double2);
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
    const size_t sm = (size_t)(mmax + 2 * nmax) * sizeof(double2);
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(recon_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm));
    dim3 g((unsigned)T, (unsigned)nrhs);
    recon_kernel<<<g, 256, sm, st>>>(d_bodies, T, v, Mtot, w_hat, N, qmfs, Nm);
    MBS_CHECK_LAUNCH();
}
