// FP64-accurate G_hat matvec in double-float arithmetic on the FP32 pipe
// (Sec. 1 eq. Gmtx-entries; Sec. 2.2): y_i = sum over skeleton sources j of
// other bodies of phi(x_i - x_j) q_j, for the FP64 residuals of iterative
// refinement.  GB300 issues 64 FP32 operations per FP64 one; this kernel
// spends ~1000 FP32 operations per pair where the FP64 kernel spends ~90 FP64.
//
// Per body pair (FP64): centre difference D and phi0 = kappa |D| [+ pi/4]
// mod 2 pi in double-double (phi0_pair).  Per (target, source body): the
// constants of s = r^2 - |D|^2 (df_target_const).  Per point pair: phi in
// double-float with the phase split (phi_df.h) and an exact-product
// multiply-add into compensated accumulators, renormalised every 16 sources.
// 2D pairs with kappa r below the fits (neighbouring bodies at low kappa) take
// the FP64 power series.  The building blocks are checked on the host against
// the oracle's FP64 matvec (tests/test_gdf.py); on a GB300 the kernel agrees
// with the FP64 kernel to 1.5e-13 (2D with and without the series fallback,
// 3D).  Selected by mbs_options.fp64_kernel = 1.
#include "bessel.cuh"
#include "common.cuh"
#include "gdf_core.h"

namespace {

template <int N>
struct DfTab {
    float hi[N], lo[N];
};

template <int N>
constexpr DfTab<N> df_tab(const double (&c)[N]) {
    DfTab<N> t{};
    for (int k = 0; k < N; ++k) {
        t.hi[k] = (float)c[k];
        t.lo[k] = (float)(c[k] - (double)(float)c[k]);
    }
    return t;
}

constexpr double k64F[] = MBS_F64_X64_F, k64G[] = MBS_F64_X64_G;
constexpr double k16F[] = MBS_F64_X16_F, k16G[] = MBS_F64_X16_G;
constexpr double k4F[] = MBS_F64_X4_F, k4G[] = MBS_F64_X4_G;
__constant__ DfTab<MBS_F64_X64_DEG + 1> c_df64F = df_tab(k64F), c_df64G = df_tab(k64G);
__constant__ DfTab<MBS_F64_X16_DEG + 1> c_df16F = df_tab(k16F), c_df16G = df_tab(k16G);
__constant__ DfTab<MBS_F64_X4_DEG + 1> c_df4F = df_tab(k4F), c_df4G = df_tab(k4G);

constexpr int DF_TPB = 128;  // targets per CTA, one per thread
constexpr int DF_SB = 64;    // sources staged in shared memory per round (<= DF_TPB)

// NR right-hand sides per pass (4, 8 or 16): phi is evaluated once per pair
// and pass, so the pass width follows the number of right-hand sides
template <int DIM, int NR>
__global__ void __launch_bounds__(DF_TPB) g_df_kernel(const int64_t N, const double* __restrict__ xw,
                                                      const int* __restrict__ body,
                                                      const int64_t* __restrict__ off,
                                                      const double* __restrict__ centres,
                                                      const double kappa, const int nrhs, const int r0,
                                                      const double2* __restrict__ q,
                                                      double2* __restrict__ part,
                                                      const int* __restrict__ split_body) {
    __shared__ float s_d[DIM][2][DF_SB];  // source offsets delta_j (hi, lo)
    __shared__ float s_d2[2][DF_SB];      // |delta_j|^2
    __shared__ float4 s_q[DF_SB][NR];     // q_j: (re hi, re lo, im hi, im lo)
    const DfFit fits[3] = {
        DfFit{(float)MBS_F64_X64_XA, MBS_F64_X64_DEG, c_df64F.hi, c_df64F.lo, c_df64G.hi, c_df64G.lo},
        DfFit{(float)MBS_F64_X16_XA, MBS_F64_X16_DEG, c_df16F.hi, c_df16F.lo, c_df16G.hi, c_df16G.lo},
        DfFit{(float)MBS_F64_X4_XA, MBS_F64_X4_DEG, c_df4F.hi, c_df4F.lo, c_df4G.hi, c_df4G.lo}};
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * DF_TPB + tid;
    const bool valid = i < N;
    const int tb = valid ? body[i] : -1;
    double ci[3] = {0.0, 0.0, 0.0};
    dfl di[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
    if (valid)
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            ci[a] = centres[3 * tb + a];
            di[a] = df_from_double(xw[(int64_t)a * N + i] - ci[a]);
        }
    const dfl kd = df_from_double(kappa);
    DfAcc ar[NR], ai[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) ar[r] = ai[r] = DfAcc{0.f, 0.f};
    const int sb0 = split_body[blockIdx.y], sb1 = split_body[blockIdx.y + 1];
    for (int sb = sb0; sb < sb1; ++sb) {
        const bool act = valid && tb != sb;
        const double* cs = centres + 3 * sb;
        DfTarget t{};
        if (act) {
            double D64[3] = {0.0, 0.0, 0.0};
            dfl D[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                D64[a] = ci[a] - cs[a];
                D[a] = df_from_double(D64[a]);
            }
            t = df_target_const(DIM, D, di, df_from_double(phi0_pair(kappa, D64, DIM, DIM == 2)));
        }
        for (int64_t jc = off[sb]; jc < off[sb + 1]; jc += DF_SB) {
            const int n = (int)min((int64_t)DF_SB, off[sb + 1] - jc);
            __syncthreads();
            if (tid < n) {
                const int64_t j = jc + tid;
                dfl dj2 = df_make(0.f);
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    const dfl d = df_from_double(xw[(int64_t)a * N + j] - cs[a]);
                    s_d[a][0][tid] = d.hi;
                    s_d[a][1][tid] = d.lo;
                    dj2 = df_fma(d, d, dj2);
                }
                s_d2[0][tid] = dj2.hi;
                s_d2[1][tid] = dj2.lo;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const double2 qq = (r0 + r < nrhs) ? q[(int64_t)(r0 + r) * N + j] : make_double2(0.0, 0.0);
                    const dfl qr = df_from_double(qq.x), qi = df_from_double(qq.y);
                    s_q[tid][r] = make_float4(qr.hi, qr.lo, qi.hi, qi.lo);
                }
            }
            __syncthreads();
            if (!act) continue;
            for (int jj = 0; jj < n; ++jj) {
                dfl dj[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
#pragma unroll
                for (int a = 0; a < DIM; ++a) dj[a] = dfl{s_d[a][0][jj], s_d[a][1][jj]};
                const dfl s = df_pair_s(DIM, t, dj, dfl{s_d2[0][jj], s_d2[1][jj]});
                dfl pr, pim;
                if (DIM == 3) {
                    phi3d_df(kd, t.R, s, t.phi0, pr, pim);
                } else if (!phi2d_df(kd, t.R, s, t.phi0, fits, 3, pr, pim)) {
                    const double r2 = df_to_double(df_add(df_mul(t.R, t.R), s));
                    const double2 p = phi2d_f64(kappa * sqrt(r2));
                    pr = df_from_double(p.x);
                    pim = df_from_double(p.y);
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float4 qq = s_q[jj][r];
                    df_cmac(ar[r], ai[r], pr, pim, dfl{qq.x, qq.y}, dfl{qq.z, qq.w});
                }
                if ((jj & 15) == 15)
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        df_acc_norm(ar[r]);
                        df_acc_norm(ai[r]);
                    }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                df_acc_norm(ar[r]);
                df_acc_norm(ai[r]);
            }
        }
    }
    if (!valid) return;
    double2* out = part + (int64_t)blockIdx.y * nrhs * N;
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (r0 + r < nrhs)
            out[(int64_t)(r0 + r) * N + i] =
                make_double2((double)ar[r].hi + (double)ar[r].lo, (double)ai[r].hi + (double)ai[r].lo);
}

template <int DIM, int NR>
void launch_df_pass(const GLayout& L, const double* d_centres, double kappa, int nrhs, int r0,
                    const double2* q, double2* part, int nsplit, const int* d_split_body, cudaStream_t st) {
    const dim3 grid((unsigned)((L.N + DF_TPB - 1) / DF_TPB), (unsigned)nsplit);
    g_df_kernel<DIM, NR><<<grid, DF_TPB, 0, st>>>(L.N, L.xw64, L.body, L.off, d_centres, kappa, nrhs, r0,
                                                  q, part, d_split_body);
    MBS_CHECK_LAUNCH();
}

template <int DIM>
void launch_df_dim(const GLayout& L, const double* d_centres, double kappa, int nrhs, const double2* q,
                   double2* part, int nsplit, const int* d_split_body, cudaStream_t st) {
    int r0 = 0;
    while (r0 < nrhs) {
        const int left = nrhs - r0;
        if (left <= 4) {
            launch_df_pass<DIM, 4>(L, d_centres, kappa, nrhs, r0, q, part, nsplit, d_split_body, st);
            r0 += 4;
        } else if (left <= 8) {
            launch_df_pass<DIM, 8>(L, d_centres, kappa, nrhs, r0, q, part, nsplit, d_split_body, st);
            r0 += 8;
        } else {
            launch_df_pass<DIM, 16>(L, d_centres, kappa, nrhs, r0, q, part, nsplit, d_split_body, st);
            r0 += 16;
        }
    }
}

}  // namespace

void launch_G_df(const GLayout& L, const double* d_centres, double kappa, int nrhs, const double2* q,
                 double2* y, double2* part, int nsplit, const int* d_split_body, cudaStream_t st,
                 cudaEvent_t ev0, cudaEvent_t ev1) {
    if (L.N == 0 || nrhs == 0) return;
    if (ev0) record_event(ev0, st);
    if (L.dim == 2)
        launch_df_dim<2>(L, d_centres, kappa, nrhs, q, part, nsplit, d_split_body, st);
    else
        launch_df_dim<3>(L, d_centres, kappa, nrhs, q, part, nsplit, d_split_body, st);
    if (ev1) record_event(ev1, st);
    launch_reduce_splits64(part, nsplit, L.N * nrhs, y, st);
}
