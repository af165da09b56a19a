// Shared device/host definitions of the multibody scattering library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdio>
#include <string>

#include "mbs.h"

#define MBS_PI 3.14159265358979323846
#define MBS_TWO_PI 6.28318530717958647692
#define MBS_EULER_GAMMA 0.57721566490153286061

// ----------------------------------------------------------------------------
// complex helpers (interleaved re/im in float2 / double2)
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) {
    return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) {
    return make_double2(a.x * s, a.y * s);
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// Complex multiply-adds as four fused multiply-adds each (the FP64 pipe issues
// one per slot; a product then a sum would take six):
// acc + a b, acc + conj(a) b, acc - a b, acc - conj(a) b, and s + |a|^2.
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 acc) {
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ double2 cfmsc(double2 a, double2 b, double2 acc) {
    return make_double2(fma(-a.x, b.x, fma(-a.y, b.y, acc.x)), fma(-a.x, b.y, fma(a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ double abs2_acc(double2 a, double s) { return fma(a.x, a.x, fma(a.y, a.y, s)); }
__host__ __device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ----------------------------------------------------------------------------
// error reporting
// ----------------------------------------------------------------------------
struct MbsError {
    mbs_status st;
    std::string msg;
};

#define MBS_CUDA_TRY(call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            throw MbsError{e_ == cudaErrorMemoryAllocation ? MBS_ERR_NOMEM : MBS_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_)};         \
        }                                                                               \
    } while (0)

// Every kernel launch of the library is followed by MBS_CHECK_LAUNCH(), which
// also counts it (mbs_launch_count).
extern std::atomic<long long> g_mbs_launches;
#define MBS_CHECK_LAUNCH()                                    \
    do {                                                      \
        g_mbs_launches.fetch_add(1, std::memory_order_relaxed); \
        MBS_CUDA_TRY(cudaGetLastError());                     \
    } while (0)

// ----------------------------------------------------------------------------
// device-side geometry of the skeleton layout, shared by the G_hat kernels
// ----------------------------------------------------------------------------
struct GLayout {
    int dim;
    int T;                    // bodies
    int64_t N;                // skeleton points
    const int* body;          // [N] body id of each skeleton point (sorted)
    const int64_t* off;       // [T+1] first skeleton point of each body
    const float* loc32;       // [dim][N] local offsets delta_i = R_tau x_local (FP32)
    const double* xw64;       // [dim][N] world coordinates (FP64)
    const float4* pair;       // [T*T] per body pair: D = c_tau - c_sigma, |D| (2D: Dx,Dy,R,phi0; 3D: Dx,Dy,Dz,R)
    const float* pair_phi0;   // [T*T] 3D only: (kappa R) mod 2 pi
};

// Launch wrappers (gmatvec.cu)
void launch_pair_table(int dim, int T, const double* d_centres, const double* d_brad,
                       double kappa, float4* pair, float* pair_phi0, cudaStream_t st);
// ev0/ev1 (nullable) are recorded on st around the G_hat kernel launches
// (not the split reduction), for live timing of the dominant kernel.
// mac_path: 0 auto (FP32 pipe), 1 FP32 pipe, 2 mma.sync tensor-core
// multiply-add, 3 tcgen05 tensor-core multiply-add (needs U).
struct UmmaLayout;
void launch_G_f32(const GLayout& L, double kappa, int nrhs, const float2* q, float2* y,
                  float2* part, int nsplit, const int* d_split_body, cudaStream_t st,
                  cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, int mac_path = 0,
                  const UmmaLayout* U = nullptr);
void launch_G_f64(const GLayout& L, double kappa, int nrhs, const double2* q, double2* y,
                  double2* part, int nsplit, const int* d_split_body, cudaStream_t st,
                  cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// FP64-accurate G_hat in double-float arithmetic on the FP32 pipe (gdf.cu);
// d_centres: [T][3] body centres (FP64).  Selected by mbs_options.fp64_kernel = 1.
// ev0/ev1 as for launch_G_f64: around the kernel passes, not the reduction.
void launch_G_df(const GLayout& L, const double* d_centres, double kappa, int nrhs, const double2* q,
                 double2* y, double2* part, int nsplit, const int* d_split_body, cudaStream_t st,
                 cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// y = sum over the nsplit partial sums part[s * len + e], in split order
// (deterministic); shared by the FP64-accurate G_hat kernels.
void launch_reduce_splits64(const double2* part, int nsplit, int64_t len, double2* y, cudaStream_t st);
// Event record that works inside and outside stream capture.
void record_event(cudaEvent_t e, cudaStream_t st);
// tbody (nullable): per target a body whose skeleton sources are left out (-1: none).
void launch_field_f64(const GLayout& L, double kappa, int64_t M, const double* tgt, int nrhs,
                      const double2* q, double2* u, double2* part, int nsplit,
                      const int* d_split_body, cudaStream_t st, const int* tbody = nullptr);

// MFS sources of one placed body (Sec. 4.6 reconstruction): y_world = c + R y_local.
struct MfsBody {
    const double* y;  // local MFS sources, SoA dim x n (the shape's device copy)
    int n;
    int64_t moff;     // first row of this body in q_mfs
    double c[3];
    double R[9];      // row-major rotation
};
// u(t) += sum_j phi(t - y_j^tau) q_mfs_tau,j for every target with tb[t] = tau >= 0;
// pts SoA dim x M, u and q_mfs [nrhs][M] / [nrhs][Nm].
void launch_mfs_near(int dim, int64_t M, const double* pts, const int* tb, const MfsBody* bodies,
                     double kappa, int nrhs, const double2* qmfs, int64_t Nm, double2* u,
                     cudaStream_t st);

// Tensor-core FP32 G_hat (gumma.cu).  Sources are taken in chunks of
// umma_chunk() that never straddle a body: chunk_off[T+1] (prefix sums of
// ceil(k_tau / umma_chunk())) and
// chunk_body[nchunks]; pack holds one record per chunk (umma_pack_bytes);
// err is set to 1 if a bounded wait of the kernel ran out.  part holds
// nsplit * nrhs * N values for tiles of umma_tile() targets.
struct UmmaLayout {
    int64_t nchunks;
    const int* chunk_off;
    const int* chunk_body;
    unsigned char* pack;
    size_t pack_bytes;
    int* err;
};
size_t umma_pack_bytes(int64_t nchunks, int nrhs);
int umma_tile();
int umma_chunk();
void launch_G_umma(const GLayout& L, const UmmaLayout& U, double kappa, int nrhs, const float2* q,
                   float2* part, int nsplit, const int* d_split_body, cudaStream_t st);

// S application and vector kernels (blas.cu)
struct SBlocks {
    int T;
    const int* k;             // [T] skeleton count per body
    const int64_t* off;       // [T+1]
    const double2* const* S64;  // [T] pointer to body's S (k x k column-major), FP64
    const float2* const* S32;   // [T] same, FP32
};
void launch_sapply_f32(const SBlocks& B, int64_t N, int nrhs, const float2* x, const float2* y,
                       float2* z, int kmax, cudaStream_t st);
void launch_sapply_f64(const SBlocks& B, int64_t N, int nrhs, const double2* x, const double2* y,
                       double2* z, int kmax, cudaStream_t st);

// Multi-RHS Krylov kernels: vectors are [nrhs][N]; bases are [j][nrhs][N].
template <typename V>
void launch_dots(const V* basis, int nvec, const V* w, int64_t N, int nrhs, double2* out,
                 double2* scratch, int nblk, cudaStream_t st);
template <typename V>
void launch_update(const V* basis, int nvec, const double2* h, V* w, int64_t N, int nrhs,
                   double sign, cudaStream_t st);
template <typename V>
void launch_scale(V* w, const double* inv, V* out, int64_t N, int nrhs, cudaStream_t st);
void launch_norms64(const double2* x, int64_t N, int nrhs, double* out, double* scratch,
                    int nblk, cudaStream_t st);
void launch_f64_to_f32_scaled(const double2* x, const double* scale, float2* y, int64_t N,
                              int nrhs, cudaStream_t st);
void launch_axpy_f32_into_f64(const float2* d, const double* scale, double2* x, int64_t N,
                              int nrhs, cudaStream_t st);
void launch_sub64(const double2* b, const double2* ax, double2* r, int64_t N, int nrhs,
                  cudaStream_t st);
template <typename V>
void launch_sub(const V* b, const V* ax, V* r, int64_t n, cudaStream_t st);
void launch_f32_to_f64(const float2* a, double2* b, int64_t n, cudaStream_t st);
// Tall-skinny block products of block GMRES (fixed reduction order):
// C = A^H B (ka x kb, column-major, FP64), B += alpha A H, B <- B R^{-1}
// (R upper triangular, FP64).  ts_gram needs scratch of nblk * ka * kb
// double2 with nblk = ts_gram_blocks(N, ka, kb, V is float2); kb <= 16 for
// update/trsm.  With FP32 vectors, kb <= 8 and even N the products take the
// 16-byte-load kernels; the update then needs coef, ka * 8 float2 of scratch
// (without it the general kernel runs).
int ts_gram_blocks(int64_t N, int ka, int kb, bool f32);
// Cholesky G = R^H R of an s x s Hermitian matrix on the device (s <= 16);
// *ok = 1, or 0 (and R = I) if G is not numerically positive definite.
void launch_chol_small(const double2* G, int s, double2* R, double* ok, cudaStream_t st);
// The FP32 kernels stream the basis through shared memory with bounded waits
// and need err, the context's device error flag (set if a wait ran out; the
// outputs are then NaN).
template <typename V>
void launch_ts_gram(const V* A, int ka, const V* B, int kb, int64_t N, double2* C,
                    double2* scratch, int nblk, cudaStream_t st, int* err);
template <typename V>
void launch_ts_update(const V* A, int ka, const double2* H, double alpha, V* B, int kb, int64_t N,
                      cudaStream_t st, float2* coef = nullptr, int* err = nullptr);
template <typename V>
void launch_ts_trsm(V* B, int kb, int64_t N, const double2* R, cudaStream_t st);
void launch_f64_to_f32(const double2* a, float2* b, int64_t n, cudaStream_t st);

int mbs_num_sms();
