// Block-diagonal S application and the multi-RHS Krylov vector kernels.
//
// z_tau = x_tau + S_tau y_tau for every body tau (the "I +" and "S" of
// eq. mbody2, Sec. 2.2), with S_tau k_tau x k_tau column-major and shared
// between bodies of one shape.  Vectors are stored [nrhs][N].
#include <cuda.h>

#include <atomic>
#include <string>

#include "bulk.cuh"
#include "common.cuh"

namespace {

template <typename V>
struct Acc;
template <>
struct Acc<float2> {
    using T = float;
};
template <>
struct Acc<double2> {
    using T = double;
};

template <typename V>
__device__ __forceinline__ const V* sptr(const SBlocks& B, int t);
template <>
__device__ __forceinline__ const float2* sptr<float2>(const SBlocks& B, int t) {
    return B.S32[t];
}
template <>
__device__ __forceinline__ const double2* sptr<double2>(const SBlocks& B, int t) {
    return B.S64[t];
}

constexpr int SA_RC = 8;  // right-hand sides per pass

// One CTA per body; y_tau staged in shared memory SA_RC columns at a time.
// With k < blockDim the columns of S_tau are split over P = blockDim / k
// thread groups (P <= SA_P); their partial sums are added in group order.
constexpr int SA_P = 8;
template <typename V>
__global__ void __launch_bounds__(256) sapply_kernel(const SBlocks B, const int64_t N,
                                                     const int nrhs, const V* __restrict__ x,
                                                     const V* __restrict__ y, V* __restrict__ z,
                                                     const int kmax) {
    using T = typename Acc<V>::T;
    extern __shared__ unsigned char smem_raw[];
    const int tau = blockIdx.x;
    const int k = B.k[tau];
    const int64_t o = B.off[tau];
    const V* __restrict__ S = sptr<V>(B, tau);
    V* s_y = reinterpret_cast<V*>(smem_raw);  // [SA_RC][kmax]
    V* s_part = s_y + (size_t)SA_RC * kmax;    // [P][SA_RC][k], P k <= blockDim.x
    const int P = k > 0 ? max(1, min(SA_P, (int)blockDim.x / k)) : 1;
    const int span = (k + P - 1) / P;
    for (int rc = 0; rc < nrhs; rc += SA_RC) {
        const int nr = min(SA_RC, nrhs - rc);
        __syncthreads();
        for (int idx = threadIdx.x; idx < k * nr; idx += blockDim.x) {
            const int r = idx / k, i = idx - r * k;
            s_y[r * k + i] = y[(int64_t)(rc + r) * N + o + i];
        }
        __syncthreads();
        if (P > 1) {
            // thread (i, part): rows i, columns [part * span, +span) of S_tau
            const int i = threadIdx.x % k, part = threadIdx.x / k;
            if (part < P) {
                T ar[SA_RC], ai[SA_RC];
#pragma unroll
                for (int r = 0; r < SA_RC; ++r) ar[r] = ai[r] = T(0);
                const int j1 = min(k, (part + 1) * span);
                for (int j = part * span; j < j1; ++j) {
                    const V sv = S[(int64_t)j * k + i];
#pragma unroll
                    for (int r = 0; r < SA_RC; ++r) {
                        if (r < nr) {
                            const V v = s_y[r * k + j];
                            ar[r] = fma(sv.x, v.x, fma(-sv.y, v.y, ar[r]));
                            ai[r] = fma(sv.x, v.y, fma(sv.y, v.x, ai[r]));
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < SA_RC; ++r) {
                    V pv;
                    pv.x = ar[r];
                    pv.y = ai[r];
                    s_part[((size_t)part * SA_RC + r) * k + i] = pv;
                }
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < k * nr; idx += blockDim.x) {
                const int r = idx / k, i = idx - r * k;
                T sr = T(0), si = T(0);
                for (int q = 0; q < P; ++q) {
                    const V pv = s_part[((size_t)q * SA_RC + r) * k + i];
                    sr += pv.x;
                    si += pv.y;
                }
                const int64_t g = (int64_t)(rc + r) * N + o + i;
                V out;
                const V xv = x[g];
                out.x = xv.x + sr;
                out.y = xv.y + si;
                z[g] = out;
            }
            continue;
        }
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            T ar[SA_RC], ai[SA_RC];
#pragma unroll
            for (int r = 0; r < SA_RC; ++r) ar[r] = ai[r] = T(0);
            for (int j = 0; j < k; ++j) {
                const V sv = S[(int64_t)j * k + i];
#pragma unroll
                for (int r = 0; r < SA_RC; ++r) {
                    if (r < nr) {
                        const V v = s_y[r * k + j];
                        ar[r] = fma(sv.x, v.x, fma(-sv.y, v.y, ar[r]));
                        ai[r] = fma(sv.x, v.y, fma(sv.y, v.x, ai[r]));
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < SA_RC; ++r) {
                if (r < nr) {
                    const int64_t g = (int64_t)(rc + r) * N + o + i;
                    V out;
                    const V xv = x[g];
                    out.x = xv.x + ar[r];
                    out.y = xv.y + ai[r];
                    z[g] = out;
                }
            }
        }
    }
}

constexpr int DOT_E = 8;  // w elements cached per thread: a block covers <= 256 * DOT_E rows

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// partial[(i*nrhs + r) * nblk + blk] = sum over the block's slice of conj(basis_{i,r}) . w_r
// for every i < nvec.  The block keeps its slice of w_r in registers and walks
// the basis vectors; per-thread sums are in the vector's precision, the
// cross-warp sums in FP64 and in a fixed order (bitwise reproducible).
template <typename V>
__global__ void __launch_bounds__(256) dots_kernel(const V* __restrict__ basis, const int nvec,
                                                   const V* __restrict__ w, const int64_t N,
                                                   const int nrhs, double2* __restrict__ partial,
                                                   const int nblk) {
    using T = typename Acc<V>::T;
    extern __shared__ double2 s_acc[];  // [warp][nvec]
    const int r = blockIdx.y, blk = blockIdx.x;
    const int64_t chunk = (N + nblk - 1) / nblk;
    const int64_t n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
    V wv[DOT_E];
#pragma unroll
    for (int e = 0; e < DOT_E; ++e) {
        const int64_t n = n0 + threadIdx.x + (int64_t)e * blockDim.x;
        V z;
        z.x = z.y = T(0);
        wv[e] = n < n1 ? w[(int64_t)r * N + n] : z;
    }
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int i = 0; i < nvec; ++i) {
        const V* __restrict__ vb = basis + ((int64_t)i * nrhs + r) * N;
        T sx = T(0), sy = T(0);
#pragma unroll
        for (int e = 0; e < DOT_E; ++e) {
            const int64_t n = n0 + threadIdx.x + (int64_t)e * blockDim.x;
            if (n < n1) {
                const V a = vb[n];
                sx = fma(a.x, wv[e].x, fma(a.y, wv[e].y, sx));
                sy = fma(a.x, wv[e].y, fma(-a.y, wv[e].x, sy));
            }
        }
        sx = warp_sum_t(sx);
        sy = warp_sum_t(sy);
        if ((threadIdx.x & 31) == 0) s_acc[(int64_t)warp * nvec + i] = make_double2(sx, sy);
    }
    __syncthreads();
    // warps are summed in a fixed order: the result does not depend on scheduling
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        double2 s = s_acc[i];
        for (int wi = 1; wi < nwarp; ++wi) s = cadd(s, s_acc[(int64_t)wi * nvec + i]);
        partial[((int64_t)i * nrhs + r) * nblk + blk] = s;
    }
}

// out[ir] = sum over blk of partial[ir * nblk + blk]: one warp per output,
// each lane sums a fixed stride of the partials in order, then an xor tree
// (every lane ends with the same, reproducible total).
__global__ void dots_finish_kernel(const double2* __restrict__ partial, int count, int nblk,
                                   double2* __restrict__ out) {
    const int ir = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (ir >= count) return;
    const double2* __restrict__ p = partial + (int64_t)ir * nblk;
    double sx = 0.0, sy = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 v = p[b];
        sx += v.x;
        sy += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) out[ir] = make_double2(sx, sy);
}

// w_r += sign * sum_i basis_{i,r} h[i * nrhs + r]
template <typename V>
__global__ void __launch_bounds__(256) update_kernel(const V* __restrict__ basis, const int nvec,
                                                     const double2* __restrict__ h,
                                                     V* __restrict__ w, const int64_t N,
                                                     const int nrhs, const double sign) {
    using T = typename Acc<V>::T;
    extern __shared__ unsigned char upd_raw[];
    V* s_h = reinterpret_cast<V*>(upd_raw);
    const int r = blockIdx.y;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
        const double2 c = h[i * nrhs + r];
        V cv;
        cv.x = (T)(sign * c.x);
        cv.y = (T)(sign * c.y);
        s_h[i] = cv;
    }
    __syncthreads();
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (int64_t)gridDim.x * blockDim.x) {
        V o = w[(int64_t)r * N + n];
        T ax = o.x, ay = o.y;
        for (int i = 0; i < nvec; ++i) {
            const V v = basis[((int64_t)i * nrhs + r) * N + n];
            const V c = s_h[i];
            ax = fma(v.x, c.x, fma(-v.y, c.y, ax));
            ay = fma(v.x, c.y, fma(v.y, c.x, ay));
        }
        o.x = ax;
        o.y = ay;
        w[(int64_t)r * N + n] = o;
    }
}

template <typename V>
__global__ void scale_kernel(const V* __restrict__ w, const double* __restrict__ inv,
                             V* __restrict__ out, const int64_t N, const int nrhs) {
    using T = typename Acc<V>::T;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * nrhs) return;
    const T s = (T)inv[i / N];
    V v = w[i];
    v.x *= s;
    v.y *= s;
    out[i] = v;
}

__global__ void norms_kernel(const double2* __restrict__ x, const int64_t N, const int nrhs,
                             double* __restrict__ partial, const int nblk) {
    const int r = blockIdx.y;
    double s = 0.0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (int64_t)gridDim.x * blockDim.x)
        s += cabs2(x[(int64_t)r * N + n]);
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)r * nblk + blockIdx.x] = red[0];
}

__global__ void norms_finish_kernel(const double* __restrict__ partial, int nrhs, int nblk,
                                    double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)r * nblk + b];
    out[r] = sqrt(s);
}

__global__ void f64_to_f32_scaled_kernel(const double2* __restrict__ x,
                                         const double* __restrict__ scale,
                                         float2* __restrict__ y, int64_t N, int nrhs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * nrhs) return;
    const double s = scale[i / N];
    y[i] = make_float2((float)(x[i].x * s), (float)(x[i].y * s));
}

__global__ void axpy_f32_into_f64_kernel(const float2* __restrict__ d,
                                         const double* __restrict__ scale,
                                         double2* __restrict__ x, int64_t N, int nrhs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * nrhs) return;
    const double s = scale[i / N];
    x[i].x += s * (double)d[i].x;
    x[i].y += s * (double)d[i].y;
}

__global__ void sub64_kernel(const double2* __restrict__ b, const double2* __restrict__ ax,
                             double2* __restrict__ r, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r[i] = csub(b[i], ax[i]);
}

template <typename V>
__global__ void sub_kernel(const V* __restrict__ b, const V* __restrict__ ax, V* __restrict__ r,
                           int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V o;
    o.x = b[i].x - ax[i].x;
    o.y = b[i].y - ax[i].y;
    r[i] = o;
}

__global__ void f32_to_f64_kernel(const float2* __restrict__ a, double2* __restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_double2(a[i].x, a[i].y);
}

__global__ void f64_to_f32_kernel(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

inline unsigned nblocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Cholesky G = R^H R of one s x s Hermitian matrix (column-major, s <= 16) in
// FP64 by one thread: R upper triangular, zero below the diagonal.  *ok = 1
// if every pivot exceeds 1e-13 times the largest diagonal entry of G;
// otherwise *ok = 0 and R = I, so a triangular solve with it stays finite.
// G = R^H R, right-looking: step k takes the pivot, scales row k of R by
// one reciprocal and updates the trailing upper triangle in parallel (one
// thread per entry, 16 x 16 at most); every entry is updated in the order of k.
__global__ void __launch_bounds__(256) chol_small_kernel(const double2* __restrict__ G, int s,
                                                         double2* __restrict__ R,
                                                         double* __restrict__ ok) {
    __shared__ double2 g[16 * 16];  // g[j * s + i] = G(i, j), overwritten by R(i, j)
    __shared__ double s_inv, s_gmax;
    __shared__ int s_bad;
    const int t = threadIdx.x;
    for (int e = t; e < s * s; e += blockDim.x) g[e] = G[e];
    __syncthreads();
    if (t == 0) {
        double gmax = 0.0;
        for (int i = 0; i < s; ++i) gmax = fmax(gmax, g[i * s + i].x);
        s_gmax = gmax;
        s_bad = 0;
    }
    const int ti = t % 16, tj = t / 16;  // this thread's entry (ti, tj) of the upper triangle
    for (int k = 0; k < s; ++k) {
        __syncthreads();
        if (t == 0) {
            const double d = g[k * s + k].x;
            if (!(d > 1e-13 * s_gmax)) {
                s_bad = 1;
            } else {
                const double r = sqrt(d);
                g[k * s + k] = make_double2(r, 0.0);
                s_inv = 1.0 / r;
            }
        }
        __syncthreads();
        if (s_bad) break;
        if (t > k && t < s) {  // R(k, t) = G(k, t) / R(k, k)
            const double2 v = g[t * s + k];
            g[t * s + k] = make_double2(v.x * s_inv, v.y * s_inv);
        }
        __syncthreads();
        if (tj < s && ti > k && ti <= tj)  // G(i, j) -= conj(R(k, i)) R(k, j)
            g[tj * s + ti] = csub(g[tj * s + ti], cmulc(g[ti * s + k], g[tj * s + k]));
    }
    __syncthreads();
    const bool good = s_bad == 0;
    for (int e = t; e < s * s; e += blockDim.x) {
        const int i = e % s, j = e / s;
        R[e] = good ? (i <= j ? g[e] : make_double2(0.0, 0.0))
                    : make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    if (t == 0) *ok = good ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// Tall-skinny products of block GMRES.  A block of k vectors of length N is
// stored [k][N].  Every reduction runs in a fixed order, so a solve returns
// bitwise the same result whatever else runs on the device at the same time.
//   ts_gram:   C (ka x kb, column-major) = A^H B            (FP64 result)
//   ts_update: B += alpha A H, H ka x kb column-major (FP64)
//   ts_trsm:   B <- B R^{-1}, R kb x kb upper triangular (FP64)
// ---------------------------------------------------------------------------
constexpr int TSG_A = 4, TSG_B = 8;  // output tile of one ts_gram block

// partial[(b * ka + a) * nblk + blk] = sum over the block's rows of conj(A_a) B_b
template <typename V>
__global__ void __launch_bounds__(256) ts_gram_kernel(const V* __restrict__ A, const int ka,
                                                      const V* __restrict__ B, const int kb,
                                                      const int64_t N, double2* __restrict__ partial,
                                                      const int nblk) {
    using T = typename Acc<V>::T;
    __shared__ double2 s_w[8][TSG_A * TSG_B];
    const int blk = blockIdx.x, a0 = blockIdx.y * TSG_A, b0 = blockIdx.z * TSG_B;
    const int64_t chunk = (N + nblk - 1) / nblk;
    const int64_t n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
    T ax[TSG_A][TSG_B], ay[TSG_A][TSG_B];
#pragma unroll
    for (int a = 0; a < TSG_A; ++a)
#pragma unroll
        for (int b = 0; b < TSG_B; ++b) ax[a][b] = ay[a][b] = T(0);
    for (int64_t n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
        V bv[TSG_B];
#pragma unroll
        for (int b = 0; b < TSG_B; ++b) {
            if (b0 + b < kb) {
                bv[b] = B[(int64_t)(b0 + b) * N + n];
            } else {
                bv[b].x = T(0);
                bv[b].y = T(0);
            }
        }
#pragma unroll
        for (int a = 0; a < TSG_A; ++a) {
            if (a0 + a < ka) {
                const V av = A[(int64_t)(a0 + a) * N + n];
#pragma unroll
                for (int b = 0; b < TSG_B; ++b) {
                    ax[a][b] = fma(av.x, bv[b].x, fma(av.y, bv[b].y, ax[a][b]));
                    ay[a][b] = fma(av.x, bv[b].y, fma(-av.y, bv[b].x, ay[a][b]));
                }
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < TSG_A; ++a)
#pragma unroll
        for (int b = 0; b < TSG_B; ++b) {
            const T sx = warp_sum_t(ax[a][b]);
            const T sy = warp_sum_t(ay[a][b]);
            if (lane == 0) s_w[warp][a * TSG_B + b] = make_double2((double)sx, (double)sy);
        }
    __syncthreads();
    if (threadIdx.x < TSG_A * TSG_B) {
        const int a = threadIdx.x / TSG_B, b = threadIdx.x % TSG_B;
        if (a0 + a < ka && b0 + b < kb) {
            double2 s = s_w[0][threadIdx.x];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = cadd(s, s_w[w][threadIdx.x]);
            partial[((int64_t)(b0 + b) * ka + (a0 + a)) * nblk + blk] = s;
        }
    }
}

constexpr int TSU_CH = 128;  // coefficient rows staged per round

// B_b += alpha sum_a A_a H(a, b) for b < kb <= KB; one row per thread.
template <typename V, int KB>
__global__ void __launch_bounds__(256) ts_update_kernel(const V* __restrict__ A, const int ka,
                                                        const double2* __restrict__ H,
                                                        const double alpha, V* __restrict__ B,
                                                        const int kb, const int64_t N) {
    using T = typename Acc<V>::T;
    __shared__ V s_h[TSU_CH][KB];
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T bx[KB], by[KB];
#pragma unroll
    for (int b = 0; b < KB; ++b) bx[b] = by[b] = T(0);
    for (int c0 = 0; c0 < ka; c0 += TSU_CH) {
        const int nc = min(TSU_CH, ka - c0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nc * KB; idx += blockDim.x) {
            const int a = idx / KB, b = idx - a * KB;
            V hv;
            if (b < kb) {
                const double2 h = H[(int64_t)b * ka + c0 + a];
                hv.x = (T)(alpha * h.x);
                hv.y = (T)(alpha * h.y);
            } else {
                hv.x = T(0);
                hv.y = T(0);
            }
            s_h[a][b] = hv;
        }
        __syncthreads();
        if (n < N) {
            for (int a = 0; a < nc; ++a) {
                const V av = A[(int64_t)(c0 + a) * N + n];
#pragma unroll
                for (int b = 0; b < KB; ++b) {
                    const V h = s_h[a][b];
                    bx[b] = fma(av.x, h.x, fma(-av.y, h.y, bx[b]));
                    by[b] = fma(av.x, h.y, fma(av.y, h.x, by[b]));
                }
            }
        }
    }
    if (n < N) {
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            if (b < kb) {
                V o = B[(int64_t)b * N + n];
                o.x += bx[b];
                o.y += by[b];
                B[(int64_t)b * N + n] = o;
            }
        }
    }
}

// B <- B R^{-1} (forward substitution along each row); R upper, kb <= KB.
template <typename V, int KB>
__global__ void __launch_bounds__(256) ts_trsm_kernel(V* __restrict__ B, const int kb,
                                                      const int64_t N,
                                                      const double2* __restrict__ R) {
    using T = typename Acc<V>::T;
    __shared__ V s_r[KB][KB];  // s_r[i][j] = R(i, j), i <= j
    __shared__ V s_inv[KB];    // 1 / R(j, j)
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        const int i = idx % kb, j = idx / kb;
        const double2 r = R[(int64_t)j * kb + i];
        V rv;
        rv.x = (T)r.x;
        rv.y = (T)r.y;
        s_r[i][j] = rv;
        if (i == j) {
            const double d = cabs2(r);
            V iv;
            iv.x = (T)(r.x / d);
            iv.y = (T)(-r.y / d);
            s_inv[j] = iv;
        }
    }
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    T xr[KB], xi[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) {
        if (j < kb) {
            const V v = B[(int64_t)j * N + n];
            T sr = v.x, si = v.y;
#pragma unroll
            for (int k = 0; k < j; ++k) {
                const V r = s_r[k][j];
                sr = fma(-xr[k], r.x, fma(xi[k], r.y, sr));
                si = fma(-xr[k], r.y, fma(-xi[k], r.x, si));
            }
            const V iv = s_inv[j];
            xr[j] = sr * iv.x - si * iv.y;
            xi[j] = sr * iv.y + si * iv.x;
            V o;
            o.x = xr[j];
            o.y = xi[j];
            B[(int64_t)j * N + n] = o;
        } else {
            xr[j] = xi[j] = T(0);
        }
    }
}

// FP32 tall-skinny products for block widths kb <= 8 and even N: the basis
// streamed through shared memory by bulk copies, 16-byte operands (two
// consecutive rows of one column), no cross-warp reduction in the Gram product.

// One step of a warp reduce-scatter: 2*HALF values per lane become HALF,
// lanes with bit MASK set keep the upper half.  The additions happen in an
// order fixed by the lane index, so the result is reproducible.
template <int HALF, int MASK>
__device__ __forceinline__ void fold_half(float (&v)[64], int lane) {
    const bool up = (lane & MASK) != 0;
#pragma unroll
    for (int i = 0; i < HALF; ++i) {
        const float send = up ? v[i] : v[i + HALF];
        const float keep = up ? v[i + HALF] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, MASK);
    }
}

// FP32 block Gram product V^H W, the basis streamed through a ring of
// shared-memory stages by 2D tensor copies (TMA).
//
// CTA (blk, y): basis columns 32 y .. 32 y + 31 over rows [blk chunk,
// (blk + 1) chunk).  The copy warp (warp 8, one lane) fills stage t with two
// boxes: rows n0 + 64 t .. n0 + 64 t + 63 of those columns (a bca x 512-byte
// box of the basis's tensor map, bca = min(32, ka)) and of the kb <= 8
// columns of W (kb x 512
// bytes), column c of the stage at byte 512 c, W's columns after the 32 basis
// columns; both complete on full[t % S].  Rows past N and columns past ka
// arrive as zeros.  Compute warp w owns basis columns 4 w .. 4 w + 3; lane l
// takes row pair l of each stage (one 16-byte load per column), accumulates
// its 4 x 8 complex sums in order over the stages, and releases the stage on
// empty[t % S].  A reduce-scatter across the warp then leaves one (column,
// RHS) pair per lane.  Waits are bounded: on a timeout the CTA sets *err,
// writes NaN partials and waits (bounded) for its copies in flight.
constexpr int RG_COLS = 32;
constexpr int RG_ROWS = 64;
constexpr int RG_STAGES = 4;
constexpr int RG_THREADS = 288;
constexpr int RG_COLBYTES = RG_ROWS * 8;
constexpr int RG_STAGE = (RG_COLS + 8) * RG_COLBYTES;
constexpr int RG_SMEM = RG_STAGES * RG_STAGE;
constexpr unsigned long long RING_WAIT_NS = 2000000000ull;

__global__ void __launch_bounds__(RG_THREADS, 2) ts_gram32_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                  const int ka, const int bca,
                                                                  const __grid_constant__ CUtensorMap tmB,
                                                                  const int kb, const int64_t N,
                                                                  const int64_t chunk,
                                                                  double2* __restrict__ partial,
                                                                  const int nblk, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char rg_smem[];
    __shared__ __align__(8) uint64_t full[RG_STAGES];
    __shared__ __align__(8) uint64_t empty[RG_STAGES];
    __shared__ volatile int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int blk = blockIdx.x;
    const int col0 = blockIdx.y * RG_COLS;
    const int ncol = min(RG_COLS, ka - col0);
    const int nact = (ncol + 3) >> 2;  // compute warps that own columns
    const int64_t n0 = (int64_t)blk * chunk, n1 = min(N, n0 + chunk);
    const int nst = n1 > n0 ? (int)((n1 - n0 + RG_ROWS - 1) / RG_ROWS) : 0;
    const uint32_t sbase = smem_u32(rg_smem);
    if (sbase & 127u) {  // tensor copies need 128-byte aligned stages: report, copy nothing
        if (threadIdx.x == 0) atomicExch(err, 1);
        return;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < RG_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), (uint32_t)nact);
        }
        mbar_init_fence();
        s_abort = 0;
    }
    // columns no copy writes (basis columns bca .. 31 when ka < 32, W columns
    // kb .. 7) are zero in every stage, so the products need no guards; the
    // copies zero-fill rows past N and columns past ka themselves
    {
        constexpr int W4 = RG_COLBYTES / 16;  // float4 per column
        for (int s = 0; s < RG_STAGES; ++s) {
            float4* st4 = reinterpret_cast<float4*>(rg_smem + s * RG_STAGE);
            for (int i = threadIdx.x; i < (RG_COLS - bca) * W4; i += blockDim.x)
                st4[bca * W4 + i] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = threadIdx.x; i < (8 - kb) * W4; i += blockDim.x)
                st4[(RG_COLS + kb) * W4 + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();
    if (warp == RG_THREADS / 32 - 1) {
        // ---------------- copy warp ----------------
        int t = 0;
        for (; t < nst; ++t) {
            const int s = t % RG_STAGES;
            if (t >= RG_STAGES) {
                int ok = 1;
                if (lane == 0)
                    ok = mbar_wait(smem_u32(&empty[s]), (uint32_t)((t / RG_STAGES - 1) & 1), RING_WAIT_NS) &&
                         !s_abort;
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    if (lane == 0) s_abort = 1;
                    break;
                }
            }
            if (lane == 0) {
                const int x = 2 * (int)(n0 + (int64_t)t * RG_ROWS);  // FP32 elements: a multiple of 128
                const uint32_t fb = smem_u32(&full[s]);
                const uint32_t st = sbase + (uint32_t)(s * RG_STAGE);
                mbar_arrive_expect(fb, (uint32_t)(bca + kb) * RG_COLBYTES);
                tensor_copy_2d(st, &tmA, x, col0, fb);
                tensor_copy_2d(st + RG_COLS * RG_COLBYTES, &tmB, x, 0, fb);
            }
            __syncwarp();
        }
        // every issued copy has landed before the CTA (and its shared memory) ends
        if (lane == 0)
            for (int u = max(0, t - RG_STAGES); u < t; ++u)
                mbar_wait(smem_u32(&full[u % RG_STAGES]), (uint32_t)((u / RG_STAGES) & 1), RING_WAIT_NS);
        return;
    }
    if (warp >= nact) return;
    // ---------------- compute warps ----------------
    const int a0 = 4 * warp;
    float v[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = 0.f;
    bool ok = true;
    for (int t = 0; t < nst; ++t) {
        const int s = t % RG_STAGES;
        if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((t / RG_STAGES) & 1), RING_WAIT_NS) || s_abort) {
            ok = false;
            break;
        }
        const unsigned char* st = rg_smem + s * RG_STAGE + lane * 16;
        float4 av[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = *reinterpret_cast<const float4*>(st + (a0 + a) * RG_COLBYTES);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float4 bv = *reinterpret_cast<const float4*>(st + (RG_COLS + b) * RG_COLBYTES);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float& re = v[(a * 8 + b) * 2];
                float& im = v[(a * 8 + b) * 2 + 1];
                re = fmaf(av[a].x, bv.x, re);
                re = fmaf(av[a].y, bv.y, re);
                re = fmaf(av[a].z, bv.z, re);
                re = fmaf(av[a].w, bv.w, re);
                im = fmaf(av[a].x, bv.y, im);
                im = fmaf(-av[a].y, bv.x, im);
                im = fmaf(av[a].z, bv.w, im);
                im = fmaf(-av[a].w, bv.z, im);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
    }
    if (!ok) {
        s_abort = 1;
        if (lane == 0) atomicExch(err, 1);
    }
    fold_half<32, 16>(v, lane);
    fold_half<16, 8>(v, lane);
    fold_half<8, 4>(v, lane);
    fold_half<4, 2>(v, lane);
    fold_half<2, 1>(v, lane);
    const int a = col0 + a0 + (lane >> 3), b = lane & 7;
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    if (a < ka && b < kb)
        partial[((int64_t)b * ka + a) * nblk + blk] = ok ? make_double2(v[0], v[1]) : make_double2(nanv, nanv);
}

// coef[a * 8 + b] = alpha H(a, b) in FP32 (H ka x kb column-major), zero for b >= kb
__global__ void ts_coef32_kernel(const double2* __restrict__ H, const int ka, const int kb,
                                 const double alpha, float2* __restrict__ coef) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ka * 8) return;
    const int a = i >> 3, b = i & 7;
    float2 c = make_float2(0.f, 0.f);
    if (b < kb) {
        const double2 h = H[(int64_t)b * ka + a];
        c = make_float2((float)(alpha * h.x), (float)(alpha * h.y));
    }
    coef[i] = c;
}

// B_b += sum_a A_a coef(a, b) (kb <= 8), the basis streamed through a ring of
// shared-memory stages by 2D tensor copies (TMA).
//
// CTA x: rows [64 x, 64 x + 64), two per lane.  The copy warp (warp 4, one
// lane) fills stage t with those rows of basis columns 16 t .. 16 t + 15 (a
// bca x 512-byte box of the basis's tensor map, bca = min(16, ka); rows past N and columns past
// ka arrive as zeros) and with their FP32 coefficients (16 x 8 float2, one
// contiguous bulk copy of up to 1 KB), both completing on full[t % S].
// Compute warp w takes columns 16 t + 4 w .. 16 t + 4 w + 3 of every stage,
// so its sums run over columns in order; after the last stage the four warp
// sums are added in warp order through shared memory (the ring, by then
// idle) and the read-modify-write of B follows.  Waits are bounded as in the
// Gram kernel.
constexpr int RU_ROWS = 64;
constexpr int RU_COLS = 16;
constexpr int RU_WARPS = 4;
constexpr int RU_STAGES = 3;
constexpr int RU_THREADS = (RU_WARPS + 1) * 32;
constexpr int RU_COLBYTES = RU_ROWS * 8;
constexpr int RU_STAGE = RU_COLS * RU_COLBYTES + RU_COLS * 8 * 8;
constexpr int RU_SMEM = RU_STAGES * RU_STAGE;
static_assert(RU_SMEM >= RU_WARPS * 8 * 32 * 16, "the ring holds the cross-warp reduction");

__global__ void __launch_bounds__(RU_THREADS, 7) ts_update32_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                   const int ka, const int bca,
                                                                   const float2* __restrict__ coef,
                                                                   float2* __restrict__ B, const int kb,
                                                                   const int64_t N, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char ru_smem[];
    __shared__ __align__(8) uint64_t full[RU_STAGES];
    __shared__ __align__(8) uint64_t empty[RU_STAGES];
    __shared__ volatile int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * RU_ROWS;
    const int rows = (int)min((int64_t)RU_ROWS, N - r0);
    const int nst = (ka + RU_COLS - 1) / RU_COLS;
    const uint32_t sbase = smem_u32(ru_smem);
    if (sbase & 127u) {  // tensor copies need 128-byte aligned stages: report, copy nothing
        if (threadIdx.x == 0) atomicExch(err, 1);
        return;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < RU_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), RU_WARPS);
        }
        mbar_init_fence();
        s_abort = 0;
    }
    // the whole ring starts at zero, so a stage's columns past ka (zero basis
    // columns from the copy, or never copied when ka < 16) meet finite
    // coefficients and the products need no guards; the proxy fence orders
    // these stores before the copies that later overwrite them
    for (int i = threadIdx.x; i < RU_SMEM / 16; i += blockDim.x)
        reinterpret_cast<float4*>(ru_smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (warp == RU_WARPS) {
        // ---------------- copy warp ----------------
        int t = 0;
        for (; t < nst; ++t) {
            const int s = t % RU_STAGES;
            if (t >= RU_STAGES) {
                int ok = 1;
                if (lane == 0)
                    ok = mbar_wait(smem_u32(&empty[s]), (uint32_t)((t / RU_STAGES - 1) & 1), RING_WAIT_NS) &&
                         !s_abort;
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    if (lane == 0) s_abort = 1;
                    break;
                }
            }
            if (lane == 0) {
                const int c0 = t * RU_COLS, cols = min(RU_COLS, ka - c0);
                const uint32_t fb = smem_u32(&full[s]);
                const uint32_t st = sbase + (uint32_t)(s * RU_STAGE);
                mbar_arrive_expect(fb, (uint32_t)(bca * RU_COLBYTES + cols * 64));
                tensor_copy_2d(st, &tmA, (int)(2 * r0), c0, fb);  // x: a multiple of 128 FP32 elements
                bulk_copy(st + RU_COLS * RU_COLBYTES, coef + (int64_t)c0 * 8, (uint32_t)cols * 64u, fb);
            }
            __syncwarp();
        }
        if (lane == 0)
            for (int u = max(0, t - RU_STAGES); u < t; ++u)
                mbar_wait(smem_u32(&full[u % RU_STAGES]), (uint32_t)((u / RU_STAGES) & 1), RING_WAIT_NS);
        return;
    }
    // ---------------- compute warps ----------------
    float acc[8][4];
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[b][0] = acc[b][1] = acc[b][2] = acc[b][3] = 0.f;
    bool ok = true;
    const bool live = 2 * lane < rows;
    for (int t = 0; t < nst; ++t) {
        const int s = t % RU_STAGES;
        if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((t / RU_STAGES) & 1), RING_WAIT_NS) || s_abort) {
            ok = false;
            break;
        }
        const unsigned char* st = ru_smem + s * RU_STAGE;
        const float4* c4 = reinterpret_cast<const float4*>(st + RU_COLS * RU_COLBYTES);
#pragma unroll
        for (int k = 0; k < RU_COLS / RU_WARPS; ++k) {
            const int c = RU_COLS / RU_WARPS * warp + k;
            {
                const float4 av = *reinterpret_cast<const float4*>(st + c * RU_COLBYTES + lane * 16);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 h = c4[c * 4 + q];
                    float* x = acc[2 * q];
                    float* y = acc[2 * q + 1];
                    x[0] = fmaf(av.x, h.x, fmaf(-av.y, h.y, x[0]));
                    x[1] = fmaf(av.x, h.y, fmaf(av.y, h.x, x[1]));
                    x[2] = fmaf(av.z, h.x, fmaf(-av.w, h.y, x[2]));
                    x[3] = fmaf(av.z, h.y, fmaf(av.w, h.x, x[3]));
                    y[0] = fmaf(av.x, h.z, fmaf(-av.y, h.w, y[0]));
                    y[1] = fmaf(av.x, h.w, fmaf(av.y, h.z, y[1]));
                    y[2] = fmaf(av.z, h.z, fmaf(-av.w, h.w, y[2]));
                    y[3] = fmaf(av.z, h.w, fmaf(av.w, h.z, y[3]));
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
    }
    if (!ok) {
        s_abort = 1;
        if (lane == 0) atomicExch(err, 1);
    }
    // cross-warp sums through the ring: every stage has been consumed by every
    // compute warp once all of them pass this barrier (the copy warp is not in it)
    asm volatile("bar.sync 1, %0;" ::"n"(RU_WARPS * 32) : "memory");
    float4* red = reinterpret_cast<float4*>(ru_smem);  // [warp][b][lane]
#pragma unroll
    for (int b = 0; b < 8; ++b) red[(warp * 8 + b) * 32 + lane] = make_float4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
    asm volatile("bar.sync 1, %0;" ::"n"(RU_WARPS * 32) : "memory");
    const bool abort = s_abort != 0;
#pragma unroll
    for (int k = 0; k < 8 / RU_WARPS; ++k) {
        const int b = warp * (8 / RU_WARPS) + k;
        if (b < kb && live) {
            float4 tsum = red[b * 32 + lane];
#pragma unroll
            for (int w = 1; w < RU_WARPS; ++w) {
                const float4 u = red[(w * 8 + b) * 32 + lane];
                tsum.x += u.x;
                tsum.y += u.y;
                tsum.z += u.z;
                tsum.w += u.w;
            }
            float4* o = reinterpret_cast<float4*>(B + (int64_t)b * N + r0 + 2 * lane);
            float4 x = *o;
            if (abort) {
                const float nanv = __int_as_float(0x7fc00000);
                x = make_float4(nanv, nanv, nanv, nanv);
            } else {
                x.x += tsum.x;
                x.y += tsum.y;
                x.z += tsum.z;
                x.w += tsum.w;
            }
            *o = x;
        }
    }
}

}  // namespace

int mbs_num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

void launch_sapply_f32(const SBlocks& B, int64_t N, int nrhs, const float2* x, const float2* y,
                       float2* z, int kmax, cudaStream_t st) {
    if (B.T == 0 || nrhs == 0) return;
    const size_t sm = (size_t)(kmax + 256) * SA_RC * sizeof(float2);
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(sapply_kernel<float2>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    sapply_kernel<float2><<<B.T, 256, sm, st>>>(B, N, nrhs, x, y, z, kmax);
    MBS_CHECK_LAUNCH();
}

void launch_sapply_f64(const SBlocks& B, int64_t N, int nrhs, const double2* x, const double2* y,
                       double2* z, int kmax, cudaStream_t st) {
    if (B.T == 0 || nrhs == 0) return;
    const size_t sm = (size_t)(kmax + 256) * SA_RC * sizeof(double2);
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(sapply_kernel<double2>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    sapply_kernel<double2><<<B.T, 256, sm, st>>>(B, N, nrhs, x, y, z, kmax);
    MBS_CHECK_LAUNCH();
}

template <typename V>
void launch_dots(const V* basis, int nvec, const V* w, int64_t N, int nrhs, double2* out,
                 double2* scratch, int nblk, cudaStream_t st) {
    if (nvec == 0) return;
    if ((int64_t)nblk * 256 * DOT_E < N)
        throw MbsError{MBS_ERR_ARG, "launch_dots: too few blocks for the vector length"};
    dim3 g((unsigned)nblk, (unsigned)nrhs);
    const size_t sm = (size_t)nvec * (256 / 32) * sizeof(double2);
    if (sm > 227 * 1024) throw MbsError{MBS_ERR_ARG, "launch_dots: too many basis vectors"};
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(dots_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm));
    dots_kernel<V><<<g, 256, sm, st>>>(basis, nvec, w, N, nrhs, scratch, nblk);
    MBS_CHECK_LAUNCH();
    dots_finish_kernel<<<nblocks((int64_t)nvec * nrhs * 32, 256), 256, 0, st>>>(scratch, nvec * nrhs, nblk, out);
    MBS_CHECK_LAUNCH();
}

template <typename V>
void launch_update(const V* basis, int nvec, const double2* h, V* w, int64_t N, int nrhs,
                   double sign, cudaStream_t st) {
    if (nvec == 0) return;
    const unsigned gx = (unsigned)std::min<int64_t>((N + 255) / 256, 4 * mbs_num_sms());
    dim3 g(gx, (unsigned)nrhs);
    const size_t sm = (size_t)nvec * sizeof(V);
    if (sm > 48 * 1024)
        MBS_CUDA_TRY(cudaFuncSetAttribute(update_kernel<V>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    update_kernel<V><<<g, 256, sm, st>>>(basis, nvec, h, w, N, nrhs, sign);
    MBS_CHECK_LAUNCH();
}

template <typename V>
void launch_scale(V* w, const double* inv, V* out, int64_t N, int nrhs, cudaStream_t st) {
    scale_kernel<V><<<nblocks(N * nrhs), 256, 0, st>>>(w, inv, out, N, nrhs);
    MBS_CHECK_LAUNCH();
}

template void launch_dots<float2>(const float2*, int, const float2*, int64_t, int, double2*,
                                  double2*, int, cudaStream_t);
template void launch_dots<double2>(const double2*, int, const double2*, int64_t, int, double2*,
                                   double2*, int, cudaStream_t);
template void launch_update<float2>(const float2*, int, const double2*, float2*, int64_t, int,
                                    double, cudaStream_t);
template void launch_update<double2>(const double2*, int, const double2*, double2*, int64_t, int,
                                     double, cudaStream_t);
template void launch_scale<float2>(float2*, const double*, float2*, int64_t, int, cudaStream_t);
template void launch_scale<double2>(double2*, const double*, double2*, int64_t, int, cudaStream_t);

void launch_norms64(const double2* x, int64_t N, int nrhs, double* out, double* scratch, int nblk,
                    cudaStream_t st) {
    dim3 g((unsigned)nblk, (unsigned)nrhs);
    norms_kernel<<<g, 256, 0, st>>>(x, N, nrhs, scratch, nblk);
    MBS_CHECK_LAUNCH();
    norms_finish_kernel<<<nblocks(nrhs, 64), 64, 0, st>>>(scratch, nrhs, nblk, out);
    MBS_CHECK_LAUNCH();
}

void launch_f64_to_f32_scaled(const double2* x, const double* scale, float2* y, int64_t N,
                              int nrhs, cudaStream_t st) {
    f64_to_f32_scaled_kernel<<<nblocks(N * nrhs), 256, 0, st>>>(x, scale, y, N, nrhs);
    MBS_CHECK_LAUNCH();
}

void launch_axpy_f32_into_f64(const float2* d, const double* scale, double2* x, int64_t N,
                              int nrhs, cudaStream_t st) {
    axpy_f32_into_f64_kernel<<<nblocks(N * nrhs), 256, 0, st>>>(d, scale, x, N, nrhs);
    MBS_CHECK_LAUNCH();
}

void launch_sub64(const double2* b, const double2* ax, double2* r, int64_t N, int nrhs,
                  cudaStream_t st) {
    sub64_kernel<<<nblocks(N * nrhs), 256, 0, st>>>(b, ax, r, N * nrhs);
    MBS_CHECK_LAUNCH();
}

template <typename V>
void launch_sub(const V* b, const V* ax, V* r, int64_t n, cudaStream_t st) {
    if (n == 0) return;
    sub_kernel<V><<<nblocks(n), 256, 0, st>>>(b, ax, r, n);
    MBS_CHECK_LAUNCH();
}
template void launch_sub<float2>(const float2*, const float2*, float2*, int64_t, cudaStream_t);
template void launch_sub<double2>(const double2*, const double2*, double2*, int64_t, cudaStream_t);

void launch_f32_to_f64(const float2* a, double2* b, int64_t n, cudaStream_t st) {
    if (n == 0) return;
    f32_to_f64_kernel<<<nblocks(n), 256, 0, st>>>(a, b, n);
    MBS_CHECK_LAUNCH();
}

void launch_f64_to_f32(const double2* a, float2* b, int64_t n, cudaStream_t st) {
    if (n == 0) return;
    f64_to_f32_kernel<<<nblocks(n), 256, 0, st>>>(a, b, n);
    MBS_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// tall-skinny block products (block GMRES)
// ---------------------------------------------------------------------------
namespace {
// the FP32 kernels need kb <= 8 and even N (16-byte loads of row pairs)
bool ts_fast(bool f32, int kb, int64_t N) { return f32 && kb <= 8 && (N % 2) == 0; }

// rows per Gram block of the FP32 kernel: a multiple of the stage, the grid at
// most two full waves of the two CTAs per SM that the ring's shared memory
// allows (a few CTAs of a third wave would cost a whole wave's time)
int64_t ts_gram32_chunk(int64_t N, int ka) {
    const int64_t tiles = (ka + RG_COLS - 1) / RG_COLS;
    const int64_t want = std::max<int64_t>(1, 4LL * mbs_num_sms() / tiles);  // CTAs <= 2 waves
    const int64_t rows = (N + want - 1) / want;
    return std::max<int64_t>(RG_ROWS, (rows + RG_ROWS - 1) / RG_ROWS * RG_ROWS);
}

// dynamic shared memory above 48 KB, set once per device and kernel (keeps the
// call out of captured CUDA graphs)
template <typename F>
void ring_smem_attr(F* kernel, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    MBS_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return;
    MBS_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.fetch_or(bit);
}
std::atomic<unsigned long long> g_gram_attr{0}, g_update_attr{0};

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    if (!fn) throw MbsError{MBS_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
    return fn;
}

// Tensor map over cols columns of N complex FP32 values at base (column c at
// base + c N): FP32 elements, dimensions {2 N, cols}, row stride 8 N bytes,
// box {128 elements (64 complex rows), boxcols columns}; outside it, zeros.
CUtensorMap column_map(const void* base, int64_t N, int cols, int boxcols) {
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * N), (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)(N * 8)};
    const cuuint32_t box[2] = {2 * RG_ROWS, (cuuint32_t)boxcols};
    const cuuint32_t step[2] = {1, 1};
    const CUresult r = encode_tiled()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides,
                                      box, step, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        throw MbsError{MBS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
    return m;
}

void check_aligned16(const void* p, const char* what) {
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0)
        throw MbsError{MBS_ERR_ARG, std::string(what) + ": operand not 16-byte aligned"};
}
}  // namespace

int ts_gram_blocks(int64_t N, int ka, int kb, bool f32) {
    if (ts_fast(f32, kb, N)) {
        const int64_t chunk = ts_gram32_chunk(N, ka);
        return (int)std::max<int64_t>(1, (N + chunk - 1) / chunk);
    }
    const int64_t tiles = (int64_t)((ka + TSG_A - 1) / TSG_A) * ((kb + TSG_B - 1) / TSG_B);
    const int64_t want = (8LL * mbs_num_sms() + tiles - 1) / tiles;
    return (int)std::max<int64_t>(1, std::min<int64_t>((N + 2047) / 2048, want));
}

template <typename V>
void launch_ts_gram(const V* A, int ka, const V* B, int kb, int64_t N, double2* C,
                    double2* scratch, int nblk, cudaStream_t st, int* err) {
    if (ka == 0 || kb == 0) return;
    if (N == 0) {
        MBS_CUDA_TRY(cudaMemsetAsync(C, 0, (size_t)ka * kb * sizeof(double2), st));
        return;
    }
    if (ts_fast(sizeof(V) == 8, kb, N)) {
        const int64_t chunk = ts_gram32_chunk(N, ka);
        if (nblk != (int)((N + chunk - 1) / chunk))
            throw MbsError{MBS_ERR_ARG, "launch_ts_gram: block count does not match ts_gram_blocks"};
        check_aligned16(A, "launch_ts_gram");
        check_aligned16(B, "launch_ts_gram");
        if (!err) throw MbsError{MBS_ERR_ARG, "launch_ts_gram: no device error flag"};
        ring_smem_attr(ts_gram32_kernel, RG_SMEM, g_gram_attr);
        const int bca = std::min(RG_COLS, ka);
        const CUtensorMap tmA = column_map(A, N, ka, bca), tmB = column_map(B, N, kb, kb);
        dim3 g((unsigned)nblk, (unsigned)((ka + RG_COLS - 1) / RG_COLS));
        ts_gram32_kernel<<<g, RG_THREADS, RG_SMEM, st>>>(tmA, ka, bca, tmB, kb, N, chunk, scratch, nblk, err);
    } else {
        dim3 g((unsigned)nblk, (unsigned)((ka + TSG_A - 1) / TSG_A), (unsigned)((kb + TSG_B - 1) / TSG_B));
        ts_gram_kernel<V><<<g, 256, 0, st>>>(A, ka, B, kb, N, scratch, nblk);
    }
    MBS_CHECK_LAUNCH();
    dots_finish_kernel<<<nblocks((int64_t)ka * kb * 32, 256), 256, 0, st>>>(scratch, ka * kb, nblk, C);
    MBS_CHECK_LAUNCH();
}

template <typename V>
void launch_ts_update(const V* A, int ka, const double2* H, double alpha, V* B, int kb, int64_t N,
                      cudaStream_t st, float2* coef, int* err) {
    if (ka == 0 || kb == 0 || N == 0) return;
    if (kb > 16) throw MbsError{MBS_ERR_ARG, "launch_ts_update: more than 16 columns"};
    if (coef && err && ts_fast(sizeof(V) == 8, kb, N)) {
        check_aligned16(A, "launch_ts_update");
        check_aligned16(B, "launch_ts_update");
        check_aligned16(coef, "launch_ts_update");
        ts_coef32_kernel<<<nblocks((int64_t)ka * 8, 256), 256, 0, st>>>(H, ka, kb, alpha, coef);
        MBS_CHECK_LAUNCH();
        ring_smem_attr(ts_update32_kernel, RU_SMEM, g_update_attr);
        const int bca = std::min(RU_COLS, ka);
        const CUtensorMap tmA = column_map(A, N, ka, bca);
        ts_update32_kernel<<<(unsigned)((N + RU_ROWS - 1) / RU_ROWS), RU_THREADS, RU_SMEM, st>>>(
            tmA, ka, bca, coef, reinterpret_cast<float2*>(B), kb, N, err);
    } else if (kb <= 8) {
        ts_update_kernel<V, 8><<<nblocks(N), 256, 0, st>>>(A, ka, H, alpha, B, kb, N);
    } else {
        ts_update_kernel<V, 16><<<nblocks(N), 256, 0, st>>>(A, ka, H, alpha, B, kb, N);
    }
    MBS_CHECK_LAUNCH();
}

template <typename V>
void launch_ts_trsm(V* B, int kb, int64_t N, const double2* R, cudaStream_t st) {
    if (kb == 0 || N == 0) return;
    if (kb > 16) throw MbsError{MBS_ERR_ARG, "launch_ts_trsm: more than 16 columns"};
    if (kb <= 8)
        ts_trsm_kernel<V, 8><<<nblocks(N), 256, 0, st>>>(B, kb, N, R);
    else
        ts_trsm_kernel<V, 16><<<nblocks(N), 256, 0, st>>>(B, kb, N, R);
    MBS_CHECK_LAUNCH();
}

template void launch_ts_gram<float2>(const float2*, int, const float2*, int, int64_t, double2*,
                                     double2*, int, cudaStream_t, int*);
template void launch_ts_gram<double2>(const double2*, int, const double2*, int, int64_t, double2*,
                                      double2*, int, cudaStream_t, int*);
template void launch_ts_update<float2>(const float2*, int, const double2*, double, float2*, int,
                                       int64_t, cudaStream_t, float2*, int*);
template void launch_ts_update<double2>(const double2*, int, const double2*, double, double2*, int,
                                        int64_t, cudaStream_t, float2*, int*);
template void launch_ts_trsm<float2>(float2*, int, int64_t, const double2*, cudaStream_t);
template void launch_ts_trsm<double2>(double2*, int, int64_t, const double2*, cudaStream_t);

void launch_chol_small(const double2* G, int s, double2* R, double* ok, cudaStream_t st) {
    if (s < 1 || s > 16) throw MbsError{MBS_ERR_ARG, "launch_chol_small: 1 <= s <= 16"};
    chol_small_kernel<<<1, 256, 0, st>>>(G, s, R, ok);
    MBS_CHECK_LAUNCH();
}
