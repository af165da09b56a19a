// Block-masked all-pairs G_hat matvec and field evaluation.
//
// y_i = sum_{j : body(j) != body(i)} phi_kappa(x_hat_i - x_hat_j) q_j for every
// right-hand side (Sec. 1, eq. Gmtx-entries; the diagonal blocks of G_hat are
// zero, Sec. 2.2 eq. mbody2), and u(t) = sum_j phi(t - x_hat_j) q_j for
// arbitrary targets (Sec. 4.1, eq. out_skel).
//
// Launch shape: a CTA owns 256 consecutive targets (two per thread) and one
// contiguous range of source bodies (grid.y = source split).  Sources are
// staged body by body through shared memory and read as broadcasts; phi is
// evaluated once per pair and multiplied into every right-hand side held in
// registers.  Each split writes its own partial sums and a second kernel
// reduces them in a fixed order, so results do not depend on scheduling.
//
// FP32 path (inner solves): coordinates are split as x_hat = c_tau + delta
// with small local offsets delta.  Per body pair (tau, sigma) a table holds
// D = c_tau - c_sigma, R = |D| and the phase (kappa R + const) mod 2 pi,
// computed once in FP64.  Per point pair, with d = delta_i - delta_j,
//     s = 2 D.d + |d|^2,  r^2 = R^2 + s,  r - R = s / (r + R),
// so the phase kappa r = kappa R + kappa (r - R) keeps FP32 accuracy even when
// kappa r is in the thousands.
#include "bessel.cuh"
#include "common.cuh"
#include "phi32.cuh"

namespace {

constexpr int TPB = 128;  // threads per CTA
constexpr int TILE = 2 * TPB;  // targets per CTA
constexpr int SB = 128;  // sources staged per round

// Body-pair table.  In 2D a body pair whose closest points can come nearer
// than 8 / kappa (kappa r < 8, outside the range of the degree-4 fit) is
// marked by storing -R; its pairs take the per-pair branch to the x >= 3 fit
// or the power series.
__global__ void pair_table_kernel(int dim, int T, const double* __restrict__ c,
                                  const double* __restrict__ brad, double kappa,
                                  float4* __restrict__ pair, float* __restrict__ phi0) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)T * T) return;
    const int a = (int)(idx / T), b = (int)(idx % T);
    const double dx = c[3 * a] - c[3 * b], dy = c[3 * a + 1] - c[3 * b + 1];
    const double dz = dim == 3 ? c[3 * a + 2] - c[3 * b + 2] : 0.0;
    const double R = sqrt(dx * dx + dy * dy + dz * dz);
    if (dim == 2) {
        // phase in [0, 2 pi); body pairs whose points are all at kappa r >= 64
        // store the same phase minus 2 pi (negative): the FP32 kernels may then
        // use the shorter x >= 64 fit of H0
        double ph = fmod(kappa * R + 0.25 * MBS_PI, MBS_TWO_PI);
        const double gap = kappa * (R - brad[a] - brad[b]);
        const bool near = gap < 8.0 * (1.0 + 1e-6);
        if (gap >= 64.0 * (1.0 + 1e-6)) ph -= MBS_TWO_PI;
        pair[idx] = make_float4((float)dx, (float)dy, near ? -(float)R : (float)R, (float)ph);
    } else {
        pair[idx] = make_float4((float)dx, (float)dy, (float)dz, (float)R);
        phi0[idx] = (float)fmod(kappa * R, MBS_TWO_PI);
    }
}

// Sources jj < n of the staged chunk against this thread's TPT targets.
// MASKED: some targets are inactive (own body or past the end) and skip phi,
// and some body pairs may be near (per-pair choice of the H0 evaluation).
template <int DIM, int NR, int TPT, bool MASKED>
__device__ __forceinline__ void pair_loop_f32(const int n, const float (*s_loc)[SB],
                                              const float2* s_q, const float (&d)[TPT][DIM],
                                              const float4 (&P)[TPT], const float (&R2)[TPT],
                                              const float (&f0)[TPT], const bool (&act)[TPT],
                                              const F32Const& K, float2 (&a)[TPT][NR]) {
#pragma unroll 2
    for (int jj = 0; jj < n; ++jj) {
        float dj[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) dj[c] = s_loc[c][jj];
        float2 p[TPT];
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            if (MASKED)
                p[t] = act[t] ? pair_phi_f32<DIM, false>(d[t], dj, P[t], R2[t], f0[t], K)
                              : make_float2(0.f, 0.f);
            else
                p[t] = pair_phi_f32<DIM, true>(d[t], dj, P[t], R2[t], f0[t], K);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const float2 qq = s_q[jj * NR + r];
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                a[t][r].x = fmaf(p[t].x, qq.x, fmaf(-p[t].y, qq.y, a[t][r].x));
                a[t][r].y = fmaf(p[t].x, qq.y, fmaf(p[t].y, qq.x, a[t][r].y));
            }
        }
    }
}

// Targets of thread tid: tile + tid + t * TPB for t < TPT (coalesced loads/stores).
template <int DIM, int NR, int TPT>
__global__ void __launch_bounds__(TPB) g_f32_kernel(const GLayout L, const F32Const K,
                                                    const int nrhs, const int r0,
                                                    const float2* __restrict__ q,
                                                    float2* __restrict__ part,
                                                    const int* __restrict__ split_body) {
    __shared__ float s_loc[DIM][SB];
    __shared__ float2 s_q[SB * NR];
    const int64_t N = L.N;
    const int T = L.T;
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (TPB * TPT) + tid;
    bool valid[TPT];
    int tb[TPT];
    float d[TPT][DIM];
    float2 a[TPT][NR];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int64_t i = base + (int64_t)t * TPB;
        valid[t] = i < N;
        tb[t] = valid[t] ? L.body[i] : -1;
#pragma unroll
        for (int c = 0; c < DIM; ++c) d[t][c] = valid[t] ? L.loc32[c * N + i] : 0.f;
#pragma unroll
        for (int r = 0; r < NR; ++r) a[t][r] = make_float2(0.f, 0.f);
    }
    const int sb0 = split_body[blockIdx.y], sb1 = split_body[blockIdx.y + 1];
    for (int sb = sb0; sb < sb1; ++sb) {
        const int64_t js = L.off[sb], je = L.off[sb + 1];
        bool act[TPT];
        float4 P[TPT];
        float R2[TPT], f0[TPT];
        bool all = true, any = false;
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            act[t] = valid[t] && tb[t] != sb;  // zero diagonal blocks of G_hat
            any = any || act[t];
            P[t] = act[t] ? L.pair[(int64_t)tb[t] * T + sb] : make_float4(0.f, 0.f, 1.f, 1.f);
            f0[t] = (DIM == 3 && act[t]) ? L.pair_phi0[(int64_t)tb[t] * T + sb] : 0.f;
            if (DIM == 2) {  // a negative R marks a near body pair
                all = all && act[t] && P[t].z > 0.f;
                P[t].z = fabsf(P[t].z);
            } else {
                all = all && act[t];
            }
            const float R = DIM == 2 ? P[t].z : P[t].w;
            R2[t] = R * R;
        }
        for (int64_t jc = js; jc < je; jc += SB) {
            const int n = (int)min((int64_t)SB, je - jc);
            __syncthreads();
            if (tid < n) {
#pragma unroll
                for (int c = 0; c < DIM; ++c) s_loc[c][tid] = L.loc32[c * N + jc + tid];
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    s_q[tid * NR + r] =
                        (r0 + r < nrhs) ? q[(int64_t)(r0 + r) * N + jc + tid] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            if (all)
                pair_loop_f32<DIM, NR, TPT, false>(n, s_loc, s_q, d, P, R2, f0, act, K, a);
            else if (any)
                pair_loop_f32<DIM, NR, TPT, true>(n, s_loc, s_q, d, P, R2, f0, act, K, a);
        }
    }
    float2* out = part + (int64_t)blockIdx.y * nrhs * N;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (r0 + r < nrhs) {
#pragma unroll
            for (int t = 0; t < TPT; ++t)
                if (valid[t]) out[(int64_t)(r0 + r) * N + base + (int64_t)t * TPB] = a[t][r];
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 G_hat with the multiply-add on the tensor cores.
//
// phi is computed on the FP32 pipe exactly as above; the product of a tile of
// phi (8 targets x 4 sources) with the staged right-hand sides (4 sources x 8
// RHS) is one mma.m16n8k8 in the real embedding
//     [Yr; Yi] = [Phi_r  -Phi_i; Phi_i  Phi_r] [Qr; Qi]
// (rows 0-7: real parts of the 8 targets, rows 8-15: imaginary parts; k 0-3:
// real parts of the 4 sources' q, k 4-7: imaginary parts).  In the m16n8k8
// fragment layout, lane (g = lane/4, t = lane%4) holds A[g][t], A[g+8][t],
// A[g][t+4], A[g+8][t+4] = Phi_r, Phi_i, -Phi_i, Phi_r of ONE pair (target g,
// source t), so every lane evaluates exactly one phi per MMA.  FP32 accuracy
// comes from the 3xTF32 split x = hi + lo (hi = round-to-TF32(x)):
// phi q ~ hi(phi) hi(q) + hi(phi) lo(q) + lo(phi) hi(q), accumulated in FP32.
// ---------------------------------------------------------------------------
// High part of the split: x with its 13 low mantissa bits cleared (a TF32
// value; one logic op instead of a conversion on the XU pipe).  The low part
// x - hi is exact in FP32; the MMA reads its top 10 mantissa bits, so a
// product keeps ~2^-20 relative accuracy.
__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    return __float_as_uint(x) & 0xffffe000u;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int TC_WARPS = 4;
constexpr int TC_TW = 4;  // 8-target tiles per warp
constexpr int TC_TARGETS = TC_WARPS * TC_TW * 8;

template <int DIM, int NRB>
__global__ void __launch_bounds__(TC_WARPS * 32) g_tc_kernel(const GLayout L, const F32Const K,
                                                             const int nrhs, const int r0,
                                                             const float2* __restrict__ q,
                                                             float2* __restrict__ part,
                                                             const int* __restrict__ split_body) {
    // staged sources: local offsets and the TF32 split of q, [part][rb][source][rhs]
    // with part = {hi re, hi im, lo re, lo im}
    __shared__ float s_loc[DIM][SB];
    __shared__ uint32_t s_q[4][NRB][SB][8];
    const int64_t N = L.N;
    const int T = L.T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t tile0 = (int64_t)blockIdx.x * TC_TARGETS + warp * (TC_TW * 8);
    bool valid[TC_TW];
    int tb[TC_TW];
    float d[TC_TW][DIM];
    float acc[TC_TW][NRB][4];
#pragma unroll
    for (int k = 0; k < TC_TW; ++k) {
        const int64_t i = tile0 + 8 * k + g;
        valid[k] = i < N;
        tb[k] = valid[k] ? L.body[i] : -1;
#pragma unroll
        for (int c = 0; c < DIM; ++c) d[k][c] = valid[k] ? L.loc32[c * N + i] : 0.f;
#pragma unroll
        for (int rb = 0; rb < NRB; ++rb)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[k][rb][e] = 0.f;
    }
    const int sb0 = split_body[blockIdx.y], sb1 = split_body[blockIdx.y + 1];
    for (int sb = sb0; sb < sb1; ++sb) {
        const int64_t js = L.off[sb], je = L.off[sb + 1];
        bool act[TC_TW];
        float4 P[TC_TW];
        float R2[TC_TW], f0[TC_TW];
        bool fast_lane = true;
#pragma unroll
        for (int k = 0; k < TC_TW; ++k) {
            act[k] = valid[k] && tb[k] != sb;  // zero diagonal blocks of G_hat
            P[k] = act[k] ? L.pair[(int64_t)tb[k] * T + sb] : make_float4(0.f, 0.f, 1.f, 1.f);
            f0[k] = (DIM == 3 && act[k]) ? L.pair_phi0[(int64_t)tb[k] * T + sb] : 0.f;
            if (DIM == 2) {  // a negative R marks a near body pair
                fast_lane = fast_lane && act[k] && P[k].z > 0.f;
                P[k].z = fabsf(P[k].z);
            } else {
                fast_lane = fast_lane && act[k];
            }
            const float R = DIM == 2 ? P[k].z : P[k].w;
            R2[k] = R * R;
        }
        const bool fast = __all_sync(0xffffffffu, fast_lane);
        for (int64_t jc = js; jc < je; jc += SB) {
            const int n = (int)min((int64_t)SB, je - jc);
            const int n4 = (n + 3) & ~3;
            __syncthreads();
            for (int j = tid; j < n4; j += blockDim.x) {
                const bool sv = j < n;
#pragma unroll
                for (int c = 0; c < DIM; ++c) s_loc[c][j] = sv ? L.loc32[c * N + jc + j] : 0.f;
#pragma unroll
                for (int rb = 0; rb < NRB; ++rb)
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const int rr = r0 + rb * 8 + r;
                        const float2 v = (sv && rr < nrhs) ? q[(int64_t)rr * N + jc + j]
                                                           : make_float2(0.f, 0.f);
                        const uint32_t hr = f32_to_tf32(v.x), hi = f32_to_tf32(v.y);
                        s_q[0][rb][j][r] = hr;
                        s_q[1][rb][j][r] = hi;
                        s_q[2][rb][j][r] = __float_as_uint(v.x - __uint_as_float(hr));
                        s_q[3][rb][j][r] = __float_as_uint(v.y - __uint_as_float(hi));
                    }
            }
            __syncthreads();
            // the tensor cores accumulate one staged chunk (<= 128 sources) into a
            // fresh tile; the chunk sums are added on the FP32 pipe, so rounding in
            // the MMA accumulator does not grow with the number of sources
            float tacc[TC_TW][NRB][4];
#pragma unroll
            for (int k = 0; k < TC_TW; ++k)
#pragma unroll
                for (int rb = 0; rb < NRB; ++rb)
#pragma unroll
                    for (int e = 0; e < 4; ++e) tacc[k][rb][e] = 0.f;
            for (int c4 = 0; c4 < n4; c4 += 4) {
                const int j = c4 + t;
                const bool sv = j < n;
                float dj[DIM];
#pragma unroll
                for (int c = 0; c < DIM; ++c) dj[c] = s_loc[c][j];
                uint32_t bh0[NRB], bh1[NRB], bl0[NRB], bl1[NRB];
#pragma unroll
                for (int rb = 0; rb < NRB; ++rb) {
                    bh0[rb] = s_q[0][rb][j][g];
                    bh1[rb] = s_q[1][rb][j][g];
                    bl0[rb] = s_q[2][rb][j][g];
                    bl1[rb] = s_q[3][rb][j][g];
                }
#pragma unroll
                for (int k = 0; k < TC_TW; ++k) {
                    float2 ph;
                    if (fast)
                        ph = pair_phi_f32<DIM, true>(d[k], dj, P[k], R2[k], f0[k], K);
                    else
                        ph = (act[k] && sv) ? pair_phi_f32<DIM, false>(d[k], dj, P[k], R2[k], f0[k], K)
                                            : make_float2(0.f, 0.f);
                    __syncwarp();
                    const uint32_t hr = f32_to_tf32(ph.x), hi = f32_to_tf32(ph.y);
                    const uint32_t lr = __float_as_uint(ph.x - __uint_as_float(hr));
                    const uint32_t li = __float_as_uint(ph.y - __uint_as_float(hi));
                    const uint32_t ah[4] = {hr, hi, hi ^ 0x80000000u, hr};
                    const uint32_t al[4] = {lr, li, li ^ 0x80000000u, lr};
#pragma unroll
                    for (int rb = 0; rb < NRB; ++rb) {
                        mma_tf32(tacc[k][rb], ah, bh0[rb], bh1[rb]);
                        mma_tf32(tacc[k][rb], ah, bl0[rb], bl1[rb]);
                        mma_tf32(tacc[k][rb], al, bh0[rb], bh1[rb]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < TC_TW; ++k)
#pragma unroll
                for (int rb = 0; rb < NRB; ++rb)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[k][rb][e] += tacc[k][rb][e];
        }
    }
    // acc[k][rb] = {Yr(g, 2t), Yr(g, 2t+1), Yi(g, 2t), Yi(g, 2t+1)}
    float2* out = part + (int64_t)blockIdx.y * nrhs * N;
#pragma unroll
    for (int k = 0; k < TC_TW; ++k) {
        if (!valid[k]) continue;
        const int64_t i = tile0 + 8 * k + g;
#pragma unroll
        for (int rb = 0; rb < NRB; ++rb) {
            const int rr = r0 + rb * 8 + 2 * t;
            if (rr < nrhs) out[(int64_t)rr * N + i] = make_float2(acc[k][rb][0], acc[k][rb][2]);
            if (rr + 1 < nrhs) out[(int64_t)(rr + 1) * N + i] = make_float2(acc[k][rb][1], acc[k][rb][3]);
        }
    }
}

// FP64 path: world coordinates, no phase split.  Used for the FP64 operator,
// the refinement residual and field evaluation (tbody == nullptr: no mask).
template <int DIM, int NR>
__global__ void __launch_bounds__(TPB) g_f64_kernel(
    const int64_t Nt, const double* __restrict__ tgt, const int* __restrict__ tbody,
    const int64_t Ns, const double* __restrict__ src, const int64_t* __restrict__ soff,
    const double kappa, const int nrhs, const int r0, const double2* __restrict__ q,
    double2* __restrict__ part, const int* __restrict__ split_body) {
    __shared__ double s_x[DIM][SB];
    __shared__ double2 s_q[SB * NR];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * TILE + tid;
    const int64_t i1 = i0 + TPB;
    const bool v0 = i0 < Nt, v1 = i1 < Nt;
    const int tb0 = (v0 && tbody) ? tbody[i0] : -1;
    const int tb1 = (v1 && tbody) ? tbody[i1] : -1;
    double x0[DIM], x1[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        x0[c] = v0 ? tgt[c * Nt + i0] : 0.0;
        x1[c] = v1 ? tgt[c * Nt + i1] : 0.0;
    }
    double2 a0[NR], a1[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        a0[r] = make_double2(0.0, 0.0);
        a1[r] = make_double2(0.0, 0.0);
    }
    const int sb0 = split_body[blockIdx.y], sb1 = split_body[blockIdx.y + 1];
    for (int sb = sb0; sb < sb1; ++sb) {
        const int64_t js = soff[sb], je = soff[sb + 1];
        const bool act0 = v0 && tb0 != sb;
        const bool act1 = v1 && tb1 != sb;
        for (int64_t jc = js; jc < je; jc += SB) {
            const int n = (int)min((int64_t)SB, je - jc);
            __syncthreads();
            if (tid < n) {
#pragma unroll
                for (int c = 0; c < DIM; ++c) s_x[c][tid] = src[c * Ns + jc + tid];
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    s_q[tid * NR + r] = (r0 + r < nrhs) ? q[(int64_t)(r0 + r) * Ns + jc + tid]
                                                        : make_double2(0.0, 0.0);
            }
            __syncthreads();
            if (act0 || act1) {
                for (int jj = 0; jj < n; ++jj) {
                    double r20 = 0.0, r21 = 0.0;
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        const double sx = s_x[c][jj];
                        const double e0 = x0[c] - sx, e1 = x1[c] - sx;
                        r20 = fma(e0, e0, r20);
                        r21 = fma(e1, e1, r21);
                    }
                    double2 p0 = make_double2(0.0, 0.0), p1 = make_double2(0.0, 0.0);
                    if (act0) p0 = phi_f64_r2<DIM>(kappa, r20);
                    if (act1) p1 = phi_f64_r2<DIM>(kappa, r21);
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const double2 qq = s_q[jj * NR + r];
                        a0[r].x = fma(p0.x, qq.x, fma(-p0.y, qq.y, a0[r].x));
                        a0[r].y = fma(p0.x, qq.y, fma(p0.y, qq.x, a0[r].y));
                        a1[r].x = fma(p1.x, qq.x, fma(-p1.y, qq.y, a1[r].x));
                        a1[r].y = fma(p1.x, qq.y, fma(p1.y, qq.x, a1[r].y));
                    }
                }
            }
        }
    }
    double2* out = part + (int64_t)blockIdx.y * nrhs * Nt;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (r0 + r < nrhs) {
            if (v0) out[(int64_t)(r0 + r) * Nt + i0] = a0[r];
            if (v1) out[(int64_t)(r0 + r) * Nt + i1] = a1[r];
        }
    }
}

template <typename V>
__global__ void reduce_splits_kernel(const V* __restrict__ part, int nsplit, int64_t len,
                                     V* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    V acc = part[i];
    for (int s = 1; s < nsplit; ++s) {
        const V v = part[(int64_t)s * len + i];
        acc.x += v.x;
        acc.y += v.y;
    }
    y[i] = acc;
}

// Targets per thread of the FP32 kernel.  Measured on GB300 (1000-body 2D
// workload, 8 right-hand sides): 2 targets per thread 9.6 ms per launch,
// 4 targets 11.3 ms (146 registers, 3 CTAs per SM); 8 targets is slower still.
template <int NR>
constexpr int f32_tpt() {
    return 2;
}

template <int DIM, int NR>
void launch_f32_chunk(const GLayout& L, const F32Const& K, int nrhs, int r0,
                      const float2* q, float2* part, int nsplit, const int* sb, cudaStream_t st) {
    constexpr int TPT = f32_tpt<NR>();
    constexpr int tile = TPB * TPT;
    dim3 grid((unsigned)((L.N + tile - 1) / tile), (unsigned)nsplit);
    g_f32_kernel<DIM, NR, TPT><<<grid, TPB, 0, st>>>(L, K, nrhs, r0, q, part, sb);
}

template <int DIM>
void launch_f32_dim(const GLayout& L, const F32Const& K, int nrhs, int path,
                    const float2* q, float2* part, int nsplit, const int* sb, cudaStream_t st) {
    const bool tensor = path == 2;
    int r0 = 0;
    while (r0 < nrhs) {
        const int left = nrhs - r0;
        if (tensor && left > 8) {
            dim3 grid((unsigned)((L.N + TC_TARGETS - 1) / TC_TARGETS), (unsigned)nsplit);
            g_tc_kernel<DIM, 2><<<grid, TC_WARPS * 32, 0, st>>>(L, K, nrhs, r0, q, part, sb);
            r0 += 16;
        } else if (tensor) {
            dim3 grid((unsigned)((L.N + TC_TARGETS - 1) / TC_TARGETS), (unsigned)nsplit);
            g_tc_kernel<DIM, 1><<<grid, TC_WARPS * 32, 0, st>>>(L, K, nrhs, r0, q, part, sb);
            r0 += 8;
        } else if (left >= 16) {
            launch_f32_chunk<DIM, 16>(L, K, nrhs, r0, q, part, nsplit, sb, st);
            r0 += 16;
        } else if (left > 4) {
            launch_f32_chunk<DIM, 8>(L, K, nrhs, r0, q, part, nsplit, sb, st);
            r0 += 8;
        } else if (left > 2) {
            launch_f32_chunk<DIM, 4>(L, K, nrhs, r0, q, part, nsplit, sb, st);
            r0 += 4;
        } else if (left == 2) {
            launch_f32_chunk<DIM, 2>(L, K, nrhs, r0, q, part, nsplit, sb, st);
            r0 += 2;
        } else {
            launch_f32_chunk<DIM, 1>(L, K, nrhs, r0, q, part, nsplit, sb, st);
            r0 += 1;
        }
        MBS_CHECK_LAUNCH();
    }
}

template <int DIM, int NR>
void launch_f64_chunk(int64_t Nt, const double* tgt, const int* tbody, int64_t Ns,
                      const double* src, const int64_t* soff, double kappa, int nrhs, int r0,
                      const double2* q, double2* part, int nsplit, const int* sb, cudaStream_t st) {
    dim3 grid((unsigned)((Nt + TILE - 1) / TILE), (unsigned)nsplit);
    g_f64_kernel<DIM, NR><<<grid, TPB, 0, st>>>(Nt, tgt, tbody, Ns, src, soff, kappa, nrhs, r0, q,
                                               part, sb);
}

template <int DIM>
void launch_f64_dim(int64_t Nt, const double* tgt, const int* tbody, int64_t Ns,
                    const double* src, const int64_t* soff, double kappa, int nrhs,
                    const double2* q, double2* part, int nsplit, const int* sb, cudaStream_t st) {
    int r0 = 0;
    while (r0 < nrhs) {
        const int left = nrhs - r0;
        if (left > 4) {
            launch_f64_chunk<DIM, 8>(Nt, tgt, tbody, Ns, src, soff, kappa, nrhs, r0, q, part,
                                     nsplit, sb, st);
            r0 += 8;
        } else if (left > 2) {
            launch_f64_chunk<DIM, 4>(Nt, tgt, tbody, Ns, src, soff, kappa, nrhs, r0, q, part,
                                     nsplit, sb, st);
            r0 += 4;
        } else if (left == 2) {
            launch_f64_chunk<DIM, 2>(Nt, tgt, tbody, Ns, src, soff, kappa, nrhs, r0, q, part,
                                     nsplit, sb, st);
            r0 += 2;
        } else {
            launch_f64_chunk<DIM, 1>(Nt, tgt, tbody, Ns, src, soff, kappa, nrhs, r0, q, part,
                                     nsplit, sb, st);
            r0 += 1;
        }
        MBS_CHECK_LAUNCH();
    }
}

// Sec. 4.6: the field of body tau at a target inside its proxy surface from its
// reconstructed MFS sources, added to u.  One thread per (target, RHS).
template <int DIM>
__global__ void mfs_near_kernel(const int64_t M, const double* __restrict__ pts,
                                const int* __restrict__ tb, const MfsBody* __restrict__ bodies,
                                const double kappa, const double2* __restrict__ qmfs,
                                const int64_t Nm, double2* __restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= M) return;
    const int t = tb[i];
    if (t < 0) return;
    const MfsBody& B = bodies[t];
    double x[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) x[c] = pts[c * M + i] - B.c[c];
    const double2* q = qmfs + (int64_t)r * Nm + B.moff;
    double2 acc = u[(int64_t)r * M + i];
    for (int j = 0; j < B.n; ++j) {
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double yw = 0.0;
#pragma unroll
            for (int b = 0; b < DIM; ++b) yw = fma(B.R[3 * a + b], B.y[b * B.n + j], yw);
            const double e = x[a] - yw;
            r2 = fma(e, e, r2);
        }
        const double2 p = phi_f64_r2<DIM>(kappa, r2);
        acc = cadd(acc, cmul(p, q[j]));
    }
    u[(int64_t)r * M + i] = acc;
}

}  // namespace

// Timing event on st: inside a stream capture it must become an external
// event-record node of the graph (recorded on every replay); outside a capture
// the external flag is not allowed.
void record_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MBS_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusActive)
        MBS_CUDA_TRY(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal));
    else
        MBS_CUDA_TRY(cudaEventRecord(e, st));
}

void launch_pair_table(int dim, int T, const double* d_centres, const double* d_brad,
                       double kappa, float4* pair, float* pair_phi0, cudaStream_t st) {
    const int64_t n = (int64_t)T * T;
    if (n == 0) return;
    pair_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dim, T, d_centres, d_brad,
                                                                   kappa, pair, pair_phi0);
    MBS_CHECK_LAUNCH();
}

void launch_G_f32(const GLayout& L, double kappa, int nrhs, const float2* q, float2* y,
                  float2* part, int nsplit, const int* d_split_body, cudaStream_t st,
                  cudaEvent_t ev0, cudaEvent_t ev1, int mac_path, const UmmaLayout* U) {
    if (L.N == 0 || nrhs == 0) return;
    const F32Const K = make_f32const(kappa);
    // mac_path: 1 FP32 pipe, 2 mma.sync tensor-core multiply-add (3xTF32), 3 the
    // tcgen05 kernel of gumma.cu (the caller picks the path; 0 means 1 here).
    const int path = mac_path == 0 ? 1 : mac_path;
    if (ev0) record_event(ev0, st);
    if (path == 3) {
        if (!U) throw MbsError{MBS_ERR_ARG, "launch_G_f32: the tcgen05 path needs its chunk layout"};
        launch_G_umma(L, *U, kappa, nrhs, q, part, nsplit, d_split_body, st);
    } else if (L.dim == 2) {
        launch_f32_dim<2>(L, K, nrhs, path, q, part, nsplit, d_split_body, st);
    } else {
        launch_f32_dim<3>(L, K, nrhs, path, q, part, nsplit, d_split_body, st);
    }
    if (ev1) record_event(ev1, st);
    const int64_t len = L.N * nrhs;
    reduce_splits_kernel<float2><<<(unsigned)((len + 255) / 256), 256, 0, st>>>(part, nsplit, len, y);
    MBS_CHECK_LAUNCH();
}

void launch_G_f64(const GLayout& L, double kappa, int nrhs, const double2* q, double2* y,
                  double2* part, int nsplit, const int* d_split_body, cudaStream_t st,
                  cudaEvent_t ev0, cudaEvent_t ev1) {
    if (L.N == 0 || nrhs == 0) return;
    if (ev0) record_event(ev0, st);
    if (L.dim == 2)
        launch_f64_dim<2>(L.N, L.xw64, L.body, L.N, L.xw64, L.off, kappa, nrhs, q, part, nsplit,
                          d_split_body, st);
    else
        launch_f64_dim<3>(L.N, L.xw64, L.body, L.N, L.xw64, L.off, kappa, nrhs, q, part, nsplit,
                          d_split_body, st);
    if (ev1) record_event(ev1, st);
    launch_reduce_splits64(part, nsplit, L.N * nrhs, y, st);
}

void launch_reduce_splits64(const double2* part, int nsplit, int64_t len, double2* y, cudaStream_t st) {
    reduce_splits_kernel<double2><<<(unsigned)((len + 255) / 256), 256, 0, st>>>(part, nsplit, len, y);
    MBS_CHECK_LAUNCH();
}

// Field evaluation at arbitrary targets: the FP64 kernel, with an optional
// per-target body whose skeleton sources are left out (near targets, whose own
// body is represented by its MFS sources instead).
void launch_field_f64(const GLayout& L, double kappa, int64_t M, const double* tgt, int nrhs,
                      const double2* q, double2* u, double2* part, int nsplit,
                      const int* d_split_body, cudaStream_t st, const int* tbody) {
    if (M == 0 || nrhs == 0) return;
    if (L.dim == 2)
        launch_f64_dim<2>(M, tgt, tbody, L.N, L.xw64, L.off, kappa, nrhs, q, part, nsplit,
                          d_split_body, st);
    else
        launch_f64_dim<3>(M, tgt, tbody, L.N, L.xw64, L.off, kappa, nrhs, q, part, nsplit,
                          d_split_body, st);
    const int64_t len = M * nrhs;
    reduce_splits_kernel<double2><<<(unsigned)((len + 255) / 256), 256, 0, st>>>(part, nsplit, len, u);
    MBS_CHECK_LAUNCH();
}

void launch_mfs_near(int dim, int64_t M, const double* pts, const int* tb, const MfsBody* bodies,
                     double kappa, int nrhs, const double2* qmfs, int64_t Nm, double2* u,
                     cudaStream_t st) {
    if (M == 0 || nrhs == 0) return;
    dim3 g((unsigned)((M + 127) / 128), (unsigned)nrhs);
    if (dim == 2)
        mfs_near_kernel<2><<<g, 128, 0, st>>>(M, pts, tb, bodies, kappa, qmfs, Nm, u);
    else
        mfs_near_kernel<3><<<g, 128, 0, st>>>(M, pts, tb, bodies, kappa, qmfs, Nm, u);
    MBS_CHECK_LAUNCH();
}
