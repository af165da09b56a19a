// FP32 G_hat matvec with the multiply-add on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory).
//
// y_i = sum_{j : body(j) != body(i)} phi_kappa(x_hat_i - x_hat_j) q_j (Sec. 1,
// eq. Gmtx-entries; zero diagonal blocks, Sec. 2.2 eq. mbody2) for a block of
// NR right-hand sides.
//
// Split of the work.  phi is a generated kernel, so it is evaluated on the
// FP32 pipe, once per point pair; the contraction of the generated tile with
// the right-hand sides is a dense product that runs on the tensor cores:
//   - a CTA owns 128 consecutive targets, one per thread, i.e. one lane of
//     tensor memory each (the M = 128 rows of the MMA);
//   - sources are taken in chunks of 16 (never straddling a body); per chunk
//     each thread writes its 16 phi values into tensor memory as the row of A,
//     [Re phi_0, Im phi_0, Re phi_1, ...] (K = 32), with A = A_hi + A_lo the
//     3xTF32 split (A_hi = A with the low 13 mantissa bits cleared);
//   - B (K = 32 x N = 2 NR) holds, per source j and right-hand side r,
//         row 2j:   [ Re q_jr | Im q_jr ],   row 2j+1: [ -Im q_jr | Re q_jr ],
//     so that D[:, r] = Re(phi q) and D[:, NR + r] = Im(phi q); B_hi and B_lo
//     are prepared once per matvec by g_umma_pack_kernel in the K-major
//     core-matrix layout of the tensor cores and streamed into a ring of
//     shared-memory stages by bulk copies (cp.async.bulk + mbarrier);
//   - one thread of the producer warp issues D += A_hi B_hi + A_hi B_lo +
//     A_lo B_hi (twelve kind::tf32 MMAs, K = 8 each) per chunk and commits
//     them to an mbarrier; the phi warps and the producer synchronise only
//     through mbarriers;
//   - A and D are single-buffered in tensor memory: a phi warp evaluates the
//     first half of the next chunk, then waits for the previous chunk's MMAs
//     before it overwrites A; D accumulates one source body (a "segment") at a
//     time, and when a body ends every thread adds its row of D into FP32
//     registers before it signals the next chunk, whose first MMA resets D,
//     so the tensor-core accumulation never runs over more than one body.
// Every wait is bounded (about 2 s): on a timeout the kernel sets *err, writes
// NaN to its outputs, waits (bounded) for its work in flight, frees its tensor
// memory and returns.
//
// Per point pair the FP32 pipe computes (2D, kappa r >= 8 for every pair of
// the body pair) s = |d|^2 + 2 D.d expanded as A_i + B_i . delta_j + |delta_j|^2
// with per-target, per-body constants, then r, r - R = s / (r + R), the fitted
// modulus/phase of H0 and exp(i phase); near body pairs take the per-pair
// branches of pair_phi_f32.
#include "bulk.cuh"
#include "phi32.cuh"

namespace {

constexpr int UM_T = 128;       // targets per CTA = TMEM lanes (phi warps 0-3)
constexpr int UM_THREADS = UM_T + 32;  // plus the producer / MMA warp
constexpr int UM_KC = 16;       // sources per chunk (K = 32: four kind::tf32 K-steps)
constexpr int UM_STAGES = 4;    // shared-memory ring of chunk records
constexpr int UM_COLS = 128;    // tensor-memory columns allocated per CTA
constexpr int UM_SMEM = 52 * 1024;  // dynamic shared memory: caps residency at 4 CTAs per SM,
                                    // so 4 x 128 columns never exceed the SM's 512
constexpr uint32_t TF32_MASK = 0xffffe000u;
constexpr unsigned long long UM_WAIT_NS = 2000000000ull;

template <int NR>
struct UmmaCfg {
    static constexpr int NM = 2 * NR;            // MMA N: [Re | Im] columns of D
    static constexpr int TILE = NM * 2 * UM_KC * 4;  // one B tile (N x K tf32) in bytes
    static constexpr int REC = 2 * TILE + UM_KC * 16;  // B_hi, B_lo, the sources as float4
    static constexpr uint32_t LBO = (NM / 8) * 128;    // K-direction core-matrix stride
    static constexpr uint32_t SBO = 128;               // N-direction core-matrix stride
    // kind::tf32, D f32, A/B tf32, both K-major, N = NM, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) |
                                      ((uint32_t)(NM >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
};

// word offset of B(n, k) inside a tile: core matrix (k / 4, n / 8) of 8 rows x 16 bytes
template <int NM>
__device__ __forceinline__ int b_word(int n, int k) {
    return ((k >> 2) * (NM / 8) + (n >> 3)) * 32 + (n & 7) * 4 + (k & 3);
}

// Wait for the phase of the given parity; false after UM_WAIT_NS.
__device__ __forceinline__ bool um_wait(uint32_t bar, uint32_t parity) { return mbar_wait(bar, parity, UM_WAIT_NS); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family; no swizzle
    return d;
}

__device__ __forceinline__ void umma_tf32(uint32_t dcol, uint32_t acol, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dcol),
        "r"(acol), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    mbar_arrive_expect(bar, bytes);
    bulk_copy(dst, src, bytes, bar);
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, "
        "%31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
        "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
        "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Chunk records of one block of NR right-hand sides: for chunk g of body
// sigma (sources off[sigma] + 8 (g - chunk_off[sigma]) + 0..7), B_hi and B_lo
// in the core-matrix layout and the sources' (delta, |delta|^2) as float4.
// Missing sources of a ragged last chunk have q = 0 and delta = 0.
template <int DIM, int NR>
__global__ void __launch_bounds__(128) g_umma_pack_kernel(const GLayout L, const int nrhs, const int r0,
                                                         const float2* __restrict__ q,
                                                         const int* __restrict__ chunk_off,
                                                         const int* __restrict__ chunk_body,
                                                         unsigned char* __restrict__ pack) {
    using C = UmmaCfg<NR>;
    const int64_t N = L.N;
    const int g = blockIdx.x;
    const int sig = chunk_body[g];
    const int64_t j0 = L.off[sig] + (int64_t)UM_KC * (g - chunk_off[sig]);
    const int cnt = (int)min((int64_t)UM_KC, L.off[sig + 1] - j0);
    unsigned char* rec = pack + (size_t)g * C::REC;
    uint32_t* bhi = reinterpret_cast<uint32_t*>(rec);
    uint32_t* blo = reinterpret_cast<uint32_t*>(rec + C::TILE);
    for (int idx = threadIdx.x; idx < UM_KC * NR; idx += blockDim.x) {
        const int j = idx / NR, r = idx - j * NR;
        float2 v = make_float2(0.f, 0.f);
        if (j < cnt && r0 + r < nrhs) v = q[(int64_t)(r0 + r) * N + j0 + j];
        const float e[4] = {v.x, v.y, -v.y, v.x};  // B(r, 2j), B(NR+r, 2j), B(r, 2j+1), B(NR+r, 2j+1)
        const int nn[4] = {r, NR + r, r, NR + r};
        const int kk[4] = {2 * j, 2 * j, 2 * j + 1, 2 * j + 1};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t hi = __float_as_uint(e[t]) & TF32_MASK;
            const int w = b_word<C::NM>(nn[t], kk[t]);
            bhi[w] = hi;
            blo[w] = __float_as_uint(e[t] - __uint_as_float(hi));
        }
    }
    if (threadIdx.x < UM_KC) {
        const int j = threadIdx.x;
        float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < cnt) {
            const float x = L.loc32[j0 + j], y = L.loc32[N + j0 + j];
            const float z = DIM == 3 ? L.loc32[2 * N + j0 + j] : 0.f;
            sv = make_float4(x, y, z, fmaf(x, x, fmaf(y, y, z * z)));
        }
        reinterpret_cast<float4*>(rec + 2 * C::TILE)[j] = sv;
    }
}

// phi of the point pair (target i, staged source sj) for a far body pair,
// with the per-(target, body) constants of the expanded form (see above).
// 2D: VF selects the x >= 64 fit of H0 (degree 2) for body pairs whose points
// are all that far apart, else the x >= 8 fit (degree 4) (modulus fits with
// the amplitude constant folded in, in K); glast is the last phase
// coefficient plus the body-pair phase.
template <int DIM, bool VF>
__device__ __forceinline__ float2 far_pair(const float4 sj, const float A0, const float Bx,
                                           const float By, const float Bz, const float R,
                                           const float R2, const float glast, const float phi0,
                                           const F32Const& K) {
    if (DIM == 2) {
        constexpr int DEG = VF ? MBS_F32_X64_DEG : MBS_F32_X8_DEG;
        const float* gc = VF ? c_f32_64G : c_f32_8G;
        const float* fcoef = VF ? K.f64a : K.f8a;
        const float s = fmaf(Bx, sj.x, fmaf(By, sj.y, A0 + sj.w));
        const float r2 = R2 + s;
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float dr = __fdividef(s, r + R);
        const float u = fmaf(VF ? K.c64 : K.c8, rinv, -1.f);
        float f = fcoef[0], gp = gc[0];
#pragma unroll
        for (int k = 1; k < DEG; ++k) {
            f = fmaf(f, u, fcoef[k]);
            gp = fmaf(gp, u, gc[k]);
        }
        f = fmaf(f, u, fcoef[DEG]);
        gp = fmaf(gp, u, glast);
        const float2 e = expi_f32(fmaf(K.kappa, dr, gp));
        const float amp = f * rsqrtf(r);
        return make_float2(amp * e.x, amp * e.y);
    } else {
        const float s = fmaf(Bx, sj.x, fmaf(By, sj.y, fmaf(Bz, sj.z, A0 + sj.w)));
        const float r2 = R2 + s;
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float dr = __fdividef(s, r + R);
        const float2 e = expi_f32(fmaf(K.kappa, dr, phi0));
        const float amp = 0.0795774715459476679f * rinv;  // 1 / (4 pi r)
        return make_float2(amp * e.x, amp * e.y);
    }
}

__device__ __forceinline__ void split_tf32(const float2 p, uint32_t& hx, uint32_t& hy, uint32_t& lx,
                                           uint32_t& ly) {
    hx = __float_as_uint(p.x) & TF32_MASK;
    hy = __float_as_uint(p.y) & TF32_MASK;
    lx = __float_as_uint(p.x - __uint_as_float(hx));
    ly = __float_as_uint(p.y - __uint_as_float(hy));
}

// Warp roles: warps 0-3 evaluate phi for targets 0-127 of the tile (warp w
// owns tensor-memory lanes 32w..32w+31) and read their rows of D back; warp 4
// (one lane) issues the bulk copies of the chunk records and the MMAs.
// Barriers: full[s] (copy into ring stage s landed), afull (all four phi warps
// have written A for the current chunk; count 4), mdone (the MMAs of the last
// issued chunk have completed).
// Tensor memory: A = columns [0, 64) ([hi | lo] of sources 4kk..4kk+3 at
// 16 kk), D = columns [64, 64 + 2 NR).  A and D are single-buffered: a phi warp
// waits for the previous chunk's MMAs before it overwrites A (by then it has
// evaluated half of the next chunk), and it reads a finished body's D back
// before it signals the next chunk, whose first MMA resets D.
template <int DIM, int NR>
__global__ void __launch_bounds__(UM_THREADS, 4) g_umma_kernel(const GLayout L, const F32Const K,
                                                               const int nrhs, const int r0,
                                                               const unsigned char* __restrict__ pack,
                                                               const int* __restrict__ chunk_off,
                                                               float2* __restrict__ part,
                                                               const int* __restrict__ split_body,
                                                               int* __restrict__ err) {
    using C = UmmaCfg<NR>;
    extern __shared__ __align__(1024) unsigned char um_smem[];
    __shared__ __align__(8) uint64_t bar_full[UM_STAGES];
    __shared__ __align__(8) uint64_t bar_afull;
    __shared__ __align__(8) uint64_t bar_mdone;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t N = L.N;
    const int T = L.T;

    // chunk sequence of this CTA: the chunks of its source split, minus the
    // chunks of a body that holds every target of the tile
    const int64_t t0 = (int64_t)blockIdx.x * UM_T, t1 = min(N, t0 + UM_T) - 1;
    const int bfirst = L.body[t0], blast = L.body[t1];
    const int sb0 = split_body[blockIdx.y], sb1 = split_body[blockIdx.y + 1];
    const int skipb = bfirst == blast ? bfirst : -1;
    const int c0 = chunk_off[sb0], c1 = chunk_off[sb1];
    int sk0 = 0, skn = 0;
    if (skipb >= sb0 && skipb < sb1) {
        sk0 = chunk_off[skipb];
        skn = chunk_off[skipb + 1] - sk0;
    }
    const int G = c1 - c0 - skn;

    const uint32_t smem0 = smem_u32(um_smem);
    const uint32_t b_afull = smem_u32(&bar_afull), b_mdone = smem_u32(&bar_mdone);
    if (tid == 0) {
        for (int st = 0; st < UM_STAGES; ++st)
            mbar_init(smem_u32(&bar_full[st]), 1);
        mbar_init(b_afull, 4);
        mbar_init(b_mdone, 1);
        mbar_init_fence();
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(UM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == UM_T / 32) {
        // ---------------- producer / MMA warp ----------------
        if (lane == 0) {
            auto load = [&](int gg) {
                const int x = c0 + gg;
                const int cid = (skn > 0 && x >= sk0) ? x + skn : x;
                const int st = gg % UM_STAGES;
                bulk_load(smem0 + st * C::REC, pack + (size_t)cid * C::REC, C::REC,
                          smem_u32(&bar_full[st]));
            };
            int issued = 0;
            for (; issued < min(UM_STAGES, G); ++issued) load(issued);
            int g = 0, stage = 0;
            bool ok = true, first = true;
            int cend = -1;  // last chunk of the current body (sequence index)
            int sig = sb0;
            for (; g < G; ++g) {
                if (g > cend) {  // next body of the sequence
                    while (sig == skipb || chunk_off[sig] == chunk_off[sig + 1]) ++sig;
                    cend = g + chunk_off[sig + 1] - chunk_off[sig] - 1;
                    ++sig;
                    first = true;
                }
                if (!um_wait(b_afull, (uint32_t)(g & 1)) || s_abort) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dcol = tmem + 64;
                const uint32_t sb = smem0 + stage * C::REC;
#pragma unroll
                for (int kk = 0; kk < 2 * UM_KC / 8; ++kk) {
                    const uint32_t koff = (uint32_t)kk * 2u * C::LBO;
                    const uint64_t dhi = sdesc(sb + koff, C::LBO, C::SBO);
                    const uint64_t dlo = sdesc(sb + C::TILE + koff, C::LBO, C::SBO);
                    umma_tf32(dcol, tmem + 16 * kk, dhi, C::IDESC, (first && kk == 0) ? 0u : 1u);
                    umma_tf32(dcol, tmem + 16 * kk, dlo, C::IDESC, 1u);
                    umma_tf32(dcol, tmem + 16 * kk + 8, dhi, C::IDESC, 1u);
                }
                umma_commit(b_mdone);
                first = false;
                if (issued < G) {
                    // this chunk's stage is refilled once its MMAs are done
                    if (!um_wait(b_mdone, (uint32_t)(g & 1))) {
                        ok = false;
                        ++g;
                        break;
                    }
                    load(issued);
                    ++issued;
                }
                stage = stage + 1 == UM_STAGES ? 0 : stage + 1;
            }
            if (!ok) {
                s_abort = 1;
                if (g > 0) um_wait(b_mdone, (uint32_t)((g - 1) & 1));  // bounded drain
            }
            for (int gg = g; gg < issued; ++gg)
                um_wait(smem_u32(&bar_full[gg % UM_STAGES]), (uint32_t)((gg / UM_STAGES) & 1));
        }
        __syncwarp();
    } else {
        // ---------------- phi warps ----------------
        const int64_t i = t0 + tid;
        const bool valid = i < N;
        const int tb = valid ? L.body[i] : -1;
        float di[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < DIM; ++c) di[c] = valid ? L.loc32[c * N + i] : 0.f;
        const float q2i = fmaf(di[0], di[0], fmaf(di[1], di[1], di[2] * di[2]));
        const uint32_t a_lane = tmem + ((uint32_t)(warp * 32) << 16);


        float accr[NR], acci[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) accr[r] = acci[r] = 0.f;
        auto read_d = [&]() {
            uint32_t v[16];
#pragma unroll
            for (int h = 0; h < C::NM / 16; ++h) {
                tmem_ld16(a_lane + 64 + 16 * h, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int col = 16 * h + e;
                    if (col < NR)
                        accr[col] += __uint_as_float(v[e]);
                    else
                        acci[col - NR] += __uint_as_float(v[e]);
                }
            }
        };

        // body-pair entries are fetched one body ahead so their latency hides
        // behind the previous body's chunks
        auto fetch = [&](int sg, float4& P, float& f0) {
            const bool a = sg < sb1 && valid && tb != sg;
            P = a ? L.pair[(int64_t)tb * T + sg] : make_float4(0.f, 0.f, 1.f, 1.f);
            f0 = (DIM == 3 && a) ? L.pair_phi0[(int64_t)tb * T + sg] : 0.f;
        };
        float4 P_next;
        float f0_next;
        fetch(sb0, P_next, f0_next);
        int g = 0, stage = 0;
        uint32_t fphase = 0;      // parity of the current pass over the ring
        bool pending = false;     // a finished body's D awaits read-back
        bool abort = false;
        for (int sig = sb0; sig < sb1 && !abort; ++sig) {
            float4 P = P_next;
            const float f0_cur = f0_next;
            fetch(sig + 1, P_next, f0_next);
            if (sig == skipb) continue;
            const int cb = chunk_off[sig], ce = chunk_off[sig + 1];
            if (cb == ce) continue;
            // per-target constants of the body pair (tb, sig)
            const bool act = valid && tb != sig;
            const int klast = (int)(L.off[sig + 1] - L.off[sig]) - UM_KC * (ce - cb - 1);
            float phi0 = 0.f;
            bool near = false;
            if (DIM == 2) {
                near = P.z < 0.f;
                P.z = fabsf(P.z);
                phi0 = P.w;
            } else {
                phi0 = f0_cur;
            }
            const bool wfast = __all_sync(0xffffffffu, act && !near);  // warp-uniform fast path
            // 2D: every pair of the body pair at kappa r >= 64 (phase stored minus 2 pi)
            const bool wvfar = DIM == 2 && __all_sync(0xffffffffu, act && !near && P.w < 0.f);
            const float R = DIM == 2 ? P.z : P.w;
            const float R2 = R * R;
            const float Dz = DIM == 3 ? P.z : 0.f;
            const float Bx = -2.f * (P.x + di[0]), By = -2.f * (P.y + di[1]), Bz = -2.f * (Dz + di[2]);
            const float A0 = fmaf(2.f * P.x, di[0], fmaf(2.f * P.y, di[1], fmaf(2.f * Dz, di[2], q2i)));
            const float glast = (wvfar ? c_f32_64G[MBS_F32_X64_DEG] : c_f32_8G[MBS_F32_X8_DEG]) + phi0;

            for (int c = cb; c < ce; ++c, ++g) {
                if (!um_wait(smem_u32(&bar_full[stage]), fphase)) s_abort = 1;
                const float4* src = reinterpret_cast<const float4*>(um_smem + stage * C::REC + 2 * C::TILE);
                const int cnt = c == ce - 1 ? klast : UM_KC;  // staged sources of this chunk
                // the fast path also takes a body's ragged last chunk: its padding
                // sources sit at delta = 0 (the source body's centre, away from
                // every target of another body, so phi is finite) and have q = 0
                // in B, so their products vanish
                const bool full_fast = wfast;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    // A columns of sources 8 half .. 8 half + 7:
                    // [hi re/im of 4 sources | their lo | hi of the next 4 | lo]
                    uint32_t av[32];
                    if (full_fast && wvfar) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float2 p = far_pair<DIM, true>(src[8 * half + j], A0, Bx, By, Bz, R, R2,
                                                                 glast, phi0, K);
                            const int o = (j >> 2) * 16 + (j & 3) * 2;
                            split_tf32(p, av[o], av[o + 1], av[o + 8], av[o + 9]);
                        }
                    } else if (full_fast) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float2 p = far_pair<DIM, false>(src[8 * half + j], A0, Bx, By, Bz, R, R2,
                                                                  glast, phi0, K);
                            const int o = (j >> 2) * 16 + (j & 3) * 2;
                            split_tf32(p, av[o], av[o + 1], av[o + 8], av[o + 9]);
                        }
                    } else {
#pragma unroll 1
                        for (int j = 0; j < 8; ++j) {
                            const int js = 8 * half + j;
                            const float4 sj = src[js];
                            float2 p = make_float2(0.f, 0.f);
                            if (js >= cnt) {
                                // padding of a ragged last chunk: q = 0 there
                            } else if (act && !near) {
                                p = wvfar ? far_pair<DIM, true>(sj, A0, Bx, By, Bz, R, R2, glast, phi0, K)
                                          : far_pair<DIM, false>(sj, A0, Bx, By, Bz, R, R2, glast, phi0, K);
                            } else if (act) {
                                const float dj[3] = {sj.x, sj.y, sj.z};
                                p = pair_phi_f32<DIM, false>(di, dj, P, R2, phi0, K);
                            }
                            uint32_t hx, hy, lx, ly;
                            split_tf32(p, hx, hy, lx, ly);
                            // keep the register array statically indexed
#pragma unroll
                            for (int jj = 0; jj < 8; ++jj) {
                                if (jj == j) {
                                    const int o = (jj >> 2) * 16 + (jj & 3) * 2;
                                    av[o] = hx;
                                    av[o + 1] = hy;
                                    av[o + 8] = lx;
                                    av[o + 9] = ly;
                                }
                            }
                        }
                    }
                    if (half == 0 && g > 0) {
                        // the previous chunk's MMAs are done: A is free, and a body
                        // that ended with that chunk has its D complete
                        if (!um_wait(b_mdone, (uint32_t)((g - 1) & 1))) s_abort = 1;
                        tc_fence_after();
                        if (pending) {
                            read_d();
                            pending = false;
                        }
                    }
                    __syncwarp();
                    tmem_st32(a_lane + 32 * half, av);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(b_afull);
                pending = c == ce - 1;
                stage = stage + 1 == UM_STAGES ? 0 : stage + 1;
                fphase ^= stage == 0 ? 1u : 0u;
                if (__shfl_sync(0xffffffffu, s_abort, 0)) {
                    abort = true;
                    ++g;
                    break;
                }
            }
        }
        if (!abort && G > 0) {
            // the MMAs of the last chunk have not been waited for yet
            if (!um_wait(b_mdone, (uint32_t)((G - 1) & 1))) abort = true;
            tc_fence_after();
            abort = __any_sync(0xffffffffu, abort);
            if (!abort && pending) read_d();
        }
        if (abort) s_abort = 1;
        float2* out = part + (int64_t)blockIdx.y * nrhs * N;
        if (valid) {
            const float nanv = __int_as_float(0x7fc00000);
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (r0 + r < nrhs)
                    out[(int64_t)(r0 + r) * N + i] = abort ? make_float2(nanv, nanv) : make_float2(accr[r], acci[r]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && s_abort) atomicExch(err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UM_COLS)
                     : "memory");
}

template <int DIM, int NR>
void launch_umma_block(const GLayout& L, const F32Const& K, const UmmaLayout& U, int nrhs, int r0,
                       const float2* q, float2* part, int nsplit, const int* sb, cudaStream_t st) {
    using C = UmmaCfg<NR>;
    if ((size_t)U.nchunks * C::REC > U.pack_bytes)
        throw MbsError{MBS_ERR_ARG, "launch_G_umma: pack buffer too small"};
    g_umma_pack_kernel<DIM, NR><<<(unsigned)U.nchunks, 128, 0, st>>>(L, nrhs, r0, q, U.chunk_off,
                                                                     U.chunk_body, U.pack);
    MBS_CHECK_LAUNCH();
    // once per device (keeps the call out of captured CUDA graphs)
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    MBS_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        MBS_CUDA_TRY(cudaFuncSetAttribute(g_umma_kernel<DIM, NR>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, UM_SMEM));
        attr_set.fetch_or(bit);
    }
    dim3 grid((unsigned)((L.N + UM_T - 1) / UM_T), (unsigned)nsplit);
    g_umma_kernel<DIM, NR><<<grid, UM_THREADS, UM_SMEM, st>>>(L, K, nrhs, r0, U.pack, U.chunk_off, part,
                                                        sb, U.err);
    MBS_CHECK_LAUNCH();
}

}  // namespace

size_t umma_pack_bytes(int64_t nchunks, int nrhs) {
    const int nr = nrhs >= 16 ? 16 : 8;
    return (size_t)nchunks * (nr == 16 ? UmmaCfg<16>::REC : UmmaCfg<8>::REC);
}

int umma_tile() { return UM_T; }

int umma_chunk() { return UM_KC; }

void launch_G_umma(const GLayout& L, const UmmaLayout& U, double kappa, int nrhs, const float2* q,
                   float2* part, int nsplit, const int* d_split_body, cudaStream_t st) {
    F32Const K = make_f32const(kappa);
    int r0 = 0;
    while (r0 < nrhs) {
        const int left = nrhs - r0;
        if (left >= 16) {
            if (L.dim == 2)
                launch_umma_block<2, 16>(L, K, U, nrhs, r0, q, part, nsplit, d_split_body, st);
            else
                launch_umma_block<3, 16>(L, K, U, nrhs, r0, q, part, nsplit, d_split_body, st);
            r0 += 16;
        } else {
            if (L.dim == 2)
                launch_umma_block<2, 8>(L, K, U, nrhs, r0, q, part, nsplit, d_split_body, st);
            else
                launch_umma_block<3, 8>(L, K, U, nrhs, r0, q, part, nsplit, d_split_body, st);
            r0 += 8;
        }
    }
}
