// C ABI of the multibody scattering library: context, S build driver,
// layout, right-hand side, operator, GMRES / GMRES-IR solve and field
// evaluation.  See include/mbs.h for the contract of every call.
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>


#include "blsq.h"
#include "common.cuh"
#include "sbuild.cuh"

std::atomic<long long> g_mbs_launches{0};

namespace {

using cd = std::complex<double>;

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

struct ShapeHost {
    int m = 0, n = 0, p = 0, kfix = 0;
    double eps = 0, proxy_radius = 0, bound_radius = 0;
    std::vector<double> x, y, z;  // SoA local coordinates
    bool used = false;
    int k = 0, rankA = 0, rankB = 0, rankS = 0, sweepsA = 0;
    double eps_ach = 0;
    double snorm = 0;  // Frobenius norm of S
    std::vector<int> skel;
    bool rhs_ok = true;  // false after a skeleton was injected without its W
    bool injected = false;  // scattering data replaced by mbs_inject_scattering
    // device (owned by the context allocation list)
    double *dx = nullptr, *dy = nullptr, *dz = nullptr;
    double2 *AU = nullptr, *Zs = nullptr, *C = nullptr, *S64 = nullptr, *W = nullptr,
            *JA = nullptr, *FA = nullptr;
    float2* S32 = nullptr;
};

// One captured block-GMRES step (operator, block Gram-Schmidt, CholQR2 and the
// readback), replayed by cudaGraphLaunch.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;  // G_hat timing inside the graph (profiling)
    int prec = 0;                             // 0: FP32 G_hat, 1: FP64
    long long launches = 0;                   // library kernels in the graph
};

}  // namespace

struct mbs_ctx {
    int dim = 2;
    double kappa = 1.0;
    mbs_options opt{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::mutex mu;
    std::string err;

    // geometry
    std::vector<ShapeHost> shapes;
    std::vector<mbs_body> bodies;
    int T = 0;
    int64_t N = 0, Mtot = 0, Nm = 0;  // skeleton points, collocation points, MFS sources
    // FP64-accurate G_hat in solves under fp64_kernel = 2: double-float when its
    // error (~1e-14 relative per unit of ||S||) stays below a tenth of tol
    double snorm_rms = 0.0;  // root mean square over bodies of the Frobenius norm of S
    bool in_solve = false;
    bool df_active = false;
    std::vector<int64_t> off, voff;
    std::vector<int> kb;  // per-body skeleton count
    std::vector<double> skel_world;  // dim * N SoA
    bool built = false;
    bool layout_dirty = false;  // injected scattering data not yet in the device layout
    int kmax = 0, mmax = 0, nmax = 0;

    // device layout
    int* d_body = nullptr;
    int64_t* d_off = nullptr;
    float* d_loc32 = nullptr;
    double* d_xw64 = nullptr;
    float4* d_pair = nullptr;
    float* d_pair_phi0 = nullptr;
    double* d_centres = nullptr;
    // tensor-core G_hat: source chunks of 8 within a body
    int64_t nchunks = 0;
    int* d_chunk_off = nullptr;   // [T+1]
    int* d_chunk_body = nullptr;  // [nchunks]
    int* d_err = nullptr;         // set by a bounded device wait that ran out
    int* d_k = nullptr;
    const double2** d_S64p = nullptr;
    const float2** d_S32p = nullptr;
    RhsBody* d_rhsb = nullptr;
    MfsBody* d_mfsb = nullptr;
    std::map<std::pair<int64_t, int>, int*> split_cache;  // (targets, nsplit) -> split_body


    // live timing of the G_hat kernels (mbs_profile)
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev32, ev64;

    // pinned host staging for the per-step readback of block GMRES
    double2* pinned = nullptr;
    size_t pinned_n = 0;

    // CUDA graphs of block-GMRES steps, keyed by (vector type, s, step, restart,
    // buffer addresses); dropped whenever a buffer they use may move
    std::map<std::array<int64_t, 8>, StepGraph> graphs;
    bool capturing = false;
    bool graphs_off = false;  // a capture failed on this context: run steps directly
    cudaEvent_t cap_e0 = nullptr, cap_e1 = nullptr;
    double graph_ms[2] = {0.0, 0.0};  // profiled G_hat time of replayed steps (FP32, FP64)
    int last_path = 0, last_nsplit = 0;  // launch shape of the latest FP32 G_hat
    int last_sbuild_threads = 0;         // CTA size of the last S build
    long long graph_n[2] = {0, 0};

    // allocations
    std::vector<void*> geom_allocs;  // freed on rebuild
    std::unordered_map<std::string, DevBuf> bufs;
    size_t bytes_held = 0;
    std::map<void*, size_t> sizes;
};

namespace {

void* dalloc(mbs_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->opt.hbm_budget && c->bytes_held + bytes > c->opt.hbm_budget)
        throw MbsError{MBS_ERR_NOMEM, "HBM budget exceeded (" + std::to_string(c->bytes_held + bytes) +
                                          " > " + std::to_string(c->opt.hbm_budget) + " bytes)"};
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw MbsError{MBS_ERR_NOMEM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                          "): " + cudaGetErrorString(e)};
    }
    c->bytes_held += bytes;
    c->sizes[p] = bytes;
    return p;
}

void dfree(mbs_ctx* c, void* p) {
    if (!p) return;
    auto it = c->sizes.find(p);
    if (it != c->sizes.end()) {
        c->bytes_held -= it->second;
        c->sizes.erase(it);
    }
    cudaFree(p);
}

template <typename T>
T* galloc(mbs_ctx* c, size_t count) {
    T* p = static_cast<T*>(dalloc(c, count * sizeof(T)));
    c->geom_allocs.push_back(p);
    return p;
}

void clear_graphs(mbs_ctx* c) {
    if (c->graphs.empty()) return;
    if (c->st) cudaStreamSynchronize(c->st);
    for (auto& kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.e0) cudaEventDestroy(kv.second.e0);
        if (kv.second.e1) cudaEventDestroy(kv.second.e1);
    }
    c->graphs.clear();
}

template <typename T>
T* scratch(mbs_ctx* c, const std::string& name, size_t count) {
    DevBuf& b = c->bufs[name];
    const size_t need = count * sizeof(T);
    if (b.n < need) {
        if (c->capturing) throw MbsError{MBS_ERR_STATE, "buffer growth inside a graph capture"};
        clear_graphs(c);  // captured steps may refer to the old buffer
        if (b.p) {
            MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
            dfree(c, b.p);
            b.p = nullptr;
            b.n = 0;
        }
        b.p = dalloc(c, need);
        b.n = need;
    }
    return static_cast<T*>(b.p);
}

void free_geometry(mbs_ctx* c) {
    clear_graphs(c);
    if (c->st) cudaStreamSynchronize(c->st);
    for (void* p : c->geom_allocs) dfree(c, p);
    c->geom_allocs.clear();
    for (auto& kv : c->split_cache) dfree(c, kv.second);
    c->split_cache.clear();
    c->shapes.clear();
    c->bodies.clear();
    c->built = false;
    c->T = 0;
    c->N = 0;
    c->d_body = nullptr;
    c->d_off = nullptr;
    c->d_loc32 = nullptr;
    c->d_xw64 = nullptr;
    c->d_pair = nullptr;
    c->d_pair_phi0 = nullptr;
    c->d_centres = nullptr;
    c->nchunks = 0;
    c->d_chunk_off = nullptr;
    c->d_chunk_body = nullptr;
    c->d_k = nullptr;
    c->d_S64p = nullptr;
    c->d_S32p = nullptr;
    c->d_rhsb = nullptr;
    c->d_mfsb = nullptr;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller's complex input array (copied if it lives on the host).
const double2* in_dev(mbs_ctx* c, const double* p, size_t ncomplex, const char* name) {
    if (is_device_ptr(p)) return reinterpret_cast<const double2*>(p);
    double2* d = scratch<double2>(c, name, ncomplex);
    MBS_CUDA_TRY(cudaMemcpyAsync(d, p, ncomplex * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    return d;
}
const double* in_dev_real(mbs_ctx* c, const double* p, size_t n, const char* name) {
    if (is_device_ptr(p)) return p;
    double* d = scratch<double>(c, name, n);
    MBS_CUDA_TRY(cudaMemcpyAsync(d, p, n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    return d;
}

struct OutBuf {
    double* user;
    double2* dev;
    size_t n;
    bool host;
};
OutBuf out_dev(mbs_ctx* c, double* p, size_t ncomplex, const char* name) {
    OutBuf o{p, nullptr, ncomplex, !is_device_ptr(p)};
    o.dev = o.host ? scratch<double2>(c, name, ncomplex) : reinterpret_cast<double2*>(p);
    return o;
}
void finish_out(mbs_ctx* c, const OutBuf& o) {
    if (o.host)
        MBS_CUDA_TRY(cudaMemcpyAsync(o.user, o.dev, o.n * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
    MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
}

void refresh_layout(mbs_ctx* c);

// A built context with an up-to-date device layout (injections are applied
// lazily, so many shapes can be injected at the cost of one layout rebuild).
void require_built(mbs_ctx* c) {
    if (!c->built) throw MbsError{MBS_ERR_STATE, "scattering matrices not built"};
    if (c->layout_dirty) {
        refresh_layout(c);
        c->layout_dirty = false;
    }
}

// ---------------------------------------------------------------------------
// launch-shape helpers
// ---------------------------------------------------------------------------
int max_nsplit(const mbs_ctx* c) { return std::max(1, std::min(c->T, 64)); }

int choose_nsplit(mbs_ctx* c, int64_t ntargets) {
    if (c->opt.tile_override > 0) return std::min(c->opt.tile_override, std::max(1, c->T));
    const int64_t tiles = (ntargets + 255) / 256;
    const int64_t want = 16LL * mbs_num_sms();
    int64_t ns = (want + tiles - 1) / std::max<int64_t>(1, tiles);
    ns = std::max<int64_t>(1, std::min<int64_t>(ns, max_nsplit(c)));
    return (int)ns;
}

// split_body[s] = first source body of split s, balanced by skeleton counts.
int* split_table(mbs_ctx* c, int ns) {
    auto key = std::make_pair((int64_t)ns, 0);
    auto it = c->split_cache.find(key);
    if (it != c->split_cache.end()) return it->second;
    std::vector<int> sb(ns + 1, c->T);
    sb[0] = 0;
    int b = 0;
    for (int s = 1; s < ns; ++s) {
        const int64_t target = (c->N * s) / ns;
        while (b < c->T && c->off[b] < target) ++b;
        sb[s] = std::max(sb[s - 1], std::min(b, c->T));
    }
    sb[ns] = c->T;
    int* d = static_cast<int*>(dalloc(c, sb.size() * sizeof(int)));
    MBS_CUDA_TRY(cudaMemcpy(d, sb.data(), sb.size() * sizeof(int), cudaMemcpyHostToDevice));
    c->split_cache[key] = d;
    return d;
}

int* split_for(mbs_ctx* c, int64_t ntargets, int* nsplit_out) {
    const int ns = choose_nsplit(c, ntargets);
    *nsplit_out = ns;
    return split_table(c, ns);
}

GLayout glayout(mbs_ctx* c) {
    GLayout L;
    L.dim = c->dim;
    L.T = c->T;
    L.N = c->N;
    L.body = c->d_body;
    L.off = c->d_off;
    L.loc32 = c->d_loc32;
    L.xw64 = c->d_xw64;
    L.pair = c->d_pair;
    L.pair_phi0 = c->d_pair_phi0;
    return L;
}

SBlocks sblocks(mbs_ctx* c) {
    SBlocks B;
    B.T = c->T;
    B.k = c->d_k;
    B.off = c->d_off;
    B.S64 = c->d_S64p;
    B.S32 = c->d_S32p;
    return B;
}

cudaEvent_t take_event(mbs_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    MBS_CUDA_TRY(cudaEventCreate(&e));
    return e;
}

// The FP32 G_hat kernel for the options: 1 FP32 pipe, 2 mma.sync tensor-core
// multiply-add, 3 tcgen05 tensor-core multiply-add (4 or more right-hand
// sides; fewer take the FP32 pipe).  Automatic choice (0): tcgen05, measured
// on GB300 at 6.8 ms per launch against 9.5 ms on the FP32 pipe and 10.8 ms
// with mma.sync (1000-body 2D workload, 8 right-hand sides).
int g32_path(const mbs_ctx* c, int nrhs) {
    const int p = c->opt.mac_path == 0 ? 3 : c->opt.mac_path;
    return (p == 3 && nrhs < 4) ? 1 : p;
}

int* device_err(mbs_ctx* c) {
    if (!c->d_err) {
        c->d_err = static_cast<int*>(dalloc(c, sizeof(int)));
        MBS_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
    }
    return c->d_err;
}

// ---------------------------------------------------------------------------
// Launch-shape autotuner of the FP32 G_hat matvec.  The first FP32 matvec of a
// problem class (device, dimension, right-hand sides, kernel option and the
// power-of-two buckets of N and of the body count) times every candidate
// shape on the caller's own data: the kernel path (tcgen05 or FP32 pipe,
// unless mac_path fixes it) times the source-split count (the heuristic's,
// half and double).  The fastest is kept in a process-wide table, so every
// later matvec of that class, in any context, uses the same shape; a solve
// therefore gives the same result alone and next to other solves.
// mbs_options.autotune = 0 (or a tile_override) keeps the heuristic shape.
// ---------------------------------------------------------------------------
struct Shape32 {
    int path;
    int nsplit;
};

// Threads per CTA of the persistent S build (128, 256 or 512).  The build is
// bound by GB300's FP64 pipe: on the 2000-ellipsoid and 10,000-body workloads
// the three sizes measured within 2 % of each other (22.0-22.5 s and
// 9.6-9.8 s), so the default is a fixed 256 and the probe below, which costs
// about half a build per new size class, runs only with sbuild_threads = -1.
// The probe times each candidate on a prefix of the jobs large enough to fill
// the GPU with the smallest CTAs and keeps the fastest in a process-wide table
// keyed by device, dimension and the power-of-two buckets of the largest
// matrix dimension and of the shape count (the probe's outputs are
// overwritten by the full build).  Different CTA sizes sum in different
// orders; the table keeps every later build of a class reproducible.
std::mutex g_sb_tune_mu;
std::map<std::array<int, 4>, int> g_sb_tune;

int log2_bucket(int64_t v);

int sbuild_threads(mbs_ctx* c, SBuildJob* d_jobs, int nj, int* d_counter, int rows_max) {
    if (c->opt.sbuild_threads > 0) return c->opt.sbuild_threads;
    if (c->opt.sbuild_threads == 0 || !c->opt.autotune) return 256;
    int dev = 0;
    MBS_CUDA_TRY(cudaGetDevice(&dev));
    const std::array<int, 4> key{dev, c->dim, log2_bucket(rows_max), log2_bucket(nj)};
    std::lock_guard<std::mutex> lk(g_sb_tune_mu);
    auto it = g_sb_tune.find(key);
    if (it != g_sb_tune.end()) return it->second;
    const int nprobe = std::min(nj, 4 * mbs_num_sms());
    cudaEvent_t a = take_event(c), b = take_event(c);
    int best = 512;
    float best_ms = 0.f;
    bool first = true;
    for (int th : {512, 256, 128}) {
        MBS_CUDA_TRY(cudaEventRecord(a, c->st));
        launch_sbuild(c->dim, d_jobs, nprobe, d_counter, rows_max, th, c->kappa, c->opt.ls_rcond, c->st);
        MBS_CUDA_TRY(cudaEventRecord(b, c->st));
        MBS_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        MBS_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        if (first || ms < best_ms) {
            best_ms = ms;
            best = th;
            first = false;
        }
    }
    c->ev_pool.push_back(a);
    c->ev_pool.push_back(b);
    g_sb_tune[key] = best;
    return best;
}

std::mutex g_tune_mu;
std::map<std::array<int, 6>, Shape32> g_tune;

int log2_bucket(int64_t v) {
    int b = 0;
    while ((int64_t(1) << b) < v) ++b;
    return b;
}

void launch_g32(mbs_ctx* c, int nrhs, const float2* x, float2* y, const Shape32& sh,
                cudaEvent_t e0, cudaEvent_t e1) {
    int* sb = split_table(c, sh.nsplit);
    float2* part = scratch<float2>(c, "part32", (size_t)sh.nsplit * nrhs * c->N);
    UmmaLayout U{};
    if (sh.path == 3) {
        U.nchunks = c->nchunks;
        U.chunk_off = c->d_chunk_off;
        U.chunk_body = c->d_chunk_body;
        U.pack_bytes = umma_pack_bytes(c->nchunks, nrhs);
        U.pack = scratch<unsigned char>(c, "umma_pack", U.pack_bytes);
        U.err = device_err(c);
    }
    launch_G_f32(glayout(c), c->kappa, nrhs, x, y, part, sh.nsplit, sb, c->st, e0, e1, sh.path,
                 sh.path == 3 ? &U : nullptr);
}

Shape32 heuristic_shape32(mbs_ctx* c, int nrhs) {
    Shape32 sh;
    sh.path = g32_path(c, nrhs);
    // the tcgen05 kernel tiles 128 targets per CTA, the others 256
    sh.nsplit = choose_nsplit(c, sh.path == 3 ? 2 * c->N : c->N);
    return sh;
}

Shape32 shape32(mbs_ctx* c, int nrhs, const float2* x, float2* y) {
    const Shape32 h = heuristic_shape32(c, nrhs);
    if (!c->opt.autotune || c->opt.tile_override > 0) return h;
    int dev = 0;
    MBS_CUDA_TRY(cudaGetDevice(&dev));
    const std::array<int, 6> key{dev, c->dim, nrhs, c->opt.mac_path, log2_bucket(c->N), log2_bucket(c->T)};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
        Shape32 sh = it->second;
        sh.nsplit = std::min(sh.nsplit, max_nsplit(c));
        return sh;
    }
    std::vector<Shape32> cand;
    std::vector<int> paths{h.path};
    if (c->opt.mac_path == 0 && h.path == 3) paths.push_back(1);
    for (int p : paths) {
        const int base = choose_nsplit(c, p == 3 ? 2 * c->N : c->N);
        for (int ns : {base, base / 2, 2 * base}) {
            ns = std::max(1, std::min(ns, max_nsplit(c)));
            bool dup = false;
            for (const Shape32& q : cand) dup = dup || (q.path == p && q.nsplit == ns);
            if (!dup) cand.push_back({p, ns});
        }
    }
    cudaEvent_t a = take_event(c), b = take_event(c);
    Shape32 best = h;
    float best_ms = 0.f;
    launch_g32(c, nrhs, x, y, cand[0], nullptr, nullptr);  // warm-up
    for (size_t ci = 0; ci < cand.size(); ++ci) {
        MBS_CUDA_TRY(cudaEventRecord(a, c->st));
        launch_g32(c, nrhs, x, y, cand[ci], nullptr, nullptr);
        MBS_CUDA_TRY(cudaEventRecord(b, c->st));
        MBS_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        MBS_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        if (ci == 0 || ms < best_ms) {
            best_ms = ms;
            best = cand[ci];
        }
    }
    c->ev_pool.push_back(a);
    c->ev_pool.push_back(b);
    g_tune[key] = best;
    return best;
}

// y = G_hat x (FP32); a first call of a problem class may run the autotuner,
// whose last timed launch is overwritten by the final one below.
void G32(mbs_ctx* c, int nrhs, const float2* x, float2* y) {
    const Shape32 sh = shape32(c, nrhs, x, y);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profile && c->capturing) {
        e0 = c->cap_e0;  // recorded on every replay of the step graph
        e1 = c->cap_e1;
    } else if (c->profile) {
        e0 = take_event(c);
        e1 = take_event(c);
        c->ev32.emplace_back(e0, e1);
    }
    launch_g32(c, nrhs, x, y, sh, e0, e1);
    c->last_path = sh.path;
    c->last_nsplit = sh.nsplit;
}
void G64(mbs_ctx* c, int nrhs, const double2* x, double2* y) {
    int ns;
    int* sb = split_for(c, c->N, &ns);
    double2* part = scratch<double2>(c, "part64", (size_t)ns * nrhs * c->N);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profile && c->capturing) {
        e0 = c->cap_e0;
        e1 = c->cap_e1;
    } else if (c->profile) {
        e0 = take_event(c);
        e1 = take_event(c);
        c->ev64.emplace_back(e0, e1);
    }
    if (c->opt.fp64_kernel == 1 || (c->opt.fp64_kernel == 2 && c->in_solve && c->df_active)) {
        // double-float arithmetic on the FP32 pipe (gdf.cu); the events bracket
        // the kernel passes, not the split reduction, as for the FP64 kernel
        launch_G_df(glayout(c), c->d_centres, c->kappa, nrhs, x, y, part, ns, sb, c->st, e0, e1);
        return;
    }
    launch_G_f64(glayout(c), c->kappa, nrhs, x, y, part, ns, sb, c->st, e0, e1);
}

// out = x + S G_hat x
void op32(mbs_ctx* c, int nrhs, const float2* x, float2* out) {
    float2* t = scratch<float2>(c, "op_t32", (size_t)nrhs * c->N);
    G32(c, nrhs, x, t);
    launch_sapply_f32(sblocks(c), c->N, nrhs, x, t, out, c->kmax, c->st);
}
void op64(mbs_ctx* c, int nrhs, const double2* x, double2* out) {
    double2* t = scratch<double2>(c, "op_t64", (size_t)nrhs * c->N);
    G64(c, nrhs, x, t);
    launch_sapply_f64(sblocks(c), c->N, nrhs, x, t, out, c->kmax, c->st);
}

template <typename V>
void apply_op(mbs_ctx* c, int nrhs, const V* x, V* out);
template <>
void apply_op<float2>(mbs_ctx* c, int nrhs, const float2* x, float2* out) {
    op32(c, nrhs, x, out);
}
template <>
void apply_op<double2>(mbs_ctx* c, int nrhs, const double2* x, double2* out) {
    op64(c, nrhs, x, out);
}

// Blocks per RHS of the dot-product kernel: each block covers at most 2048
// rows (its slice of w stays in registers); aim at ~4 blocks per SM overall.
int dot_blocks(int64_t N, int nrhs) {
    const int64_t minb = (N + 2047) / 2048;
    const int64_t want = (4LL * mbs_num_sms() + nrhs - 1) / nrhs;
    const int64_t maxb = (N + 255) / 256;
    return (int)std::max<int64_t>(1, std::max(minb, std::min(want, maxb)));
}

// Per-RHS 2-norms of a [nrhs][N] vector block (host result).
template <typename V>
std::vector<double> norms(mbs_ctx* c, const V* x, int nrhs) {
    const int nb = dot_blocks(c->N, nrhs);
    double2* d = scratch<double2>(c, "nrm_out", nrhs);
    double2* sc = scratch<double2>(c, "nrm_sc", (size_t)nrhs * nb);
    std::vector<double2> h(nrhs);
    // the "basis" is x itself with one vector per RHS: dots(x_r, x_r) for each r
    std::vector<double> out(nrhs);
    launch_dots<V>(x, 1, x, c->N, nrhs, d, sc, nb, c->st);
    MBS_CUDA_TRY(cudaMemcpyAsync(h.data(), d, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
    MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
    for (int r = 0; r < nrhs; ++r) out[r] = std::sqrt(std::max(0.0, h[r].x));
    return out;
}

// ---------------------------------------------------------------------------
// restarted GMRES on (I + S G) x = b for nrhs independent right-hand sides,
// advanced in lockstep (one operator application covers every RHS).
// Arnoldi with classical Gram-Schmidt applied twice (CGS2), complex Givens
// rotations on the Hessenberg matrices on the host (FP64).
// ---------------------------------------------------------------------------
struct GmresStats {
    int iters = 0;
    int matvecs = 0;
    std::vector<double> relres;  // estimate (rotations) per RHS at exit
    bool converged = false;
};

template <typename V>
GmresStats gmres(mbs_ctx* c, int nrhs, const V* b, V* x, bool x_zero, double tol, int restart,
                 int maxit, bool verify) {
    const int64_t N = c->N;
    const size_t NV = (size_t)nrhs * N;
    GmresStats S;
    S.relres.assign(nrhs, 0.0);
    V* basis = scratch<V>(c, std::string("gm_basis") + (sizeof(V) == 8 ? "32" : "64"),
                          (size_t)(restart + 1) * NV);
    V* w = scratch<V>(c, std::string("gm_w") + (sizeof(V) == 8 ? "32" : "64"), NV);
    V* r = scratch<V>(c, std::string("gm_r") + (sizeof(V) == 8 ? "32" : "64"), NV);
    const int nb = dot_blocks(N, nrhs);
    double2* d_h = scratch<double2>(c, "gm_h", (size_t)(2 * (restart + 1) + 1) * nrhs);
    double2* d_sc = scratch<double2>(c, "gm_sc", (size_t)(restart + 1) * nrhs * nb);
    double* d_inv = scratch<double>(c, "gm_inv", nrhs);

    const std::vector<double> bn = norms<V>(c, b, nrhs);
    // initial residual
    if (x_zero) {
        MBS_CUDA_TRY(cudaMemsetAsync(x, 0, NV * sizeof(V), c->st));
        MBS_CUDA_TRY(cudaMemcpyAsync(r, b, NV * sizeof(V), cudaMemcpyDeviceToDevice, c->st));
    } else {
        apply_op<V>(c, nrhs, x, w);
        S.matvecs++;
        launch_sub<V>(b, w, r, (int64_t)NV, c->st);
    }
    const int ld = restart + 1;
    std::vector<cd> H((size_t)nrhs * ld * restart), cs(nrhs * restart), sn(nrhs * restart),
        g((size_t)nrhs * ld);
    std::vector<double2> hh((size_t)(2 * (restart + 1) + 1) * nrhs);
    std::vector<double> inv(nrhs);
    std::vector<int> msteps(nrhs), frozen(nrhs);
    double prev_worst = 1e300;
    while (true) {
        std::vector<double> beta = norms<V>(c, r, nrhs);
        bool all = true;
        double worst = 0.0;
        for (int q = 0; q < nrhs; ++q) {
            const double rel = bn[q] > 0 ? beta[q] / bn[q] : 0.0;
            worst = std::max(worst, rel);
        }
        // a restart cycle that did not reduce the worst true residual by 10 %
        // has hit the precision floor of this arithmetic: stop
        if (worst > 0.9 * prev_worst && worst > tol) {
            for (int q = 0; q < nrhs; ++q) S.relres[q] = bn[q] > 0 ? beta[q] / bn[q] : 0.0;
            break;
        }
        prev_worst = worst;
        for (int q = 0; q < nrhs; ++q) {
            const double rel = bn[q] > 0 ? beta[q] / bn[q] : 0.0;
            S.relres[q] = rel;
            frozen[q] = rel <= tol ? 1 : 0;
            all = all && frozen[q];
            inv[q] = frozen[q] ? 0.0 : 1.0 / beta[q];
            msteps[q] = 0;
            for (int i = 0; i < ld; ++i) g[(size_t)q * ld + i] = 0.0;
            g[(size_t)q * ld] = frozen[q] ? 0.0 : beta[q];
        }
        if (all) {
            S.converged = true;
            break;
        }
        if (S.iters >= maxit) break;
        MBS_CUDA_TRY(cudaMemcpyAsync(d_inv, inv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c->st));
        launch_scale<V>(r, d_inv, basis, N, nrhs, c->st);
        int jdone = 0;
        for (int j = 0; j < restart && S.iters < maxit; ++j) {
            V* vj = basis + (size_t)j * NV;
            apply_op<V>(c, nrhs, vj, w);
            S.matvecs++;
            double2* h1 = d_h;
            double2* h2 = d_h + (size_t)(restart + 1) * nrhs;
            double2* hn = d_h + (size_t)2 * (restart + 1) * nrhs;
            launch_dots<V>(basis, j + 1, w, N, nrhs, h1, d_sc, nb, c->st);
            launch_update<V>(basis, j + 1, h1, w, N, nrhs, -1.0, c->st);
            launch_dots<V>(basis, j + 1, w, N, nrhs, h2, d_sc, nb, c->st);
            launch_update<V>(basis, j + 1, h2, w, N, nrhs, -1.0, c->st);
            launch_dots<V>(w, 1, w, N, nrhs, hn, d_sc, nb, c->st);
            MBS_CUDA_TRY(cudaMemcpyAsync(hh.data(), d_h, hh.size() * sizeof(double2),
                                         cudaMemcpyDeviceToHost, c->st));
            MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
            S.iters++;
            jdone = j + 1;
            bool allf = true;
            for (int q = 0; q < nrhs; ++q) {
                if (frozen[q]) {
                    inv[q] = 0.0;
                    continue;
                }
                cd* Hq = &H[(size_t)q * ld * restart];
                cd* col = Hq + (size_t)j * ld;
                for (int i = 0; i <= j; ++i) {
                    const double2 a = hh[(size_t)i * nrhs + q];
                    const double2 bb = hh[(size_t)(restart + 1) * nrhs + (size_t)i * nrhs + q];
                    col[i] = cd(a.x + bb.x, a.y + bb.y);
                }
                const double hnext = std::sqrt(std::max(0.0, hh[(size_t)2 * (restart + 1) * nrhs + q].x));
                col[j + 1] = hnext;
                cd* csq = &cs[(size_t)q * restart];
                cd* snq = &sn[(size_t)q * restart];
                cd* gq = &g[(size_t)q * ld];
                for (int i = 0; i < j; ++i) {
                    const cd t = std::conj(csq[i]) * col[i] + std::conj(snq[i]) * col[i + 1];
                    col[i + 1] = -snq[i] * col[i] + csq[i] * col[i + 1];
                    col[i] = t;
                }
                const cd a = col[j], bb = col[j + 1];
                const double den = std::sqrt(std::norm(a) + std::norm(bb));
                csq[j] = den > 0 ? a / den : cd(1.0);
                snq[j] = den > 0 ? bb / den : cd(0.0);
                col[j] = den;
                col[j + 1] = 0.0;
                gq[j + 1] = -snq[j] * gq[j];
                gq[j] = std::conj(csq[j]) * gq[j];
                msteps[q] = j + 1;
                const double rel = bn[q] > 0 ? std::abs(gq[j + 1]) / bn[q] : 0.0;
                S.relres[q] = rel;
                const bool breakdown = hnext <= 1e-300 || hnext <= 1e-15 * den;
                if (rel <= tol || breakdown) {
                    frozen[q] = 1;
                    inv[q] = 0.0;
                } else {
                    inv[q] = 1.0 / hnext;
                    allf = false;
                }
            }
            if (allf) break;
            if (j + 1 < restart) {
                MBS_CUDA_TRY(cudaMemcpyAsync(d_inv, inv.data(), nrhs * sizeof(double),
                                             cudaMemcpyHostToDevice, c->st));
                launch_scale<V>(w, d_inv, basis + (size_t)(j + 1) * NV, N, nrhs, c->st);
            }
        }
        // x += V y with y from the triangular systems
        std::vector<double2> y((size_t)jdone * nrhs, make_double2(0.0, 0.0));
        for (int q = 0; q < nrhs; ++q) {
            const int mq = msteps[q];
            const cd* Hq = &H[(size_t)q * ld * restart];
            const cd* gq = &g[(size_t)q * ld];
            std::vector<cd> yq(mq);
            for (int i = mq - 1; i >= 0; --i) {
                cd s = gq[i];
                for (int l = i + 1; l < mq; ++l) s -= Hq[(size_t)l * ld + i] * yq[l];
                yq[i] = s / Hq[(size_t)i * ld + i];
            }
            for (int i = 0; i < mq; ++i) y[(size_t)i * nrhs + q] = make_double2(yq[i].real(), yq[i].imag());
        }
        if (jdone > 0) {
            MBS_CUDA_TRY(cudaMemcpyAsync(d_h, y.data(), y.size() * sizeof(double2),
                                         cudaMemcpyHostToDevice, c->st));
            launch_update<V>(basis, jdone, d_h, x, N, nrhs, 1.0, c->st);
        }
        bool est_conv = true;
        for (int q = 0; q < nrhs; ++q) est_conv = est_conv && S.relres[q] <= tol;
        if (est_conv && !verify) {
            S.converged = true;
            break;
        }
        if (S.iters >= maxit && !verify) break;
        // true residual, then restart (or final check)
        apply_op<V>(c, nrhs, x, w);
        S.matvecs++;
        launch_sub<V>(b, w, r, (int64_t)NV, c->st);
        if (S.iters >= maxit) {
            std::vector<double> beta = norms<V>(c, r, nrhs);
            bool ok = true;
            for (int q = 0; q < nrhs; ++q) {
                S.relres[q] = bn[q] > 0 ? beta[q] / bn[q] : 0.0;
                ok = ok && S.relres[q] <= tol;
            }
            S.converged = ok;
            break;
        }
    }
    return S;
}

// ---------------------------------------------------------------------------
// Block GMRES: the nrhs right-hand sides share one block Krylov space
// span{R0, A R0, A^2 R0, ...} (each step applies the operator to an N x s
// block, exactly like the lockstep GMRES, but every RHS minimises over all
// s*j directions).  Block classical Gram-Schmidt applied twice with the
// tall-skinny kernels of blas.cu (fixed reduction order, so a solve is bitwise
// reproducible next to other work); the new block is orthonormalised by CholQR2
// (Gram matrix, FP64 Cholesky and triangular solve, all on the device); each
// step ends with one readback of the coefficients, and the block upper
// Hessenberg least-squares problem is reduced by Givens rotations on the host
// in FP64.
// ---------------------------------------------------------------------------
template <typename V>
void from_host_cd(const std::vector<cd>& in, V* d, cudaStream_t st, std::vector<V>& stage) {
    stage.resize(in.size());
    for (size_t i = 0; i < in.size(); ++i) {
        stage[i].x = (decltype(stage[i].x))in[i].real();
        stage[i].y = (decltype(stage[i].y))in[i].imag();
    }
    MBS_CUDA_TRY(cudaMemcpyAsync(d, stage.data(), in.size() * sizeof(V), cudaMemcpyHostToDevice, st));
}

// W (N x s, [s][N]) = Q R with Q orthonormal: two Cholesky-QR passes, all on
// the device (Gram product, s x s Cholesky, triangular solve), queued without
// a host synchronisation.  The factors land in Bs: R1 at [0, s^2), R2 at
// [s^2, 2 s^2), and the two positive-definiteness flags in the next double2.
template <typename V>
void cholqr2_dev(mbs_ctx* c, V* W, int64_t N, int s, double2* Bs, double2* d_gram, double2* d_part) {
    const int nb = ts_gram_blocks(N, s, s, sizeof(V) == 8);
    double* ok = reinterpret_cast<double*>(Bs + 2 * s * s);
    for (int pass = 0; pass < 2; ++pass) {
        double2* R = Bs + (size_t)pass * s * s;
        launch_ts_gram<V>(W, s, W, s, N, d_gram, d_part, nb, c->st, device_err(c));
        launch_chol_small(d_gram, s, R, ok + pass, c->st);
        launch_ts_trsm<V>(W, s, N, R, c->st);
    }
}

// Host side of cholqr2_dev after the readback: R = R2 R1, false if either
// pass was not positive definite (rank deficiency).
bool cholqr2_host(const double2* Bs, int s, std::vector<cd>& R) {
    const double* ok = reinterpret_cast<const double*>(Bs + 2 * s * s);
    if (!(ok[0] > 0.5 && ok[1] > 0.5)) return false;
    const double2* R1 = Bs;
    const double2* R2 = Bs + s * s;
    R.assign((size_t)s * s, cd(0.0));
    for (int j = 0; j < s; ++j)
        for (int i = 0; i <= j; ++i) {
            cd sum = 0.0;
            for (int k = i; k <= j; ++k)
                sum += cd(R2[k * s + i].x, R2[k * s + i].y) * cd(R1[j * s + k].x, R1[j * s + k].y);
            R[(size_t)j * s + i] = sum;
        }
    return true;
}

double2* pinned_stage(mbs_ctx* c, size_t count) {
    if (c->pinned_n < count) {
        if (c->pinned) cudaFreeHost(c->pinned);
        c->pinned = nullptr;
        c->pinned_n = 0;
        MBS_CUDA_TRY(cudaMallocHost(&c->pinned, count * sizeof(double2)));
        c->pinned_n = count;
    }
    return c->pinned;
}

// Run one block-GMRES step from its CUDA graph, capturing it at first use.
// Returns the graph (for its profiling events), or nullptr if the step could
// not be captured; the caller then enqueues the step directly.
template <typename F>
StepGraph* run_step_graph(mbs_ctx* c, const std::array<int64_t, 8>& key, int prec, F&& enqueue) {
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        StepGraph g;
        g.prec = prec;
        if (c->profile) {
            MBS_CUDA_TRY(cudaEventCreate(&g.e0));
            MBS_CUDA_TRY(cudaEventCreate(&g.e1));
        }
        auto fail = [&]() -> StepGraph* {
            cudaGetLastError();
            if (g.e0) cudaEventDestroy(g.e0);
            if (g.e1) cudaEventDestroy(g.e1);
            c->graphs_off = true;
            return nullptr;
        };
        if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail();
        c->capturing = true;
        c->cap_e0 = g.e0;
        c->cap_e1 = g.e1;
        const long long l0 = g_mbs_launches.load();
        bool ok = true;
        try {
            enqueue();
        } catch (const MbsError&) {
            ok = false;
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c->st, &graph);
        c->capturing = false;
        g.launches = g_mbs_launches.load() - l0;
        g_mbs_launches.fetch_sub(g.launches);  // nothing ran during the capture
        if (!ok || ee != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            return fail();
        }
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return fail();
        it = c->graphs.emplace(key, g).first;
    }
    MBS_CUDA_TRY(cudaGraphLaunch(it->second.exec, c->st));
    g_mbs_launches.fetch_add(it->second.launches);
    return &it->second;
}

// Block GMRES (the restarted GMRES of Sec. 2.4 with the s right-hand sides as
// one block): step j applies the operator to the newest block of s basis
// vectors, orthogonalises by block CGS2 and CholQR2 on the device, and reduces
// the block Hessenberg least-squares problem on the host (BlockLsq) while the
// device already runs step j+1.  Stops when every right-hand side reaches tol
// (relative to its own |b|), at maxit steps, or when a restart cycle no longer
// reduces the worst residual by 10 %.  verify: confirm convergence with the
// true residual before returning.
template <typename V>
GmresStats bgmres(mbs_ctx* c, int s, const V* b, V* x, bool x_zero, double tol, int restart,
                  int maxit, bool verify) {
    const int64_t N = c->N;
    const size_t NV = (size_t)s * N;
    GmresStats S;
    S.relres.assign(s, 0.0);
    const std::string sfx = sizeof(V) == 8 ? "32" : "64";
    V* basis = scratch<V>(c, "bg_basis" + sfx, (size_t)(restart + 1) * NV);
    V* w = scratch<V>(c, "gm_w" + sfx, NV);
    V* r = scratch<V>(c, "gm_r" + sfx, NV);
    // per step, read back in one copy: [R1 | R2 | ok | Hcol pass 1 (K s) | Hcol pass 2 (K s)]
    const size_t sq = (size_t)s * s;
    const size_t nsmall = 2 * sq + 1 + 2 * (size_t)restart * sq;
    double2* Bs = scratch<double2>(c, "bg_small", nsmall);
    double2* d_gram = scratch<double2>(c, "bg_gram", sq);
    // two readback buffers: the host reduces step j while step j+1 runs
    double2* hb0 = pinned_stage(c, 2 * nsmall);
    double2* const hbs[2] = {hb0, hb0 + nsmall};
    double2* hb = hbs[0];
    constexpr bool f32 = sizeof(V) == 8;
    // partial sums of the Gram products (nblk * ka * s for every block width ka used)
    size_t part = 0;
    for (int j = 0; j < restart; ++j) {
        const int ka = (j + 1) * s;
        part = std::max(part, (size_t)ts_gram_blocks(N, ka, s, f32) * ka * s);
    }
    double2* d_part = scratch<double2>(c, "bg_part", part);
    float2* d_coef = f32 ? scratch<float2>(c, "bg_coef", (size_t)restart * s * 8) : nullptr;
    double* d_inv = scratch<double>(c, "gm_inv", s);
    const std::vector<double> bn = norms<V>(c, b, s);
    if (x_zero) {
        MBS_CUDA_TRY(cudaMemsetAsync(x, 0, NV * sizeof(V), c->st));
        MBS_CUDA_TRY(cudaMemcpyAsync(r, b, NV * sizeof(V), cudaMemcpyDeviceToDevice, c->st));
    } else {
        apply_op<V>(c, s, x, w);
        S.matvecs++;
        launch_sub<V>(b, w, r, (int64_t)NV, c->st);
    }
    std::vector<cd> Hcol, Rk;
    BlockLsq lsq;  // the small least-squares problem of each cycle (host)
    double prev_worst = 1e300;
    bool warm = false;
    while (true) {
        const std::vector<double> beta = norms<V>(c, r, s);
        double worst = 0.0;
        bool all = true, zero_col = false;
        for (int q = 0; q < s; ++q) {
            const double rel = bn[q] > 0 ? beta[q] / bn[q] : 0.0;
            S.relres[q] = rel;
            worst = std::max(worst, rel);
            all = all && rel <= tol;
            zero_col = zero_col || beta[q] == 0.0;
        }
        if (all) {
            S.converged = true;
            break;
        }
        if (S.iters >= maxit || worst > 0.9 * prev_worst || zero_col) break;
        prev_worst = worst;
        // V_0 beta0 = R0 with unit-norm columns first (D^{-1}), so beta0 = Rq D
        std::vector<double> inv(s);
        for (int q = 0; q < s; ++q) inv[q] = 1.0 / beta[q];
        MBS_CUDA_TRY(cudaMemcpyAsync(d_inv, inv.data(), s * sizeof(double), cudaMemcpyHostToDevice, c->st));
        launch_scale<V>(r, d_inv, basis, N, s, c->st);
        std::vector<cd> Rq;
        cholqr2_dev<V>(c, basis, N, s, Bs, d_gram, d_part);
        hb = hbs[0];
        MBS_CUDA_TRY(cudaMemcpyAsync(hb, Bs, (2 * sq + 1) * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
        MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
        if (!cholqr2_host(hb, s, Rq)) break;  // R0 numerically rank deficient
        lsq.start(s, restart, Rq.data(), beta.data());
        int jdone = 0;
        bool breakdown = false;
        // the step's device work, queued without host synchronisation: operator,
        // block CGS2 (Hcol = V^H W; W -= V Hcol, twice), CholQR2 of the new block
        // and one readback of both coefficient blocks and both factors into hbs[j % 2]
        auto enqueue = [&](int j) {
            const int K = (j + 1) * s;
            V* vj = basis + (size_t)j * NV;
            apply_op<V>(c, s, vj, w);
            double2* h1 = Bs + 2 * sq + 1;
            double2* h2 = h1 + (size_t)K * s;
            for (int pass = 0; pass < 2; ++pass) {
                double2* hp = pass == 0 ? h1 : h2;
                launch_ts_gram<V>(basis, K, w, s, N, hp, d_part, ts_gram_blocks(N, K, s, f32), c->st,
                                  device_err(c));
                launch_ts_update<V>(basis, K, hp, -1.0, w, s, N, c->st, d_coef, device_err(c));
            }
            V* vn = basis + (size_t)(j + 1) * NV;
            MBS_CUDA_TRY(cudaMemcpyAsync(vn, w, NV * sizeof(V), cudaMemcpyDeviceToDevice, c->st));
            cholqr2_dev<V>(c, vn, N, s, Bs, d_gram, d_part);
            MBS_CUDA_TRY(cudaMemcpyAsync(hbs[j & 1], Bs, (2 * sq + 1 + 2 * (size_t)K * s) * sizeof(double2),
                                         cudaMemcpyDeviceToHost, c->st));
        };
        // after one direct step (autotuning, buffer allocation) the steps run
        // from CUDA graphs captured once per context and step index
        auto launch_step = [&](int j) -> StepGraph* {
            StepGraph* sg = nullptr;
            if (warm && c->opt.cuda_graphs && !c->graphs_off) {
                const std::array<int64_t, 8> key{(int64_t)sizeof(V), s, j, restart, (int64_t)(intptr_t)basis,
                                                 (int64_t)(intptr_t)w, (int64_t)(intptr_t)Bs,
                                                 (int64_t)(intptr_t)hbs[j & 1]};
                sg = run_step_graph(c, key, f32 ? 0 : 1, [&]() { enqueue(j); });
            }
            if (!sg) enqueue(j);
            return sg;
        };
        StepGraph* sg_next = nullptr;
        bool pending = false;  // a queued step not yet reduced on the host
        size_t mark32 = 0, mark64 = 0;
        auto launch_next = [&](int j) {
            mark32 = c->ev32.size();
            mark64 = c->ev64.size();
            sg_next = launch_step(j);
            pending = true;
        };
        if (restart > 0 && S.iters < maxit) launch_next(0);
        for (int j = 0; j < restart && S.iters < maxit; ++j) {
            const int K = (j + 1) * s;
            StepGraph* sg = sg_next;
            pending = false;
            MBS_CUDA_TRY(cudaStreamSynchronize(c->st));  // step j is complete
            S.matvecs++;
            warm = true;
            if (sg && sg->e0) {
                float ms = 0.f;
                MBS_CUDA_TRY(cudaEventElapsedTime(&ms, sg->e0, sg->e1));
                c->graph_ms[sg->prec] += ms;
                c->graph_n[sg->prec] += 1;
            }
            // step j+1 depends on step j's device results only: it runs while the
            // host reduces step j, and is discarded unless step j leaves the cycle
            // open (its matvec is then not counted)
            sg_next = nullptr;
            if (j + 1 < restart && S.iters + 1 < maxit) launch_next(j + 1);
            hb = hbs[j & 1];
            Hcol.assign((size_t)K * s, cd(0.0));
            for (size_t e = 0; e < (size_t)K * s; ++e) {
                const double2 a1 = hb[2 * sq + 1 + e], a2 = hb[2 * sq + 1 + (size_t)K * s + e];
                Hcol[e] = cd(a1.x + a2.x, a1.y + a2.y);
            }
            if (!cholqr2_host(hb, s, Rk)) {
                breakdown = true;  // the new block adds no direction: the solution is in the space
                Rk.assign(sq, cd(0.0));
            }
            S.iters++;
            jdone = j + 1;
            // block column j of the Hessenberg matrix: Hcol above, Rk below
            lsq.add(j, Hcol.data(), Rk.data());
            bool conv = true;
            for (int q = 0; q < s; ++q) {
                S.relres[q] = bn[q] > 0 ? lsq.residual(q) / bn[q] : 0.0;
                conv = conv && S.relres[q] <= tol;
            }
            if (conv || breakdown) break;
        }
        if (pending) {
            // the step queued past the end of the cycle is discarded: a direct
            // launch's profiling events leave the lists (a graph's are only read
            // when its step is reduced)
            MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
            if (!sg_next) {
                for (size_t i = mark32; i < c->ev32.size(); ++i) {
                    c->ev_pool.push_back(c->ev32[i].first);
                    c->ev_pool.push_back(c->ev32[i].second);
                }
                for (size_t i = mark64; i < c->ev64.size(); ++i) {
                    c->ev_pool.push_back(c->ev64[i].first);
                    c->ev_pool.push_back(c->ev64[i].second);
                }
                c->ev32.resize(std::min(mark32, c->ev32.size()));
                c->ev64.resize(std::min(mark64, c->ev64.size()));
            }
        }
        // Y = R^{-1} G over the steps of this cycle, X += V Y
        const int Mj = jdone * s;
        std::vector<cd> Y;
        lsq.solve(jdone, Y);
        if (Mj > 0) {
            double2* d_y = scratch<double2>(c, "bg_y", (size_t)restart * s * s);
            std::vector<double2> stage;
            from_host_cd(Y, d_y, c->st, stage);
            launch_ts_update<V>(basis, Mj, d_y, 1.0, x, s, N, c->st, d_coef, device_err(c));
        }
        bool est_conv = true;
        for (int q = 0; q < s; ++q) est_conv = est_conv && S.relres[q] <= tol;
        if (est_conv && !verify) {
            S.converged = true;
            break;
        }
        if (S.iters >= maxit && !verify) break;
        apply_op<V>(c, s, x, w);
        S.matvecs++;
        launch_sub<V>(b, w, r, (int64_t)NV, c->st);
        if (S.iters >= maxit) {
            const std::vector<double> bt = norms<V>(c, r, s);
            bool ok = true;
            for (int q = 0; q < s; ++q) {
                S.relres[q] = bn[q] > 0 ? bt[q] / bn[q] : 0.0;
                ok = ok && S.relres[q] <= tol;
            }
            S.converged = ok;
            break;
        }
    }
    MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
    return S;
}

// Krylov solver choice: block GMRES for 2..16 right-hand sides (unless
// disabled), lockstep GMRES otherwise.  The host-side Givens reduction of the
// block Hessenberg matrix costs O(j s^3) per step, which grows too fast beyond
// 16 right-hand sides.
template <typename V>
GmresStats krylov(mbs_ctx* c, int nrhs, const V* b, V* x, bool x_zero, double tol, int restart,
                  int maxit, bool verify) {
    if (nrhs > 1 && nrhs <= 16 && c->opt.block_krylov)
        return bgmres<V>(c, nrhs, b, x, x_zero, tol, restart, maxit, verify);
    return gmres<V>(c, nrhs, b, x, x_zero, tol, restart, maxit, verify);
}

void validate_options(const mbs_options& o) {
    if (o.precision != MBS_PREC_FP64 && o.precision != MBS_PREC_MIXED && o.precision != MBS_PREC_FP32)
        throw MbsError{MBS_ERR_ARG, "precision must be MBS_PREC_FP64, MBS_PREC_MIXED or MBS_PREC_FP32"};
    if (!(o.tol > 0) || !(o.inner_tol > 0) || o.restart < 1 || o.restart > 1800 || o.max_iter < 1 || o.max_sweeps < 1 ||
        !(o.ls_rcond > 0 && o.ls_rcond < 1))
        throw MbsError{MBS_ERR_ARG, "invalid tolerance / restart / iteration options"};
    if (o.mac_path < 0 || o.mac_path > 3)
        throw MbsError{MBS_ERR_ARG, "mac_path must be 0, 1, 2 or 3"};
    if (o.fp64_kernel < 0 || o.fp64_kernel > 2)
        throw MbsError{MBS_ERR_ARG, "fp64_kernel must be 0, 1 or 2"};
    if (o.sbuild_threads != 0 && o.sbuild_threads != -1 && o.sbuild_threads != 128 && o.sbuild_threads != 256 &&
        o.sbuild_threads != 512)
        throw MbsError{MBS_ERR_ARG, "sbuild_threads must be 0, -1, 128, 256 or 512"};
    if (o.id_sketch < 0) throw MbsError{MBS_ERR_ARG, "id_sketch must be >= 0"};
}

template <typename F>
mbs_status guarded(mbs_ctx* c, F&& f) {
    if (!c) return MBS_ERR_ARG;
    std::lock_guard<std::mutex> g(c->mu);
    try {
        const mbs_status s = f();
        if (c->d_err) {
            // a bounded wait of a device kernel ran out during this call
            int e = 0;
            MBS_CUDA_TRY(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
            MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
            if (e) {
                MBS_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
                throw MbsError{MBS_ERR_TIMEOUT, "a bounded device wait ran out (tensor-core G_hat or block Gram-Schmidt kernel)"};
            }
        }
        if (s == MBS_OK) c->err.clear();
        return s;
    } catch (const MbsError& e) {
        c->err = e.msg;
        return e.st;
    } catch (const std::exception& e) {
        c->err = e.what();
        return MBS_ERR_CUDA;
    }
}

// For every target (SoA dim x M, host or device), the body whose proxy
// surface strictly contains it, or -1; proxies are disjoint, so there is at
// most one.  A hash grid of cell size = the largest proxy radius finds the
// candidate bodies.  Throws MBS_ERR_ARG on a non-finite target.
std::vector<int> proxy_bodies(mbs_ctx* c, const double* pts, int64_t M);

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

std::vector<int> proxy_bodies(mbs_ctx* c, const double* pts, int64_t M) {
    const int d = c->dim;
    std::vector<double> hp((size_t)d * M);
    if (is_device_ptr(pts))
        MBS_CUDA_TRY(cudaMemcpy(hp.data(), pts, hp.size() * sizeof(double), cudaMemcpyDeviceToHost));
    else
        std::memcpy(hp.data(), pts, hp.size() * sizeof(double));
    if (!finite_all(hp.data(), hp.size())) throw MbsError{MBS_ERR_ARG, "non-finite target"};
    double reach = 0;
    for (int t = 0; t < c->T; ++t) reach = std::max(reach, c->shapes[c->bodies[t].shape].proxy_radius);
    const double h = std::max(reach, 1e-12);
    std::unordered_map<int64_t, std::vector<int>> grid;
    auto key = [&](int64_t ix, int64_t iy, int64_t iz) {
        return ((ix & 0x1FFFFF) << 42) | ((iy & 0x1FFFFF) << 21) | (iz & 0x1FFFFF);
    };
    for (int t = 0; t < c->T; ++t) {
        const double* cc = c->bodies[t].c;
        grid[key((int64_t)std::floor(cc[0] / h), (int64_t)std::floor(cc[1] / h),
                 d == 3 ? (int64_t)std::floor(cc[2] / h) : 0)]
            .push_back(t);
    }
    std::vector<int> tb((size_t)M, -1);
    for (int64_t i = 0; i < M; ++i) {
        double p3[3] = {hp[i], hp[(size_t)M + i], d == 3 ? hp[(size_t)2 * M + i] : 0.0};
        const int64_t ix = (int64_t)std::floor(p3[0] / h), iy = (int64_t)std::floor(p3[1] / h),
                      iz = d == 3 ? (int64_t)std::floor(p3[2] / h) : 0;
        for (int64_t a = -1; a <= 1; ++a)
            for (int64_t b2 = -1; b2 <= 1; ++b2)
                for (int64_t e = (d == 3 ? -1 : 0); e <= (d == 3 ? 1 : 0); ++e) {
                    auto it = grid.find(key(ix + a, iy + b2, iz + e));
                    if (it == grid.end()) continue;
                    for (int t : it->second) {
                        const double pr = c->shapes[c->bodies[t].shape].proxy_radius;
                        double r2 = 0;
                        for (int q = 0; q < d; ++q) r2 += (p3[q] - c->bodies[t].c[q]) * (p3[q] - c->bodies[t].c[q]);
                        if (r2 < pr * pr * (1.0 - 1e-12)) tb[i] = t;
                    }
                }
    }
    return tb;
}

void world_point(const mbs_body& B, int dim, const double* loc, double* out) {
    for (int a = 0; a < dim; ++a) {
        double s = B.c[a];
        for (int b2 = 0; b2 < dim; ++b2) s += B.R[3 * a + b2] * loc[b2];
        out[a] = s;
    }
}

// Every collocation point of every body must lie strictly outside the proxy
// radius of every other body (Sec. 4.1: S_tau handles sources outside Psi_tau).
void check_geometry(mbs_ctx* c) {
    const int T = c->T, d = c->dim;
    double reach = 0;
    for (int t = 0; t < T; ++t) {
        const ShapeHost& s = c->shapes[c->bodies[t].shape];
        reach = std::max(reach, s.proxy_radius + s.bound_radius);
    }
    const double h = std::max(reach, 1e-12);
    std::unordered_map<int64_t, std::vector<int>> grid;
    auto key = [&](int64_t ix, int64_t iy, int64_t iz) {
        return ((ix & 0x1FFFFF) << 42) | ((iy & 0x1FFFFF) << 21) | (iz & 0x1FFFFF);
    };
    for (int t = 0; t < T; ++t) {
        const double* cc = c->bodies[t].c;
        grid[key((int64_t)std::floor(cc[0] / h), (int64_t)std::floor(cc[1] / h),
                 d == 3 ? (int64_t)std::floor(cc[2] / h) : 0)]
            .push_back(t);
    }
    std::vector<double> loc(3), wp(3);
    for (int t = 0; t < T; ++t) {
        const mbs_body& Bt = c->bodies[t];
        const ShapeHost& st = c->shapes[Bt.shape];
        const int64_t ix = (int64_t)std::floor(Bt.c[0] / h), iy = (int64_t)std::floor(Bt.c[1] / h),
                      iz = d == 3 ? (int64_t)std::floor(Bt.c[2] / h) : 0;
        for (int64_t a = -1; a <= 1; ++a)
            for (int64_t b2 = -1; b2 <= 1; ++b2)
                for (int64_t e = (d == 3 ? -1 : 0); e <= (d == 3 ? 1 : 0); ++e) {
                    auto it = grid.find(key(ix + a, iy + b2, iz + e));
                    if (it == grid.end()) continue;
                    for (int s : it->second) {
                        if (s == t) continue;
                        const mbs_body& Bs = c->bodies[s];
                        const ShapeHost& ss = c->shapes[Bs.shape];
                        double cd2 = 0;
                        for (int q = 0; q < d; ++q) cd2 += (Bt.c[q] - Bs.c[q]) * (Bt.c[q] - Bs.c[q]);
                        const double lim = st.proxy_radius + ss.bound_radius;
                        if (cd2 > lim * lim) continue;
                        for (int i = 0; i < ss.m; ++i) {
                            for (int q = 0; q < d; ++q) loc[q] = ss.x[(size_t)q * ss.m + i];
                            world_point(Bs, d, loc.data(), wp.data());
                            double r2 = 0;
                            for (int q = 0; q < d; ++q) r2 += (wp[q] - Bt.c[q]) * (wp[q] - Bt.c[q]);
                            if (r2 <= st.proxy_radius * st.proxy_radius)
                                throw MbsError{MBS_ERR_GEOMETRY,
                                               "body " + std::to_string(s) +
                                                   " reaches inside the proxy surface of body " +
                                                   std::to_string(t)};
                        }
                    }
                }
    }
}

// Skeleton layout, body-pair table, S pointer tables, right-hand-side descriptors.
void setup_layout(mbs_ctx* c) {
    clear_graphs(c);  // captured steps refer to the layout's tables
    const int T = c->T, d = c->dim;
    c->off.assign(T + 1, 0);
    c->voff.assign(T + 1, 0);
    std::vector<int64_t> moff(T + 1, 0);
    c->kb.assign(T, 0);
    c->kmax = c->mmax = c->nmax = 0;
    for (int t = 0; t < T; ++t) {
        const ShapeHost& s = c->shapes[c->bodies[t].shape];
        c->kb[t] = s.k;
        c->off[t + 1] = c->off[t] + s.k;
        c->voff[t + 1] = c->voff[t] + s.m;
        moff[t + 1] = moff[t] + s.n;
        c->kmax = std::max(c->kmax, s.k);
        c->mmax = std::max(c->mmax, s.m);
        c->nmax = std::max(c->nmax, s.n);
    }
    double ss = 0.0;
    for (int t = 0; t < T; ++t) ss += c->shapes[c->bodies[t].shape].snorm * c->shapes[c->bodies[t].shape].snorm;
    c->snorm_rms = T > 0 ? std::sqrt(ss / T) : 0.0;
    c->N = c->off[T];
    c->Mtot = c->voff[T];
    c->Nm = moff[T];
    const int64_t N = c->N;
    std::vector<int> body(N);
    std::vector<float> loc32((size_t)d * N);
    c->skel_world.assign((size_t)d * N, 0.0);
    // centres (3 per body) followed by the bounding radius of every body
    std::vector<double> cen((size_t)4 * T, 0.0);
    for (int t = 0; t < T; ++t) {
        const mbs_body& B = c->bodies[t];
        const ShapeHost& s = c->shapes[B.shape];
        for (int a = 0; a < 3; ++a) cen[3 * t + a] = (a < d) ? B.c[a] : 0.0;
        cen[(size_t)3 * T + t] = s.bound_radius;
        for (int i = 0; i < s.k; ++i) {
            const int64_t g = c->off[t] + i;
            body[g] = t;
            const int col = s.skel[i];
            for (int a = 0; a < d; ++a) {
                double dl = 0.0;
                for (int b2 = 0; b2 < d; ++b2) dl += B.R[3 * a + b2] * s.x[(size_t)b2 * s.m + col];
                loc32[(size_t)a * N + g] = (float)dl;
                c->skel_world[(size_t)a * N + g] = B.c[a] + dl;
            }
        }
    }
    c->d_body = galloc<int>(c, N);
    c->d_off = galloc<int64_t>(c, T + 1);
    c->d_loc32 = galloc<float>(c, (size_t)d * N);
    c->d_xw64 = galloc<double>(c, (size_t)d * N);
    c->d_centres = galloc<double>(c, (size_t)4 * T);
    c->d_pair = galloc<float4>(c, (size_t)T * T);
    c->d_pair_phi0 = d == 3 ? galloc<float>(c, (size_t)T * T) : nullptr;
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_body, body.data(), N * sizeof(int), cudaMemcpyHostToDevice, c->st));
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_off, c->off.data(), (T + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->st));
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_loc32, loc32.data(), loc32.size() * sizeof(float), cudaMemcpyHostToDevice, c->st));
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_xw64, c->skel_world.data(), c->skel_world.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, c->st));
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_centres, cen.data(), cen.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_pair_table(d, T, c->d_centres, c->d_centres + (size_t)3 * T, c->kappa, c->d_pair,
                      c->d_pair_phi0, c->st);
    // source chunks of the tensor-core G_hat kernel
    std::vector<int> chunk_off(T + 1, 0), chunk_body;
    const int kc = umma_chunk();
    for (int t = 0; t < T; ++t) {
        const int nc = (c->kb[t] + kc - 1) / kc;
        chunk_off[t + 1] = chunk_off[t] + nc;
        for (int k = 0; k < nc; ++k) chunk_body.push_back(t);
    }
    c->nchunks = chunk_off[T];
    c->d_chunk_off = galloc<int>(c, T + 1);
    c->d_chunk_body = galloc<int>(c, std::max<size_t>(1, chunk_body.size()));
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_chunk_off, chunk_off.data(), (T + 1) * sizeof(int),
                                 cudaMemcpyHostToDevice, c->st));
    if (!chunk_body.empty())
        MBS_CUDA_TRY(cudaMemcpyAsync(c->d_chunk_body, chunk_body.data(), chunk_body.size() * sizeof(int),
                                     cudaMemcpyHostToDevice, c->st));
    // S tables and RHS descriptors
    std::vector<const double2*> s64(T);
    std::vector<const float2*> s32(T);
    std::vector<RhsBody> rb(T);
    for (int t = 0; t < T; ++t) {
        const ShapeHost& s = c->shapes[c->bodies[t].shape];
        s64[t] = s.S64;
        s32[t] = s.S32;
        RhsBody& R = rb[t];
        R.m = s.m;
        R.n = s.n;
        R.k = s.k;
        R.rankA = s.rankA;
        R.rankS = s.rankS;
        R.voff = c->voff[t];
        R.boff = c->off[t];
        R.moff = moff[t];
        R.A = s.AU;
        R.J = s.JA;
        R.F = s.FA;
        R.C = s.C;
        R.Zs = s.Zs;
        R.W = s.W;
    }
    c->d_k = galloc<int>(c, T);
    c->d_S64p = (const double2**)galloc<void*>(c, T);
    c->d_S32p = (const float2**)galloc<void*>(c, T);
    c->d_rhsb = galloc<RhsBody>(c, T);
    std::vector<MfsBody> mb(T);
    for (int t = 0; t < T; ++t) {
        const ShapeHost& s = c->shapes[c->bodies[t].shape];
        mb[t].y = s.dy;
        mb[t].n = s.n;
        mb[t].moff = moff[t];
        for (int a = 0; a < 3; ++a) mb[t].c[a] = c->bodies[t].c[a];
        for (int a = 0; a < 9; ++a) mb[t].R[a] = c->bodies[t].R[a];
    }
    c->d_mfsb = galloc<MfsBody>(c, T);
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_mfsb, mb.data(), T * sizeof(MfsBody), cudaMemcpyHostToDevice, c->st));
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_k, c->kb.data(), T * sizeof(int), cudaMemcpyHostToDevice, c->st));
    MBS_CUDA_TRY(cudaMemcpyAsync((void*)c->d_S64p, s64.data(), T * sizeof(void*), cudaMemcpyHostToDevice, c->st));
    MBS_CUDA_TRY(cudaMemcpyAsync((void*)c->d_S32p, s32.data(), T * sizeof(void*), cudaMemcpyHostToDevice, c->st));
    MBS_CUDA_TRY(cudaMemcpyAsync(c->d_rhsb, rb.data(), T * sizeof(RhsBody), cudaMemcpyHostToDevice, c->st));
    for (auto& kv : c->split_cache) dfree(c, kv.second);
    c->split_cache.clear();
    MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
}

void refresh_layout(mbs_ctx* c) {
    // drop the previous layout allocations (keep shape data) and rebuild
    MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
    std::vector<void*> keep;
    const void* lay[] = {c->d_body, c->d_off, c->d_loc32, c->d_xw64, c->d_centres, c->d_pair,
                         c->d_pair_phi0, c->d_k, c->d_S64p, c->d_S32p, c->d_rhsb,
                         c->d_chunk_off, c->d_chunk_body, c->d_mfsb};
    for (void* p : c->geom_allocs) {
        bool is_lay = false;
        for (const void* q : lay)
            if (q == p) is_lay = true;
        if (is_lay)
            dfree(c, p);
        else
            keep.push_back(p);
    }
    c->geom_allocs = keep;
    setup_layout(c);
}

void build(mbs_ctx* c, int nshapes, const mbs_shape* shapes, int nbodies, const mbs_body* bodies) {
    const int d = c->dim;
    if (nshapes < 1 || !shapes || nbodies < 1 || !bodies)
        throw MbsError{MBS_ERR_ARG, "need at least one shape and one body"};
    std::vector<ShapeHost> hs(nshapes);
    for (int s = 0; s < nshapes; ++s) {
        const mbs_shape& in = shapes[s];
        ShapeHost& h = hs[s];
        if (in.m < 2 || in.n < 1 || in.n >= in.m || in.p < 1 || !in.x || !in.y || !in.z)
            throw MbsError{MBS_ERR_ARG, "shape " + std::to_string(s) + ": need 0 < n < m, p > 0 and point arrays"};
        if (in.k < 0 || in.k > std::min(in.m, in.p) || (in.k == 0 && !(in.eps > 0 && in.eps < 1)))
            throw MbsError{MBS_ERR_ARG, "shape " + std::to_string(s) + ": need 0 < k <= min(m, p) or 0 < eps < 1"};
        if (!(in.proxy_radius > 0))
            throw MbsError{MBS_ERR_ARG, "shape " + std::to_string(s) + ": proxy_radius must be > 0"};
        h.m = in.m;
        h.n = in.n;
        h.p = in.p;
        h.kfix = in.k;
        h.eps = in.eps;
        h.proxy_radius = in.proxy_radius;
        h.x.assign(in.x, in.x + (size_t)d * in.m);
        h.y.assign(in.y, in.y + (size_t)d * in.n);
        h.z.assign(in.z, in.z + (size_t)d * in.p);
        if (!finite_all(h.x.data(), h.x.size()) || !finite_all(h.y.data(), h.y.size()) ||
            !finite_all(h.z.data(), h.z.size()))
            throw MbsError{MBS_ERR_ARG, "shape " + std::to_string(s) + ": non-finite coordinates"};
        double br = 0;
        for (int i = 0; i < in.m; ++i) {
            double r2 = 0;
            for (int a = 0; a < d; ++a) r2 += h.x[(size_t)a * in.m + i] * h.x[(size_t)a * in.m + i];
            br = std::max(br, std::sqrt(r2));
        }
        h.bound_radius = br;
    }
    std::vector<mbs_body> hb(bodies, bodies + nbodies);
    for (int t = 0; t < nbodies; ++t) {
        if (hb[t].shape < 0 || hb[t].shape >= nshapes)
            throw MbsError{MBS_ERR_ARG, "body " + std::to_string(t) + ": bad shape index"};
        if (!finite_all(hb[t].c, 3) || !finite_all(hb[t].R, 9))
            throw MbsError{MBS_ERR_ARG, "body " + std::to_string(t) + ": non-finite placement"};
        hs[hb[t].shape].used = true;
    }
    free_geometry(c);
    c->shapes = std::move(hs);
    c->bodies = std::move(hb);
    c->T = nbodies;
    check_geometry(c);

    // jobs for the used shapes, in batches bounded by a workspace budget
    std::vector<int> used;
    for (int s = 0; s < nshapes; ++s)
        if (c->shapes[s].used) used.push_back(s);
    // longest processing time first: the persistent build kernel takes the jobs
    // in this order, so the big ones start first and the small ones fill the tail
    auto work = [&](int i) {
        const ShapeHost& h = c->shapes[i];
        const double p = h.p, m = h.m, n = h.n, r = std::min(h.p, h.m);
        return p * (m + n) * r + m * r * r + 10.0 * n * n * n;  // QR of B | D, of R_B^H, Jacobi
    };
    std::stable_sort(used.begin(), used.end(), [&](int a, int b2) { return work(a) > work(b2); });
    const size_t ws_budget = (size_t)8 << 30;
    size_t pos = 0;
    while (pos < used.size()) {
        std::vector<int> batch;
        size_t ws = 0;
        while (pos < used.size()) {
            const ShapeHost& s = c->shapes[used[pos]];
            const int kcap = s.kfix > 0 ? s.kfix : std::min(s.m, s.p);
            const size_t need = sizeof(double2) * ((size_t)s.p * (s.m + s.n) + (size_t)kcap * std::max(s.m, s.n) +
                                                   (size_t)std::min(s.p, s.m) * (s.n + s.m + 1) +
                                                   (size_t)s.m * s.n + (size_t)s.n * s.n + s.p + 2 * s.m) +
                                (c->opt.id_sketch > 0 && s.kfix > 0
                                     ? sizeof(double2) * (size_t)(s.kfix + c->opt.id_sketch) * (s.p + s.m + 1)
                                     : 0);
            if (!batch.empty() && ws + need > ws_budget) break;
            batch.push_back(used[pos++]);
            ws += need;
        }
        const int nj = (int)batch.size();
        std::vector<SBuildJob> jobs(nj);
        std::vector<void*> tmp;
        auto talloc = [&](size_t bytes) {
            void* p = dalloc(c, bytes);
            tmp.push_back(p);
            return p;
        };
        int pmax = 1, mmax = 1;
        for (int j = 0; j < nj; ++j) {
            ShapeHost& s = c->shapes[batch[j]];
            SBuildJob& J = jobs[j];
            std::memset(&J, 0, sizeof(J));
            const int kcap = s.kfix > 0 ? s.kfix : std::min(s.m, s.p);
            J.m = s.m;
            J.n = s.n;
            J.p = s.p;
            J.kfix = s.kfix;
            J.eps = s.eps;
            const int dsk = s.kfix + c->opt.id_sketch;
            J.sketch_d = (c->opt.id_sketch > 0 && s.kfix > 0 && dsk < s.p) ? dsk : 0;
            J.seed = c->opt.id_seed;
            J.shape_index = batch[j];
            if (J.sketch_d > 0) {
                J.OM = (double2*)talloc(sizeof(double2) * (size_t)J.sketch_d * s.p);
                J.Y = (double2*)talloc(sizeof(double2) * (size_t)J.sketch_d * s.m);
                J.permY = (int*)talloc(sizeof(int) * s.m);
                J.diagY = (double2*)talloc(sizeof(double2) * std::min(J.sketch_d, s.m));
            }
            s.dx = galloc<double>(c, s.x.size());
            s.dy = galloc<double>(c, s.y.size());
            s.dz = galloc<double>(c, s.z.size());
            MBS_CUDA_TRY(cudaMemcpyAsync(s.dx, s.x.data(), s.x.size() * 8, cudaMemcpyHostToDevice, c->st));
            MBS_CUDA_TRY(cudaMemcpyAsync(s.dy, s.y.data(), s.y.size() * 8, cudaMemcpyHostToDevice, c->st));
            MBS_CUDA_TRY(cudaMemcpyAsync(s.dz, s.z.data(), s.z.size() * 8, cudaMemcpyHostToDevice, c->st));
            J.x = s.dx;
            J.y = s.dy;
            J.z = s.dz;
            J.BD = (double2*)talloc(sizeof(double2) * (size_t)s.p * (s.m + s.n));
            s.AU = galloc<double2>(c, (size_t)s.m * (s.n + kcap));
            J.AU = s.AU;
            J.W1 = (double2*)talloc(sizeof(double2) * (size_t)kcap * std::max(s.m, s.n));
            J.W2 = (double2*)talloc(sizeof(double2) * (size_t)std::min(s.p, s.m) * s.n);
            J.W3 = (double2*)talloc(sizeof(double2) * (size_t)s.m * s.n);
            J.XB = (double2*)talloc(sizeof(double2) * (size_t)s.m * std::min(s.p, s.m));
            J.XA = (double2*)talloc(sizeof(double2) * (size_t)s.n * s.n);
            J.sig = (double*)talloc(sizeof(double) * s.n);
            J.keep = (int*)talloc(sizeof(int) * s.n);
            J.nrm2 = (double*)talloc(sizeof(double) * std::max(s.m, s.n));
            J.permB = (int*)talloc(sizeof(int) * s.m);
            J.diagB = (double2*)talloc(sizeof(double2) * std::min(s.p, s.m));
            J.permA = (int*)talloc(sizeof(int) * s.n);
            J.diagA = (double2*)talloc(sizeof(double2) * s.n);
            s.JA = galloc<double2>(c, (size_t)s.n * s.n);
            s.FA = galloc<double2>(c, (size_t)s.n * s.n);
            J.JA = s.JA;
            J.FA = s.FA;
            J.skel = (int*)talloc(sizeof(int) * kcap);
            s.Zs = galloc<double2>(c, (size_t)kcap * s.m);
            s.C = galloc<double2>(c, (size_t)s.m * s.n);
            s.S64 = galloc<double2>(c, (size_t)kcap * kcap);
            J.Zs = s.Zs;
            J.C = s.C;
            J.S = s.S64;
            pmax = std::max(pmax, s.p);
            mmax = std::max(mmax, s.m);
        }
        SBuildJob* d_jobs = (SBuildJob*)talloc(sizeof(SBuildJob) * nj);
        int* d_counter = (int*)talloc(3 * sizeof(int));
        MBS_CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(SBuildJob) * nj, cudaMemcpyHostToDevice, c->st));
        const int rows_max = std::max(pmax, mmax);
        const int threads = sbuild_threads(c, d_jobs, nj, d_counter, rows_max);
        launch_sbuild(d, d_jobs, nj, d_counter, rows_max, threads, c->kappa, c->opt.ls_rcond, c->st);
        c->last_sbuild_threads = threads;
        MBS_CUDA_TRY(cudaMemcpyAsync(jobs.data(), d_jobs, sizeof(SBuildJob) * nj, cudaMemcpyDeviceToHost, c->st));
        MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
        for (int j = 0; j < nj; ++j) {
            ShapeHost& s = c->shapes[batch[j]];
            const SBuildJob& J = jobs[j];
            s.k = J.k;
            s.rankA = J.rankA;
            s.rankB = J.rankB;
            s.rankS = J.rankS;
            s.sweepsA = J.sweepsA;
            s.snorm = J.snorm;
            s.eps_ach = J.eps_ach;
            if (s.k < 1) throw MbsError{MBS_ERR_ARG, "shape " + std::to_string(batch[j]) + ": zero skeleton"};
            s.skel.resize(s.k);
            MBS_CUDA_TRY(cudaMemcpy(s.skel.data(), J.skel, s.k * sizeof(int), cudaMemcpyDeviceToHost));
            // Z* and S were written with leading dimension k (<= kcap): already compact.
            s.S32 = galloc<float2>(c, (size_t)s.k * s.k);
            launch_f64_to_f32(s.S64, s.S32, (int64_t)s.k * s.k, c->st);
        }
        MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
        for (void* p : tmp) dfree(c, p);
    }
    setup_layout(c);
    c->built = true;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void mbs_default_options(mbs_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = MBS_PREC_FP64;
    o->tol = 1e-11;
    o->inner_tol = 1e-6;
    o->restart = 60;
    o->max_iter = 20000;
    o->max_sweeps = 8;
    o->ls_rcond = 1e-14;
    o->stream = nullptr;
    o->hbm_budget = 0;
    o->tile_override = 0;
    o->block_krylov = 1;
    o->mac_path = 0;
    o->autotune = 1;
    o->cuda_graphs = 1;
    o->fp64_kernel = 2;
    o->sbuild_threads = 0;
    o->id_sketch = 0;
    o->id_seed = 0;
}

mbs_status mbs_create(int dim, double kappa, const mbs_options* opt, mbs_ctx** out) {
    if (!out) return MBS_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !(kappa > 0) || !std::isfinite(kappa)) return MBS_ERR_ARG;
    mbs_options o;
    if (opt)
        o = *opt;
    else
        mbs_default_options(&o);
    try {
        validate_options(o);
    } catch (const MbsError& e) {
        return e.st;
    }
    mbs_ctx* c = new mbs_ctx();
    c->dim = dim;
    c->kappa = kappa;
    c->opt = o;
    if (o.stream) {
        c->st = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return MBS_ERR_CUDA;
        }
        c->own_stream = true;
    }
    *out = c;
    return MBS_OK;
}

int64_t mbs_launch_count(void) { return (int64_t)g_mbs_launches.load(); }

mbs_status mbs_profile(mbs_ctx* c, int enable) {
    return guarded(c, [&]() {
        if ((enable != 0) != c->profile) clear_graphs(c);  // graphs hold timing events or not
        c->profile = enable != 0;
        return MBS_OK;
    });
}

mbs_status mbs_kernel_times(mbs_ctx* c, double* out) {
    return guarded(c, [&]() {
        if (!out) throw MbsError{MBS_ERR_ARG, "null output"};
        MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
        double t[2] = {0.0, 0.0};
        size_t n[2] = {c->ev32.size(), c->ev64.size()};
        std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* lists[2] = {&c->ev32, &c->ev64};
        for (int a = 0; a < 2; ++a) {
            for (auto& pr : *lists[a]) {
                float ms = 0.f;
                MBS_CUDA_TRY(cudaEventElapsedTime(&ms, pr.first, pr.second));
                t[a] += ms;
                c->ev_pool.push_back(pr.first);
                c->ev_pool.push_back(pr.second);
            }
            lists[a]->clear();
        }
        out[0] = t[0] + c->graph_ms[0];
        out[1] = (double)n[0] + (double)c->graph_n[0];
        out[2] = t[1] + c->graph_ms[1];
        out[3] = (double)n[1] + (double)c->graph_n[1];
        out[4] = c->last_path;
        out[5] = c->last_nsplit;
        out[6] = c->last_sbuild_threads;
        c->graph_ms[0] = c->graph_ms[1] = 0.0;
        c->graph_n[0] = c->graph_n[1] = 0;
        return MBS_OK;
    });
}

void mbs_destroy(mbs_ctx* c) {
    if (!c) return;
    {
        std::lock_guard<std::mutex> g(c->mu);
        free_geometry(c);
        if (c->st) cudaStreamSynchronize(c->st);
        for (auto& pr : c->ev32) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        for (auto& pr : c->ev64) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
        for (auto& kv : c->bufs) dfree(c, kv.second.p);
        c->bufs.clear();
        dfree(c, c->d_err);
        c->d_err = nullptr;
        if (c->pinned) cudaFreeHost(c->pinned);
        c->pinned = nullptr;
        if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    }
    delete c;
}

mbs_status mbs_set_options(mbs_ctx* c, const mbs_options* opt) {
    return guarded(c, [&]() {
        if (!opt) throw MbsError{MBS_ERR_ARG, "null options"};
        validate_options(*opt);
        if (opt->stream && opt->stream != (void*)c->st) {
            if (c->own_stream) {
                cudaStreamSynchronize(c->st);
                cudaStreamDestroy(c->st);
                c->own_stream = false;
            }
            c->st = (cudaStream_t)opt->stream;
        }
        void* keep = c->opt.stream;
        clear_graphs(c);
        c->opt = *opt;
        if (!opt->stream) c->opt.stream = keep;
        return MBS_OK;
    });
}

const char* mbs_last_error(const mbs_ctx* c) { return c ? c->err.c_str() : "null context"; }

mbs_status mbs_build_scattering_matrices(mbs_ctx* c, int nshapes, const mbs_shape* shapes,
                                          int nbodies, const mbs_body* bodies) {
    return guarded(c, [&]() {
        build(c, nshapes, shapes, nbodies, bodies);
        return MBS_OK;
    });
}

mbs_status mbs_get_layout(mbs_ctx* c, int64_t* N, int64_t* body_offsets, double* skel_xyz) {
    return guarded(c, [&]() {
        require_built(c);
        if (N) *N = c->N;
        if (body_offsets) std::memcpy(body_offsets, c->off.data(), (c->T + 1) * sizeof(int64_t));
        if (skel_xyz) std::memcpy(skel_xyz, c->skel_world.data(), c->skel_world.size() * sizeof(double));
        return MBS_OK;
    });
}

mbs_status mbs_get_shape(mbs_ctx* c, int shape, int* k, int* skel, double* S, double* eps_achieved) {
    return guarded(c, [&]() {
        require_built(c);
        if (shape < 0 || shape >= (int)c->shapes.size() || !c->shapes[shape].used)
            throw MbsError{MBS_ERR_ARG, "shape not built"};
        const ShapeHost& s = c->shapes[shape];
        if (k) *k = s.k;
        if (skel) std::memcpy(skel, s.skel.data(), s.k * sizeof(int));
        if (eps_achieved) *eps_achieved = s.eps_ach;
        if (S) MBS_CUDA_TRY(cudaMemcpy(S, s.S64, (size_t)s.k * s.k * sizeof(double2), cudaMemcpyDeviceToHost));
        return MBS_OK;
    });
}

mbs_status mbs_get_shape_stats(mbs_ctx* c, int shape, int* rank_b, int* rank_a_qr, int* rank_a,
                               int* sweeps, double* s_norm) {
    return guarded(c, [&]() {
        require_built(c);
        if (shape < 0 || shape >= (int)c->shapes.size() || !c->shapes[shape].used)
            throw MbsError{MBS_ERR_ARG, "shape not built"};
        const ShapeHost& s = c->shapes[shape];
        if (s.injected) throw MbsError{MBS_ERR_STATE, "shape holds injected scattering data"};
        if (rank_b) *rank_b = s.rankB;
        if (rank_a_qr) *rank_a_qr = s.rankA;
        if (rank_a) *rank_a = s.rankS;
        if (sweeps) *sweeps = s.sweepsA;
        if (s_norm) *s_norm = s.snorm;
        return MBS_OK;
    });
}

mbs_status mbs_rhs(mbs_ctx* c, int nrhs, const double* v, double* b) {
    return guarded(c, [&]() {
        require_built(c);
        if (nrhs < 1 || !v || !b) throw MbsError{MBS_ERR_ARG, "bad nrhs or null pointer"};
        for (const mbs_body& B : c->bodies)
            if (!c->shapes[B.shape].rhs_ok)
                throw MbsError{MBS_ERR_STATE, "a shape's skeleton was injected without its W"};
        const double2* dv = in_dev(c, v, (size_t)c->Mtot * nrhs, "io_v");
        OutBuf ob = out_dev(c, b, (size_t)c->N * nrhs, "io_b");
        launch_rhs(c->d_rhsb, c->T, nrhs, c->mmax, c->nmax, dv, c->Mtot, ob.dev, c->N, c->st);
        finish_out(c, ob);
        return MBS_OK;
    });
}

mbs_status mbs_apply_G(mbs_ctx* c, int precision, int nrhs, const double* q, double* y) {
    return guarded(c, [&]() {
        require_built(c);
        if (nrhs < 1 || !q || !y) throw MbsError{MBS_ERR_ARG, "bad nrhs or null pointer"};
        const size_t n = (size_t)c->N * nrhs;
        const double2* dq = in_dev(c, q, n, "io_q");
        OutBuf oy = out_dev(c, y, n, "io_y");
        if (precision == MBS_PREC_FP32) {
            float2* q32 = scratch<float2>(c, "io_q32", n);
            float2* y32 = scratch<float2>(c, "io_y32", n);
            launch_f64_to_f32(dq, q32, (int64_t)n, c->st);
            G32(c, nrhs, q32, y32);
            launch_f32_to_f64(y32, oy.dev, (int64_t)n, c->st);
        } else if (precision == MBS_PREC_FP64) {
            G64(c, nrhs, dq, oy.dev);
        } else {
            throw MbsError{MBS_ERR_ARG, "precision must be FP64 or FP32"};
        }
        finish_out(c, oy);
        return MBS_OK;
    });
}

mbs_status mbs_apply_operator(mbs_ctx* c, int nrhs, const double* qhat, double* y) {
    return guarded(c, [&]() {
        require_built(c);
        if (nrhs < 1 || !qhat || !y) throw MbsError{MBS_ERR_ARG, "bad nrhs or null pointer"};
        const size_t n = (size_t)c->N * nrhs;
        const double2* dq = in_dev(c, qhat, n, "io_q");
        OutBuf oy = out_dev(c, y, n, "io_y");
        if (c->opt.precision == MBS_PREC_FP64) {
            op64(c, nrhs, dq, oy.dev);
        } else {
            float2* q32 = scratch<float2>(c, "io_q32", n);
            float2* y32 = scratch<float2>(c, "io_y32", n);
            launch_f64_to_f32(dq, q32, (int64_t)n, c->st);
            op32(c, nrhs, q32, y32);
            launch_f32_to_f64(y32, oy.dev, (int64_t)n, c->st);
        }
        finish_out(c, oy);
        return MBS_OK;
    });
}

mbs_status mbs_solve(mbs_ctx* c, int nrhs, const double* b, double* qhat, mbs_solve_info* info) {
    return guarded(c, [&]() -> mbs_status {
        require_built(c);
        if (nrhs < 1 || !b || !qhat) throw MbsError{MBS_ERR_ARG, "bad nrhs or null pointer"};
        const auto t0 = std::chrono::steady_clock::now();
        // FP64-accurate G_hat of this solve: under fp64_kernel = 2, double-float
        // when the residual floor it leaves stays below a tenth of tol.  Its
        // ~1e-13 relative error in G_hat q reaches the residual through S:
        // measured, ~1e-14 relative per unit of ||S||; over many bodies the
        // errors add in norm, so the root mean square of ||S_tau||_F counts
        const int k64 = c->opt.fp64_kernel;
        const bool df = k64 == 1 || (k64 == 2 && 1e-14 * c->snorm_rms <= 0.1 * c->opt.tol);
        if (k64 == 2 && df != c->df_active) {
            clear_graphs(c);  // captured FP64 steps hold the other kernel
            c->df_active = df;
        }
        struct InSolve {
            mbs_ctx* c;
            ~InSolve() { c->in_solve = false; }
        } in_solve_guard{c};
        c->in_solve = true;
        const size_t n = (size_t)c->N * nrhs;
        const double2* db = in_dev(c, b, n, "io_b_in");
        OutBuf ox = out_dev(c, qhat, n, "io_x");
        if (ox.host)
            MBS_CUDA_TRY(cudaMemcpyAsync(ox.dev, qhat, n * sizeof(double2), cudaMemcpyHostToDevice, c->st));
        // is the initial guess zero?
        std::vector<double> xn = norms<double2>(c, ox.dev, nrhs);
        bool xzero = true;
        for (double v : xn) xzero = xzero && v == 0.0;
        mbs_solve_info inf;
        std::memset(&inf, 0, sizeof(inf));
        bool conv = false;
        double relmax = 0.0;
        const mbs_options& o = c->opt;
        if (o.precision == MBS_PREC_FP64 || o.precision == MBS_PREC_FP32) {
            GmresStats S = krylov<double2>(c, nrhs, db, ox.dev, xzero, o.tol, o.restart, o.max_iter, true);
            inf.inner_iterations = S.iters;
            inf.matvecs_fp64 = S.matvecs;
            inf.sweeps = 1;
            conv = S.converged;
            for (double v : S.relres) relmax = std::max(relmax, v);
        } else {
            // FP32 GMRES inside FP64 iterative refinement
            double2* r64 = scratch<double2>(c, "ir_r64", n);
            double2* t64 = scratch<double2>(c, "ir_t64", n);
            float2* r32 = scratch<float2>(c, "ir_r32", n);
            float2* d32 = scratch<float2>(c, "ir_d32", n);
            double* d_sc = scratch<double>(c, "ir_scale", nrhs);
            const std::vector<double> bn = norms<double2>(c, db, nrhs);
            if (xzero) {
                MBS_CUDA_TRY(cudaMemcpyAsync(r64, db, n * sizeof(double2), cudaMemcpyDeviceToDevice, c->st));
            } else {
                op64(c, nrhs, ox.dev, t64);
                inf.matvecs_fp64++;
                launch_sub<double2>(db, t64, r64, (int64_t)n, c->st);
            }
            std::vector<double> sc(nrhs);
            double prev = 1e300;
            bool stalled = false;
            while (true) {
                const std::vector<double> rn = norms<double2>(c, r64, nrhs);
                relmax = 0.0;
                bool all = true;
                for (int q = 0; q < nrhs; ++q) {
                    const double rel = bn[q] > 0 ? rn[q] / bn[q] : 0.0;
                    relmax = std::max(relmax, rel);
                    all = all && rel <= o.tol;
                }
                if (all) {
                    conv = true;
                    break;
                }
                if (inf.inner_iterations >= o.max_iter) break;
                // refinement no longer contracts: the FP32 operator is too inaccurate
                // for this problem (e.g. large S of corner-refined bodies)
                if (inf.sweeps >= o.max_sweeps || relmax > 0.5 * prev) {
                    stalled = true;
                    break;
                }
                prev = relmax;
                // Block GMRES needs every column non-zero (a zero column makes the
                // block rank deficient and ends the solve at once): right-hand sides
                // that have converged stay in the block, where the correction only
                // lowers their residual further; the lockstep solver freezes them.
                const bool block = nrhs > 1 && nrhs <= 16 && o.block_krylov;
                for (int q = 0; q < nrhs; ++q) {
                    const double rel = bn[q] > 0 ? rn[q] / bn[q] : 0.0;
                    sc[q] = ((block || rel > o.tol) && rn[q] > 0) ? 1.0 / rn[q] : 0.0;
                }
                // The last sweep needs only the reduction that is left to reach tol
                // (with a factor 2 of margin): inner tolerance max(inner_tol, 0.5 tol /
                // residual), but always at least a 10x reduction so that the sweep
                // contracts.
                const double left = relmax > 0 ? 0.5 * o.tol / relmax : 0.0;
                const double itol = std::max(o.inner_tol, std::min(0.1, left));
                MBS_CUDA_TRY(cudaMemcpyAsync(d_sc, sc.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c->st));
                launch_f64_to_f32_scaled(r64, d_sc, r32, c->N, nrhs, c->st);
                GmresStats S = krylov<float2>(c, nrhs, r32, d32, true, itol, o.restart,
                                             o.max_iter - inf.inner_iterations, false);
                inf.inner_iterations += S.iters;
                inf.matvecs_fp32 += S.matvecs;
                for (int q = 0; q < nrhs; ++q) sc[q] = sc[q] > 0 ? rn[q] : 0.0;
                MBS_CUDA_TRY(cudaMemcpyAsync(d_sc, sc.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, c->st));
                launch_axpy_f32_into_f64(d32, d_sc, ox.dev, c->N, nrhs, c->st);
                op64(c, nrhs, ox.dev, t64);
                inf.matvecs_fp64++;
                launch_sub<double2>(db, t64, r64, (int64_t)n, c->st);
                inf.sweeps++;
            }
            if (stalled && inf.inner_iterations < o.max_iter) {
                // finish in FP64 from the refined iterate
                GmresStats S = krylov<double2>(c, nrhs, db, ox.dev, false, o.tol, o.restart,
                                               o.max_iter - inf.inner_iterations, true);
                inf.inner_iterations += S.iters;
                inf.matvecs_fp64 += S.matvecs;
                inf.fp64_finish = 1;
                conv = S.converged;
                relmax = 0.0;
                for (double v : S.relres) relmax = std::max(relmax, v);
            }
        }
        finish_out(c, ox);
        inf.converged = conv ? 1 : 0;
        inf.rel_residual = relmax;
        inf.fp64_kernel = df ? 1 : 0;
        inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (info) *info = inf;
        if (!conv) {
            char msg[160];
            std::snprintf(msg, sizeof(msg), "solve did not reach tol %.3e (relative residual %.3e)", o.tol,
                          relmax);
            c->err = msg;
            return MBS_ERR_NOCONV;
        }
        return MBS_OK;
    });
}

mbs_status mbs_evaluate_field(mbs_ctx* c, int nrhs, int64_t M, const double* pts,
                              const double* qhat, double* u) {
    return guarded(c, [&]() {
        require_built(c);
        if (nrhs < 1 || M < 0 || (M > 0 && (!pts || !qhat || !u)))
            throw MbsError{MBS_ERR_ARG, "bad sizes or null pointer"};
        if (M == 0) return MBS_OK;
        // targets must lie on or outside every proxy surface
        const std::vector<int> tb = proxy_bodies(c, pts, M);
        for (int64_t i = 0; i < M; ++i)
            if (tb[i] >= 0)
                throw MbsError{MBS_ERR_NEAR_TARGET, "target " + std::to_string(i) +
                                                        " lies inside the proxy surface of body " +
                                                        std::to_string(tb[i])};
        const double* dp = in_dev_real(c, pts, (size_t)c->dim * M, "io_pts");
        const double2* dq = in_dev(c, qhat, (size_t)c->N * nrhs, "io_q");
        OutBuf ou = out_dev(c, u, (size_t)M * nrhs, "io_u");
        int ns;
        int* sb = split_for(c, M, &ns);
        double2* part = scratch<double2>(c, "part_field", (size_t)ns * nrhs * M);
        launch_field_f64(glayout(c), c->kappa, M, dp, nrhs, dq, ou.dev, part, ns, sb, c->st);
        finish_out(c, ou);
        return MBS_OK;
    });
}

mbs_status mbs_reconstruct(mbs_ctx* c, int nrhs, const double* v, const double* qhat, double* qmfs) {
    return guarded(c, [&]() {
        require_built(c);
        if (nrhs < 1 || !v || !qhat || !qmfs) throw MbsError{MBS_ERR_ARG, "bad nrhs or null pointer"};
        for (const mbs_body& B : c->bodies)
            if (c->shapes[B.shape].injected)
                throw MbsError{MBS_ERR_STATE, "reconstruction needs the built scattering data (a shape was injected)"};
        const double2* dv = in_dev(c, v, (size_t)c->Mtot * nrhs, "io_v");
        const double2* dq = in_dev(c, qhat, (size_t)c->N * nrhs, "io_q");
        OutBuf om = out_dev(c, qmfs, (size_t)c->Nm * nrhs, "io_qmfs");
        double2* w_hat = scratch<double2>(c, "rec_w", (size_t)c->N * nrhs);
        G64(c, nrhs, dq, w_hat);  // incoming field at every skeleton point from the other bodies
        launch_recon(c->d_rhsb, c->T, nrhs, c->mmax, c->nmax, dv, c->Mtot, w_hat, c->N, om.dev, c->Nm,
                     c->st);
        finish_out(c, om);
        return MBS_OK;
    });
}

mbs_status mbs_evaluate_field_near(mbs_ctx* c, int nrhs, int64_t M, const double* pts,
                                   const double* qhat, const double* qmfs, double* u) {
    return guarded(c, [&]() {
        require_built(c);
        if (nrhs < 1 || M < 0 || (M > 0 && (!pts || !qhat || !qmfs || !u)))
            throw MbsError{MBS_ERR_ARG, "bad sizes or null pointer"};
        if (M == 0) return MBS_OK;
        const std::vector<int> tb = proxy_bodies(c, pts, M);
        int* d_tb = scratch<int>(c, "near_tb", (size_t)M);
        MBS_CUDA_TRY(cudaMemcpyAsync(d_tb, tb.data(), (size_t)M * sizeof(int), cudaMemcpyHostToDevice, c->st));
        const double* dp = in_dev_real(c, pts, (size_t)c->dim * M, "io_pts");
        const double2* dq = in_dev(c, qhat, (size_t)c->N * nrhs, "io_q");
        const double2* dm = in_dev(c, qmfs, (size_t)c->Nm * nrhs, "io_qmfs_in");
        OutBuf ou = out_dev(c, u, (size_t)M * nrhs, "io_u");
        int ns;
        int* sb = split_for(c, M, &ns);
        double2* part = scratch<double2>(c, "part_field", (size_t)ns * nrhs * M);
        // skeleton sums of every body but the one whose proxy holds the target ...
        launch_field_f64(glayout(c), c->kappa, M, dp, nrhs, dq, ou.dev, part, ns, sb, c->st, d_tb);
        // ... plus that body's reconstructed MFS sources
        launch_mfs_near(c->dim, M, dp, d_tb, c->d_mfsb, c->kappa, nrhs, dm, c->Nm, ou.dev, c->st);
        finish_out(c, ou);
        return MBS_OK;
    });
}

mbs_status mbs_inject_scattering(mbs_ctx* c, int shape, int k, const int* skel, const double* S,
                                 const double* W) {
    return guarded(c, [&]() {
        if (!c->built) throw MbsError{MBS_ERR_STATE, "scattering matrices not built"};
        if (shape < 0 || shape >= (int)c->shapes.size() || !c->shapes[shape].used)
            throw MbsError{MBS_ERR_ARG, "shape not built"};
        ShapeHost& s = c->shapes[shape];
        if (k < 1 || k > s.m || !skel || !S) throw MbsError{MBS_ERR_ARG, "bad k / skel / S"};
        for (int i = 0; i < k; ++i)
            if (skel[i] < 0 || skel[i] >= s.m) throw MbsError{MBS_ERR_ARG, "skeleton index out of range"};
        const bool same = k == s.k && std::equal(skel, skel + k, s.skel.begin());
        s.rhs_ok = W != nullptr || (same && s.rhs_ok);
        s.injected = true;
        MBS_CUDA_TRY(cudaStreamSynchronize(c->st));
        s.k = k;
        s.skel.assign(skel, skel + k);
        s.S64 = galloc<double2>(c, (size_t)k * k);
        s.S32 = galloc<float2>(c, (size_t)k * k);
        MBS_CUDA_TRY(cudaMemcpy(s.S64, S, (size_t)k * k * sizeof(double2), cudaMemcpyHostToDevice));
        launch_f64_to_f32(s.S64, s.S32, (int64_t)k * k, c->st);
        double sq = 0.0;
        for (size_t e = 0; e < (size_t)2 * k * k; ++e) sq += S[e] * S[e];
        s.snorm = std::sqrt(sq);
        if (W) {
            s.W = galloc<double2>(c, (size_t)k * s.m);
            MBS_CUDA_TRY(cudaMemcpy(s.W, W, (size_t)k * s.m * sizeof(double2), cudaMemcpyHostToDevice));
        } else {
            s.W = nullptr;
        }
        c->layout_dirty = true;  // rebuilt by the next call that needs the layout
        return MBS_OK;
    });
}

}  // extern "C"
