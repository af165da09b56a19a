// Allocation-free FP64 G_hat matvec (mbs_apply_G_noalloc).
//
// For callers that must not allocate device memory once they are running,
// for example an application that hands out all of its GPU memory from its
// own fixed pool at start-up, or a real-time loop in which a cudaMalloc (which
// may synchronise the device) is not allowed.  The caller owns every input
// and output buffer; the only extra device memory is the file-scope array
// below, reserved when the library is loaded and held by every GPU that
// loads the library until the process exits.
//
// The array keeps the source-split table and the per-split partial sums of
// the block-masked all-pairs sum.  Every call overwrites the parts it reads
// (the split table and every partial-sum entry of its size), so nothing needs
// clearing between calls; calls that overlap on the GPU (different streams or
// threads at the same time) share the array and race.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t NOALLOC_BYTES = (size_t)64 << 20;  // 64 MiB
constexpr size_t SPLIT_BYTES = 512;                 // room for the split table (<= 64 splits)
constexpr int MAX_SPLIT = 64;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_setup_mu;
void* g_scratch_ptr[MAX_DEVICES] = {nullptr};

// split_body[s] = first body b with off[b] >= s * N / nsplit (s = 0..nsplit)
__global__ void split_table_kernel(const int64_t* __restrict__ off, int T, int64_t N, int nsplit,
                                   int* __restrict__ split_body) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nsplit) return;
    if (s == 0) {
        split_body[0] = 0;
        return;
    }
    if (s == nsplit) {
        split_body[s] = T;
        return;
    }
    const int64_t target = (N * s) / nsplit;
    int lo = 0, hi = T;  // lower bound over off[0..T]
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (off[mid] < target)
            lo = mid + 1;
        else
            hi = mid;
    }
    split_body[s] = lo;
}

// Device address of the scratch array on the current device, looked up once
// per device (the array's name in host code is not a device address).
mbs_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return MBS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MBS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return MBS_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" mbs_status mbs_apply_G_noalloc(int dim, double kappa, int64_t N, int T,
                                          const int64_t* body_offsets, const int* body,
                                          const double* xw, int nrhs, const double* q, double* y,
                                          void* stream) {
    if ((dim != 2 && dim != 3) || !(kappa > 0) || N < 0 || T < 1 || nrhs < 1) return MBS_ERR_ARG;
    const size_t cap = (NOALLOC_BYTES - SPLIT_BYTES) / sizeof(double2);
    // beyond the static scratch; compared without forming N * nrhs, which could wrap
    if ((uint64_t)N > cap || (size_t)nrhs > cap / (size_t)std::max<int64_t>(N, 1)) return MBS_ERR_ARG;
    if (N == 0) return MBS_OK;
    if (!on_device(body_offsets) || !on_device(body) || !on_device(xw) || !on_device(q) ||
        !on_device(y))
        return MBS_ERR_ARG;
    void* base = nullptr;
    const mbs_status st = scratch_address(&base);
    if (st != MBS_OK) return st;
    // as many source splits as wanted for load balance and as fit in the array
    const int64_t tiles = (N + 255) / 256;
    int64_t ns = (16LL * mbs_num_sms() + tiles - 1) / tiles;
    ns = std::min<int64_t>(ns, (int64_t)(cap / ((size_t)N * nrhs)));
    ns = std::max<int64_t>(1, std::min<int64_t>(ns, std::min(T, MAX_SPLIT)));
    int* split_body = static_cast<int*>(base);
    double2* part = reinterpret_cast<double2*>(static_cast<unsigned char*>(base) + SPLIT_BYTES);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    try {
        split_table_kernel<<<1, 128, 0, s>>>(body_offsets, T, N, (int)ns, split_body);
        MBS_CHECK_LAUNCH();
        GLayout L{};
        L.dim = dim;
        L.T = T;
        L.N = N;
        L.body = body;
        L.off = body_offsets;
        L.xw64 = xw;
        launch_G_f64(L, kappa, nrhs, reinterpret_cast<const double2*>(q),
                     reinterpret_cast<double2*>(y), part, (int)ns, split_body, s);
    } catch (const MbsError& e) {
        return e.st;
    }
    return MBS_OK;
}
