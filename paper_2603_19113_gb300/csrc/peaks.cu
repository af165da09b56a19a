// Short microbenchmarks of the device's arithmetic peaks, the denominators of
// the roofline fractions: FP32 FMA (scalar and packed f32x2), FP64 FMA and
// MUFU (sin + cos + rsqrt).
#include <cstring>

#include "common.cuh"

namespace {

constexpr int PK_ITERS = 4096;

__global__ void fma32_kernel(float* out, float a, float b) {
    float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f;
    float x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f, x7 = x0 + 7.f;
#pragma unroll 16
    for (int i = 0; i < PK_ITERS; ++i) {
        x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
        x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
    const float s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 12345.678f) out[0] = s;
}

// Packed FP32: one fma.rn.f32x2 performs two independent FMAs (sm_100 family).
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__global__ void fma32x2_kernel(float* out, float a, float b) {
    const float x = threadIdx.x * 1e-3f;
    unsigned long long x0 = pack2(x, x + 1.f), x1 = pack2(x + 2.f, x + 3.f);
    unsigned long long x2 = pack2(x + 4.f, x + 5.f), x3 = pack2(x + 6.f, x + 7.f);
    const unsigned long long aa = pack2(a, a), bb = pack2(b, b);
#pragma unroll 16
    for (int i = 0; i < PK_ITERS; ++i) {
        asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x0) : "l"(aa), "l"(bb));
        asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x1) : "l"(aa), "l"(bb));
        asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x2) : "l"(aa), "l"(bb));
        asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x3) : "l"(aa), "l"(bb));
    }
    float s = 0.f;
    for (unsigned long long v : {x0, x1, x2, x3}) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
        s += lo + hi;
    }
    if (s == 12345.678f) out[0] = s;
}

__global__ void fma64_kernel(double* out, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
#pragma unroll 16
    for (int i = 0; i < PK_ITERS / 8; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    }
    const double s = x0 + x1 + x2 + x3;
    if (s == 12345.678) out[0] = s;
}

__global__ void mufu_kernel(float* out) {
    float x = threadIdx.x * 1e-3f, y = 0.5f, z = 0.25f;
#pragma unroll 8
    for (int i = 0; i < PK_ITERS / 4; ++i) {
        x = __sinf(x);
        y = __cosf(y);
        z = rsqrtf(z + 1.f);
    }
    const float s = x + y + z;
    if (s == 12345.678f) out[0] = s;
}

template <typename F>
float time_kernel(F f) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    f();  // warm-up
    cudaEventRecord(a);
    for (int r = 0; r < 5; ++r) f();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms / 5.f;
}

}  // namespace

extern "C" mbs_status mbs_measure_peaks(double* out) {
    if (!out) return MBS_ERR_ARG;
    int dev = 0, sms = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MBS_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    float* d32 = nullptr;
    double* d64 = nullptr;
    if (cudaMalloc(&d32, 16) != cudaSuccess || cudaMalloc(&d64, 16) != cudaSuccess) {
        cudaGetLastError();
        return MBS_ERR_NOMEM;
    }
    const int blocks = sms * 8, threads = 256;
    const double thr = (double)blocks * threads;
    const float t32 = time_kernel([&] { fma32_kernel<<<blocks, threads>>>(d32, 0.999f, 1e-3f); });
    const float t64 = time_kernel([&] { fma64_kernel<<<blocks, threads>>>(d64, 0.999, 1e-3); });
    const float tmu = time_kernel([&] { mufu_kernel<<<blocks, threads>>>(d32); });
    const float t2 = time_kernel([&] { fma32x2_kernel<<<blocks, threads>>>(d32, 0.999f, 1e-3f); });
    const cudaError_t e = cudaDeviceSynchronize();
    cudaFree(d32);
    cudaFree(d64);
    if (e != cudaSuccess) return MBS_ERR_CUDA;
    out[0] = thr * PK_ITERS * 8 * 2 / (t32 * 1e-3) / 1e12;        // FP32 TFLOP/s
    out[1] = thr * (PK_ITERS / 8) * 4 * 2 / (t64 * 1e-3) / 1e12;  // FP64 TFLOP/s
    out[2] = thr * (PK_ITERS / 4) * 3 / (tmu * 1e-3) / 1e12;       // MUFU Tops/s
    out[3] = sms;
    out[4] = khz;
    out[5] = thr * PK_ITERS * 8 * 2 / (t2 * 1e-3) / 1e12;         // FP32 TFLOP/s, f32x2
    return MBS_OK;
}
