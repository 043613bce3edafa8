// Arithmetic-pipe micro-benchmarks: the FP64 FMA, FP32 FMA and MUFU ex2
// throughput of the device, measured with long independent dependency chains
// (8 per thread, enough warps per SM to cover latency).  These give the
// denominators of the region-evaluation roofline, which is bound by the FP64
// pipe (all-FP64 evaluation) or by the FP32 + SFU pipes (FP32 evaluation).
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;

__global__ void k_dfma(double* out, int iters, double b, double c)
{
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678) out[threadIdx.x] = s;   // keeps the chains live
}

__global__ void k_ffma(float* out, int iters, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-3f * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_neg(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}

__global__ void k_mufu(float* out, int iters)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = ex2_neg(a[k]);   // stays in [0.5, 1]
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[threadIdx.x] = s;
}

}  // namespace

extern "C" {

// which: 0 = FP64 FMA, 1 = FP32 FMA, 2 = MUFU ex2.  Writes the best of `reps`
// runs as operations per second (an FMA counts as 2 flops; an ex2 as 1 op)
// and that run's seconds.  Returns 0, or a CUDA error code.
int pipe_peak(int which, int device, int reps, double* ops_per_s, double* seconds)
{
    if (cudaSetDevice(device) != cudaSuccess) return 1;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return 1;
    const int threads = 256;
    const int blocks = p.multiProcessorCount * 8;
    int iters = which == 0 ? 2048 : (which == 1 ? 65536 : 16384);
    void* out = nullptr;
    if (cudaMalloc(&out, threads * sizeof(double)) != cudaSuccess) return 2;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double best = 0.0, best_s = 0.0;
    for (int r = 0; r < reps + 1; ++r) {
        cudaEventRecord(a);
        if (which == 0) k_dfma<<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
        else if (which == 1) k_ffma<<<blocks, threads>>>((float*)out, iters, 0.999f, 1e-4f);
        else k_mufu<<<blocks, threads>>>((float*)out, iters);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double ops = double(blocks) * threads * kChains * iters * (which == 2 ? 1.0 : 2.0);
        if (r > 0 && ops / (ms * 1e-3) > best) { best = ops / (ms * 1e-3); best_s = ms * 1e-3; }
    }
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    *ops_per_s = best;
    *seconds = best_s;
    return e == cudaSuccess ? 0 : int(e);
}

}  // extern "C"
