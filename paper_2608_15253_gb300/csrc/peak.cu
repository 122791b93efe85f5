// Arithmetic throughput probes of the GPU the library runs on: a grid of
// independent fused multiply-add chains in FP32 or FP64, timed with CUDA
// events.  They give measured denominators for the rooflines of kernels that
// are bound by plain ALU arithmetic (the FP64 path, the one-cell replica
// kernels) rather than by memory.
#include <cuda_runtime.h>

#include "ctx.h"

namespace mm {

constexpr int kPeakChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T* out, int iters, T a, T b) {
    T x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    // a store the compiler cannot prove dead (a and b make it never happen)
    if (s == (T)-1.2345e30) out[threadIdx.x] = s;
}

template <typename T>
static mm_status measure(double* flops_per_s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return MM_ERR_DEVICE;
    T* out = nullptr;
    if (cudaMalloc(&out, 256 * sizeof(T)) != cudaSuccess) return MM_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8;
    // FP64 runs far fewer operations per second: fewer iterations keep the
    // probe short
    const int iters = sizeof(T) == 4 ? 1 << 14 : 1 << 10;
    const T a = (T)0.999999, b = (T)1e-7;
    fma_chains_kernel<T><<<blocks, 256>>>(out, 64, a, b);     // warm-up
    cudaEventRecord(e0);
    fma_chains_kernel<T><<<blocks, 256>>>(out, iters, a, b);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) return MM_ERR_CUDA;
    const double flops = 2.0 * kPeakChains * (double)iters * blocks * 256;
    *flops_per_s = flops / (ms * 1e-3);
    return MM_OK;
}

}  // namespace mm

extern "C" mm_status mm_measure_peak(int precision, double* flops_per_s) {
    if (!flops_per_s || (precision != 32 && precision != 64)) return MM_ERR_ARG;
    return precision == 32 ? mm::measure<float>(flops_per_s) : mm::measure<double>(flops_per_s);
}
