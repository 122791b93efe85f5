// Allocation-free topological charge for callers that cannot allocate
// device memory.  Examples: code that runs while a CUDA graph is being
// captured (a plain cudaMalloc is not allowed there), latency-critical
// loops that must never enter the allocator, and hosts whose device memory
// is owned by another framework's pool.  Such a caller passes its own
// input and output buffers; the only scratch, one FP64 partial sum pair per
// block, lives in a fixed file-scope device array that every GPU loading
// this library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "mm.h"

namespace mm {

// 4096 blocks x (sum, compensation) doubles = 64 KiB per device.
constexpr int kNoallocMaxBlocks = 4096;
constexpr int kNoallocCellsPerBlock = 4096;     // 256 threads x 16 cells
constexpr long long kNoallocMaxCells = (long long)kNoallocMaxBlocks * kNoallocCellsPerBlock;

static __device__ __align__(256) double g_noalloc_partials[2 * kNoallocMaxBlocks];

template <typename T>
__global__ void noalloc_topo_partial(const T* __restrict__ m, int nx, int ny, int nz, long long begin, long long end,
                                     T hx, T hy, double* __restrict__ partial) {
    const long long N = (long long)nx * ny * nz;
    CompSum acc{0.0, 0.0};
    const long long b0 = begin + (long long)blockIdx.x * kNoallocCellsPerBlock;
    const long long b1 = min(end, b0 + kNoallocCellsPerBlock);
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny);
        const v3<T> mc = mk3<T>(m[i], m[N + i], m[2 * N + i]);
        v3<T> d[2];
        for (int a = 0; a < 2; ++a) {
            const int pos = a == 0 ? x : y, n = a == 0 ? nx : ny;
            const long long st = a == 0 ? 1 : nx;
            const T h = a == 0 ? hx : hy;
            const bool hp = pos + 1 < n, hm = pos - 1 >= 0;
            const long long jp = i + st, jm = i - st;
            if (hp && hm)
                d[a] = ((T)0.5 / h) * (mk3<T>(m[jp], m[N + jp], m[2 * N + jp]) - mk3<T>(m[jm], m[N + jm], m[2 * N + jm]));
            else if (hp)
                d[a] = ((T)1 / h) * (mk3<T>(m[jp], m[N + jp], m[2 * N + jp]) - mc);
            else if (hm)
                d[a] = ((T)1 / h) * (mc - mk3<T>(m[jm], m[N + jm], m[2 * N + jm]));
            else
                d[a] = mk3<T>(0, 0, 0);
        }
        acc.add((double)dot(mc, cross(d[0], d[1])) * ((double)hx * (double)hy / (4.0 * kPi)));
    }
    acc = warp_sum(acc);
    __shared__ double s[64];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { s[2 * w] = acc.s; s[2 * w + 1] = acc.c; }
    __syncthreads();
    if (w == 0) {
        CompSum v{0.0, 0.0};
        if (l < (int)(blockDim.x >> 5)) { v.s = s[2 * l]; v.c = s[2 * l + 1]; }
        v = warp_sum(v);
        // every launched block overwrites its own pair: nothing to clear
        if (l == 0) { partial[2 * blockIdx.x] = v.s; partial[2 * blockIdx.x + 1] = v.c; }
    }
}

__global__ void noalloc_topo_finish(const double* __restrict__ partial, int count, double divisor,
                                    double* __restrict__ Q) {
    CompSum acc{0.0, 0.0};
    for (int q = threadIdx.x; q < count; q += blockDim.x) {
        acc.add(partial[2 * q]);
        acc.add(partial[2 * q + 1]);
    }
    acc = warp_sum(acc);
    __shared__ double s[64];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { s[2 * w] = acc.s; s[2 * w + 1] = acc.c; }
    __syncthreads();
    if (w == 0) {
        CompSum v{0.0, 0.0};
        if (l < (int)(blockDim.x >> 5)) { v.s = s[2 * l]; v.c = s[2 * l + 1]; }
        v = warp_sum(v);
        if (l == 0) Q[0] = (v.s + v.c) / divisor;
    }
}

// Device address of the partials array, looked up once per device with that
// device current (in host code the array's name is only a stand-in).
static double* partials_on_current_device(mm_status* st) {
    static std::mutex mu;
    static double* addr[128] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        *st = MM_ERR_DEVICE;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        double* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_noalloc_partials) != cudaSuccess || !p) {
            *st = MM_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = p;
    }
    *st = MM_OK;
    return addr[dev];
}

}  // namespace mm

extern "C" mm_status mm_topo_charge_noalloc(const void* m_dev, int precision, int nx, int ny, int nz, double dx,
                                            double dy, int layer, double* Q_dev, void* stream) {
    using namespace mm;
    if (!m_dev || !Q_dev || (precision != 32 && precision != 64) || nx <= 0 || ny <= 0 || nz <= 0 || !(dx > 0) ||
        !(dy > 0) || layer >= nz || layer < -1)
        return MM_ERR_ARG;
    const long long plane = (long long)nx * ny;
    const long long cells = layer >= 0 ? plane : plane * nz;
    if (cells > kNoallocMaxCells) return MM_ERR_ARG;   // more partial blocks than the fixed array holds
    // An error already pending on this thread belongs to earlier work: it is
    // left in place for its owner and nothing is launched (a failed launch of
    // this call could not be told apart from it).
    if (cudaPeekAtLastError() != cudaSuccess) return MM_ERR_STATE;
    mm_status st;
    double* partial = partials_on_current_device(&st);
    if (!partial) return st;
    const long long begin = layer >= 0 ? layer * plane : 0;
    const int blocks = (int)((cells + kNoallocCellsPerBlock - 1) / kNoallocCellsPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == 32)
        noalloc_topo_partial<float><<<blocks, 256, 0, s>>>((const float*)m_dev, nx, ny, nz, begin, begin + cells,
                                                           (float)dx, (float)dy, partial);
    else
        noalloc_topo_partial<double><<<blocks, 256, 0, s>>>((const double*)m_dev, nx, ny, nz, begin, begin + cells,
                                                            dx, dy, partial);
    noalloc_topo_finish<<<1, 256, 0, s>>>(partial, blocks, layer >= 0 ? 1.0 : (double)nz, Q_dev);
    return cudaGetLastError() == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}
