// Observables: energy per term and topological charge, each as an FP64
// Neumaier-compensated sum of per-cell products computed in the working
// precision (warp shuffles, then one block per partial set).
//
// Energy density per cell (the energy whose variational derivative is the
// effective field of Eq. 1): e = -1/2 mu0 Ms m.H_term for exchange, DMI,
// anisotropy and demag; e = -mu0 Ms m.H_ext for Zeeman; E = V sum e.
// Topological charge: q = (1/4pi) m.(dm/dx x dm/dy) dx dy with central
// differences, one-sided next to an edge or an absent cell.
#include <cuda_runtime.h>

#include "common.cuh"
#include "ctx.h"

namespace mm {

template <typename T>
__global__ void energy_partial_kernel(const T* __restrict__ m, const T* __restrict__ H, long long N,
                                      const uint8_t* __restrict__ region, const Region<T>* __restrict__ lut,
                                      double coef, double* __restrict__ partial) {
    CompSum acc{0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const Region<T>& R = lut[region ? region[i] : 0];
        if (R.present == (T)0) continue;
        const T mh = m[i] * H[i] + m[N + i] * H[N + i] + m[2 * N + i] * H[2 * N + i];
        acc.add(coef * (double)R.Ms * (double)mh);
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
        if (l == 0) { partial[2 * blockIdx.x] = v.s; partial[2 * blockIdx.x + 1] = v.c; }
    }
}

// sums `count` (s, c) pairs into out[0] (single block)
__global__ void finish_sum_kernel(const double* __restrict__ partial, int count, double* __restrict__ out) {
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
        if (l == 0) out[0] = v.s + v.c;
    }
}

// Sum over present cells (those of z-layer `layer` when layer >= 0) of
// component `comp` of m, or of 1 (the present-cell count) when comp < 0.
template <typename T>
__global__ void mean_partial_kernel(const T* __restrict__ m, long long N, long long plane, int layer, int comp,
                                    const uint8_t* __restrict__ region, const Region<T>* __restrict__ lut,
                                    double* __restrict__ partial) {
    const long long lo = layer >= 0 ? (long long)layer * plane : 0;
    const long long hi = layer >= 0 ? lo + plane : N;
    CompSum acc{0.0, 0.0};
    for (long long i = lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hi;
         i += (long long)gridDim.x * blockDim.x) {
        const Region<T>& R = lut[region ? region[i] : 0];
        if (R.present == (T)0) continue;
        acc.add(comp < 0 ? 1.0 : (double)m[comp * N + i]);
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
        if (l == 0) { partial[2 * blockIdx.x] = v.s; partial[2 * blockIdx.x + 1] = v.c; }
    }
}

template <typename T>
__device__ __forceinline__ v3<T> ldm(const T* m, long long N, long long i) {
    return mk3<T>(m[i], m[N + i], m[2 * N + i]);
}

template <typename T>
__global__ void topo_partial_kernel(const T* __restrict__ m, int nx, int ny, int nz, int layer, T hx, T hy,
                                    const uint8_t* __restrict__ region, const Region<T>* __restrict__ lut,
                                    double* __restrict__ partial) {
    const long long N = (long long)nx * ny * nz;
    const long long plane = (long long)nx * ny;
    const long long begin = layer >= 0 ? layer * plane : 0;
    const long long end = layer >= 0 ? begin + plane : N;
    CompSum acc{0.0, 0.0};
    auto present = [&](long long j) { return lut[region ? region[j] : 0].present != (T)0; };
    for (long long i = begin + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < end;
         i += (long long)gridDim.x * blockDim.x) {
        if (!present(i)) continue;
        const int x = (int)(i % nx), y = (int)((i / nx) % ny);
        const v3<T> mc = ldm(m, N, i);
        v3<T> d[2];
        for (int a = 0; a < 2; ++a) {
            const int pos = a == 0 ? x : y, n = a == 0 ? nx : ny;
            const long long st = a == 0 ? 1 : nx;
            const T h = a == 0 ? hx : hy;
            const bool hp = pos + 1 < n && present(i + st);
            const bool hm = pos - 1 >= 0 && present(i - st);
            if (hp && hm) d[a] = ((T)0.5 / h) * (ldm(m, N, i + st) - ldm(m, N, i - st));
            else if (hp) d[a] = ((T)1 / h) * (ldm(m, N, i + st) - mc);
            else if (hm) d[a] = ((T)1 / h) * (mc - ldm(m, N, i - st));
            else d[a] = mk3<T>(0, 0, 0);
        }
        const T q = dot(mc, cross(d[0], d[1]));
        acc.add((double)q * ((double)hx * (double)hy / (4.0 * kPi)));
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
        if (l == 0) { partial[2 * blockIdx.x] = v.s; partial[2 * blockIdx.x + 1] = v.c; }
    }
}

template <typename T>
__global__ void normalize_kernel(T* m, long long N, const uint8_t* __restrict__ region,
                                 const Region<T>* __restrict__ lut) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Region<T>& R = lut[region ? region[i] : 0];
    const T x = m[i], y = m[N + i], z = m[2 * N + i];
    const T n2 = x * x + y * y + z * z;
    const T inv = (R.present != (T)0 && n2 > (T)0) ? (T)1 / sqrt(n2) : (T)0;
    m[i] = x * inv;
    m[N + i] = y * inv;
    m[2 * N + i] = z * inv;
}

static const int kRedBlocks = 304;   // 2 x 152 SMs

void energy_term_launch(mm_ctx* c, const void* m, const void* H, int which, double* d_out) {
    const double V = c->grid.dx * c->grid.dy * c->grid.dz;
    const double coef = (which == MM_E_ZEEMAN ? -1.0 : -0.5) * kMu0 * V;
    const uint8_t* reg = c->uniform ? nullptr : (const uint8_t*)c->d_region;
    {
        LaunchScope ls(c, "energy_partial", 6.0 * c->esz * c->N);
        if (c->prec == 32)
            energy_partial_kernel<float><<<kRedBlocks, 256, 0, c->stream>>>(
                (const float*)m, (const float*)H, c->N, reg, (const Region<float>*)c->d_lut, coef, c->d_red);
        else
            energy_partial_kernel<double><<<kRedBlocks, 256, 0, c->stream>>>(
                (const double*)m, (const double*)H, c->N, reg, (const Region<double>*)c->d_lut, coef, c->d_red);
    }
    LaunchScope ls(c, "sum_finish", 0.0);
    finish_sum_kernel<<<1, 256, 0, c->stream>>>(c->d_red, kRedBlocks, d_out);
}

void topo_launch(mm_ctx* c, const void* m, int layer, double* d_out) {
    const uint8_t* reg = c->uniform ? nullptr : (const uint8_t*)c->d_region;
    const mm_grid& g = c->grid;
    {
        LaunchScope ls(c, "topo_partial", 3.0 * c->esz * c->N);
        if (c->prec == 32)
            topo_partial_kernel<float><<<kRedBlocks, 256, 0, c->stream>>>(
                (const float*)m, g.nx, g.ny, g.nz, layer, (float)g.dx, (float)g.dy, reg,
                (const Region<float>*)c->d_lut, c->d_red);
        else
            topo_partial_kernel<double><<<kRedBlocks, 256, 0, c->stream>>>(
                (const double*)m, g.nx, g.ny, g.nz, layer, g.dx, g.dy, reg, (const Region<double>*)c->d_lut,
                c->d_red);
    }
    LaunchScope ls(c, "sum_finish", 0.0);
    finish_sum_kernel<<<1, 256, 0, c->stream>>>(c->d_red, kRedBlocks, d_out);
}

// d_out[0..2] = sums of m_x, m_y, m_z over the present cells (of one layer
// when layer >= 0), d_out[3] = their count.
void mean_launch(mm_ctx* c, const void* m, int layer, double* d_out) {
    const uint8_t* reg = c->uniform ? nullptr : (const uint8_t*)c->d_region;
    const long long plane = (long long)c->grid.nx * c->grid.ny;
    for (int comp = 0; comp < 4; ++comp) {
        const int cc = comp < 3 ? comp : -1;
        {
            LaunchScope ls(c, "mean_partial", (comp < 3 ? 1.0 : 0.0) * c->esz * c->N);
            if (c->prec == 32)
                mean_partial_kernel<float><<<kRedBlocks, 256, 0, c->stream>>>(
                    (const float*)m, c->N, plane, layer, cc, reg, (const Region<float>*)c->d_lut, c->d_red);
            else
                mean_partial_kernel<double><<<kRedBlocks, 256, 0, c->stream>>>(
                    (const double*)m, c->N, plane, layer, cc, reg, (const Region<double>*)c->d_lut, c->d_red);
        }
        LaunchScope ls(c, "sum_finish", 0.0);
        finish_sum_kernel<<<1, 256, 0, c->stream>>>(c->d_red, kRedBlocks, d_out + comp);
    }
}

void normalize_launch(mm_ctx* c, void* m) {
    const uint8_t* reg = c->uniform ? nullptr : (const uint8_t*)c->d_region;
    const unsigned nb = (unsigned)((c->N + 255) / 256);
    LaunchScope ls(c, "normalize", 6.0 * c->esz * c->N);
    if (c->prec == 32)
        normalize_kernel<float><<<nb, 256, 0, c->stream>>>((float*)m, c->N, reg, (const Region<float>*)c->d_lut);
    else
        normalize_kernel<double><<<nb, 256, 0, c->stream>>>((double*)m, c->N, reg, (const Region<double>*)c->d_lut);
}

}  // namespace mm
