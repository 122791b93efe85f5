// Open-boundary demagnetisation (Methods, "Physics and discretization":
// FFT convolution with the Newell tensor, zero-padded to 2N).
//
// Pipeline per field evaluation, every pass a shared-memory batched FFT:
//   X pass   R2C along x of Ms*m (only the nx nonzero inputs of the padded
//            2nx row are read; half-length complex FFT + split)
//   Y pass   forward along y (3-D only; ny nonzero inputs, Py outputs)
//   middle   last axis (z in 3-D, y in 2-D): forward FFT, H^ = K^ M^ with the
//            real, symmetry-compressed tensor spectrum, inverse FFT, keep the
//            n un-padded outputs -- one pass, the spectrum never leaves smem
//   Y pass   inverse (3-D only; Py inputs, ny outputs)
//   X pass   C2R, only the nx un-padded outputs are written.
// Setup (once per geometry): the FP64 Newell tensor on the GPU (closed form
// near, tent-weighted Gauss-Legendre of the dipole kernel far), then FP64
// FFTs of the padded tensor; -1/(Px Py Pz) is folded into K^.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "fft_ct.cuh"
#include "fft_direct.cuh"
#include "fft_rt.cuh"

namespace mm {

template <typename T> __device__ __forceinline__ const T* stage_coef_dev(const DevState* st, int s);
template <> __device__ __forceinline__ const float* stage_coef_dev<float>(const DevState* st, int s) { return st->cf32[s]; }
template <> __device__ __forceinline__ const double* stage_coef_dev<double>(const DevState* st, int s) { return st->cf64[s]; }

// ---------------------------------------------------------------------------
// X passes: real rows <-> half spectra
// ---------------------------------------------------------------------------
template <typename T>
struct XArgs {
    const T* in;            // R2C: real rows (row r at in + r*in_pitch)
    T* out_real;            // C2R: real rows
    cplx<T>* spec;          // spectrum rows
    long long in_pitch;     // reals between consecutive input rows
    int rows;               // total rows
    int rows_per_plane;     // rows of one (component, z) plane on the real side
    int spec_rows_per_plane;// rows of one plane on the spectrum side
    int nx;                 // nonzero reals per row
    int Lh, Kx, Wk;         // half length, spectrum columns, spectrum pitch
    int rpc;                // rows per CTA
    Plan plan;
    const cplx<T>* tw;      // exp(-2 pi i q / Px), q < Px
    // Ms scaling of the input (R2C only): uniform Ms, or region LUT
    T ms_uniform;
    const uint8_t* region;
    const Region<T>* lut;
    long long cells_per_comp;  // N: row r belongs to component r / (N/nx)
    // fused RK stage (FP32 warp R2C, stage >= 1): the input rows are
    // m_s = m0 + sum_j (dt a_sj) k_j, formed here and also written to ms
    const DevState* st;
    T* const* kptr;
    const T* m0;
    T* ms;
    int stage;              // runtime stage for the CTA-wide R2C kernels (0: plain rows)
};

// m_s = m0 + sum_{j<S} (dt a_sj) k_j at element q (runtime stage S >= 1)
template <typename T>
__device__ __forceinline__ T stage_value(const XArgs<T>& a, int S, int kf, long long q) {
    const T* cf = stage_coef_dev<T>(a.st, S);
    T acc = a.m0[q];
    for (int j = 0; j < S; ++j) {
        if (j == 1 && S == 6) continue;             // a_7,2 = 0
        const int slot = j == 0 ? kf : j == 6 ? 6 - kf : j;
        acc += cf[j] * __ldg(a.kptr[slot] + q);
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ long long spec_row(const XArgs<T>& a, int r) {
    return (long long)(r / a.rows_per_plane) * a.spec_rows_per_plane + (r % a.rows_per_plane);
}

// LT > 0: compile-time half length (specialised FFT), LT == 0: runtime plan
template <typename T, int LT>
__global__ void __launch_bounds__(256) fft_x_r2c_kernel(XArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.stage > 0 && !a.st->active) return;
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int Lh = LT > 0 ? LT : a.Lh;
    const int pitch = Lh + 1;
    const int r0 = blockIdx.x * a.rpc;
    const int nl = min(a.rpc, a.rows - r0);
    const int kf = a.stage > 0 ? a.st->k_first : 0;
    // load real rows as packed complex z[n] = x[2n] + i x[2n+1]
    T* smr = reinterpret_cast<T*>(sm);
    const int nreal = 2 * Lh;
    for (int l = 0; l < nl; ++l) {
        const long long g0 = (long long)(r0 + l) * a.in_pitch;
        T ms = a.ms_uniform;
        for (int q = threadIdx.x; q < nreal; q += blockDim.x) {
            T v = 0;
            if (q < a.nx) {
                if (a.stage > 0) {
                    v = stage_value<T>(a, a.stage, kf, g0 + q);
                    a.ms[g0 + q] = v;
                } else {
                    v = a.in[g0 + q];
                }
                if (a.region) v *= a.lut[a.region[(g0 + q) % a.cells_per_comp]].Ms;
                else v *= ms;
            }
            smr[2 * (l * pitch) + q] = v;
        }
    }
    __syncthreads();
    const int nin = (a.nx + 1) / 2;
    if constexpr (LT > 0) ct_fft<T, 1, LT, LT + 1, 256, kMaxV>(sm, nl, nin, a.tw, 2);
    else fft_lines<T, 1>(sm, nl, pitch, a.plan, nin, a.tw, 2);
    // split: X[k] = (Z[k] + conj Z[M-k])/2 - i/2 W^k (Z[k] - conj Z[M-k])
    const int M = Lh, Kx = Lh + 1;
    for (int l = 0; l < nl; ++l) {
        cplx<T>* out = a.spec + spec_row(a, r0 + l) * a.Wk;
        for (int k = threadIdx.x; k < Kx; k += blockDim.x) {
            const cplx<T> zk = sm[l * pitch + (k == M ? 0 : k)];
            const cplx<T> zc = cconj<T>(sm[l * pitch + (k == 0 ? 0 : M - k)]);
            const cplx<T> E = cscale<T>(cadd<T>(zk, zc), (T)0.5);
            const cplx<T> O = cscale<T>(mul_mi<T, 1>(csub<T>(zk, zc)), (T)0.5);
            const cplx<T> w = __ldg(&a.tw[k]);
            out[k] = cadd<T>(E, cmul<T>(w, O));
        }
    }
}

template <typename T, int LT>
__global__ void __launch_bounds__(256) fft_x_c2r_kernel(XArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int Lh = LT > 0 ? LT : a.Lh;
    const int pitch = Lh + 1;
    const int r0 = blockIdx.x * a.rpc;
    const int nl = min(a.rpc, a.rows - r0);
    const int M = Lh, Kx = Lh + 1;
    for (int l = 0; l < nl; ++l) {
        const cplx<T>* in = a.spec + spec_row(a, r0 + l) * a.Wk;
        for (int k = threadIdx.x; k < Kx; k += blockDim.x) sm[l * pitch + k] = in[k];
    }
    __syncthreads();
    // rebuild Z'[k] = E' + i O', E' = X[k] + conj X[M-k],
    // O' = (X[k] - conj X[M-k]) conj(W^k); pairs (k, M-k) owned by one thread
    const int half = M / 2;
    for (int l = 0; l < nl; ++l) {
        for (int k = threadIdx.x; k <= half; k += blockDim.x) {
            const int k2 = M - k;
            const cplx<T> xk = sm[l * pitch + k];
            const cplx<T> xk2 = sm[l * pitch + k2];
            const cplx<T> w1 = __ldg(&a.tw[k]);
            const cplx<T> w2 = __ldg(&a.tw[k2]);
            const cplx<T> E1 = cadd<T>(xk, cconj<T>(xk2));
            const cplx<T> O1 = cmulc<T>(csub<T>(xk, cconj<T>(xk2)), w1);
            const cplx<T> E2 = cadd<T>(xk2, cconj<T>(xk));
            const cplx<T> O2 = cmulc<T>(csub<T>(xk2, cconj<T>(xk)), w2);
            sm[l * pitch + k] = cadd<T>(E1, mul_mi<T, -1>(O1));
            if (k2 != k && k2 < M) sm[l * pitch + k2] = cadd<T>(E2, mul_mi<T, -1>(O2));
        }
    }
    __syncthreads();
    if constexpr (LT > 0) ct_fft<T, -1, LT, LT + 1, 256, kMaxV>(sm, nl, M, a.tw, 2);
    else fft_lines<T, -1>(sm, nl, pitch, a.plan, M, a.tw, 2);
    const T* smr = reinterpret_cast<const T*>(sm);
    for (int l = 0; l < nl; ++l) {
        T* out = a.out_real + (long long)(r0 + l) * a.in_pitch;
        for (int q = threadIdx.x; q < a.nx; q += blockDim.x) out[q] = smr[2 * (l * pitch) + q];
    }
}

// FP32 X passes with the first (R2C) or first and last (C2R) Stockham pass
// working straight between global memory and registers.  Rows per CTA are a
// compile-time constant (the same rule the host uses for the generic path).
__host__ __device__ constexpr int x_rows_per_cta(int Lh) {
    return (kMaxV * 256 / Lh) < 1 ? 1 : (kMaxV * 256 / Lh) > 16 ? 16 : (kMaxV * 256 / Lh);
}

template <int LT>
__global__ void __launch_bounds__(256) fft_x_r2c_direct_kernel(XArgs<float> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.stage > 0 && !a.st->active) return;
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    constexpr int NT = 256, LP = LT + 1, RPC = x_rows_per_cta(LT);
    constexpr int R0 = ct_radix(LT, 0), NB0 = LT / R0;
    constexpr int MAXB = (RPC * NB0 + NT - 1) / NT;
    const int r0 = blockIdx.x * a.rpc;            // a.rpc <= RPC (fewer rows per CTA on small grids)
    const int nl = min(a.rpc, a.rows - r0);
    const int nin = (a.nx + 1) / 2;
    const int total = nl * NB0;
    const bool vec2 = (a.nx % 2 == 0) && (a.in_pitch % 2 == 0);
    // packed complex z[n] = Ms (x[2n] + i x[2n+1]), loaded into registers
    float2 v[MAXB][R0];
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < total) {
            const int l = b / NB0, j = b % NB0;
            const long long g0 = (long long)(r0 + l) * a.in_pitch;
#pragma unroll
            for (int t = 0; t < R0; ++t) {
                const int n = j + t * NB0;
                float2 z = make_float2(0.f, 0.f);
                if (n < nin) {
                    const long long q = g0 + 2 * n;
                    const bool has_y = 2 * n + 1 < a.nx;
                    if (a.stage > 0) {
                        // fused RK45 stage (nx even): form m_s, keep it, transform it
                        const int kf = a.st->k_first;
                        z.x = stage_value<float>(a, a.stage, kf, q);
                        z.y = stage_value<float>(a, a.stage, kf, q + 1);
                        *reinterpret_cast<float2*>(a.ms + q) = z;
                    } else if (vec2) {
                        z = *reinterpret_cast<const float2*>(a.in + q);
                    } else {
                        z.x = a.in[q];
                        z.y = has_y ? a.in[q + 1] : 0.f;
                    }
                    if (a.region) {
                        z.x *= a.lut[a.region[q % a.cells_per_comp]].Ms;
                        z.y = has_y ? z.y * a.lut[a.region[(q + 1) % a.cells_per_comp]].Ms : 0.f;
                    } else {
                        z.x *= a.ms_uniform;
                        z.y *= a.ms_uniform;
                    }
                }
                v[i][t] = z;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < total) {
            const int l = b / NB0, j = b % NB0;
            dft_ct<float, 1, R0>(v[i]);
#pragma unroll
            for (int t = 0; t < R0; ++t) sm[l * LP + j * R0 + t] = v[i][t];
        }
    }
    __syncthreads();
    ct_fft<float, 1, LT, LP, NT, kMaxV, 1>(sm, nl, LT, a.tw, 2);
    // split: X[k] = (Z[k] + conj Z[M-k])/2 - i/2 W^k (Z[k] - conj Z[M-k])
    constexpr int M = LT, Kx = LT + 1;
    for (int l = 0; l < nl; ++l) {
        float2* out = a.spec + spec_row(a, r0 + l) * a.Wk;
        for (int k = threadIdx.x; k < Kx; k += NT) {
            const float2 zk = sm[l * LP + (k == M ? 0 : k)];
            const float2 zc = cconj<float>(sm[l * LP + (k == 0 ? 0 : M - k)]);
            const float2 E = cscale<float>(cadd<float>(zk, zc), 0.5f);
            const float2 O = cscale<float>(mul_mi<float, 1>(csub<float>(zk, zc)), 0.5f);
            const float2 w = __ldg(&a.tw[k]);
            out[k] = cadd<float>(E, cmul<float>(w, O));
        }
    }
}

template <int LT>
__global__ void __launch_bounds__(256) fft_x_c2r_direct_kernel(XArgs<float> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    constexpr int NT = 256, LP = LT + 1, RPC = x_rows_per_cta(LT), M = LT, Kx = LT + 1;
    constexpr int NP = ct_npass(LT);
    static_assert(NP >= 2, "first and last pass must differ");
    const int r0 = blockIdx.x * a.rpc;            // a.rpc <= RPC (fewer rows per CTA on small grids)
    const int nl = min(a.rpc, a.rows - r0);
    for (int l = 0; l < nl; ++l) {
        const float2* in = a.spec + spec_row(a, r0 + l) * a.Wk;
        for (int k = threadIdx.x; k < Kx; k += NT) sm[l * LP + k] = in[k];
    }
    __syncthreads();
    // first pass, fed by the rebuild Z'[k] = (X[k] + conj X[M-k]) + i (X[k] - conj X[M-k]) conj(W^k)
    {
        constexpr int R0 = ct_radix(LT, 0), NB0 = LT / R0;
        constexpr int MAXB = (RPC * NB0 + NT - 1) / NT;
        const int total = nl * NB0;
        float2 v[MAXB][R0];
#pragma unroll
        for (int i = 0; i < MAXB; ++i) {
            const int b = threadIdx.x + i * NT;
            if (b < total) {
                const int l = b / NB0, j = b % NB0;
#pragma unroll
                for (int t = 0; t < R0; ++t) {
                    const int k = j + t * NB0;
                    const float2 xk = sm[l * LP + k];
                    const float2 xc = cconj<float>(sm[l * LP + M - k]);
                    const float2 w = __ldg(&a.tw[k]);
                    const float2 E = cadd<float>(xk, xc);
                    const float2 O = cmulc<float>(csub<float>(xk, xc), w);
                    v[i][t] = cadd<float>(E, mul_mi<float, -1>(O));
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < MAXB; ++i) {
            const int b = threadIdx.x + i * NT;
            if (b < total) {
                const int l = b / NB0, j = b % NB0;
                dft_ct<float, -1, R0>(v[i]);
#pragma unroll
                for (int t = 0; t < R0; ++t) sm[l * LP + j * R0 + t] = v[i][t];
            }
        }
        __syncthreads();
    }
    ct_fft<float, -1, LT, LP, NT, kMaxV, 1, NP - 1>(sm, nl, LT, a.tw, 2);
    // last pass straight to the real rows: z[n] -> (x[2n], x[2n+1])
    {
        constexpr int P = NP - 1, R = ct_radix(LT, P), NS = ct_ns(LT, P), NB = LT / R;
        static_assert(NB == NS, "last pass writes natural order");
        constexpr int MAXB = (RPC * NB + NT - 1) / NT;
        const int total = nl * NB;
        const bool vec2 = (a.nx % 2 == 0) && (a.in_pitch % 2 == 0);
#pragma unroll
        for (int i = 0; i < MAXB; ++i) {
            const int b = threadIdx.x + i * NT;
            if (b < total) {
                const int l = b / NB, j = b % NB;
                float2 v[R];
#pragma unroll
                for (int t = 0; t < R; ++t) v[t] = sm[l * LP + j + t * NB];
#pragma unroll
                for (int t = 1; t < R; ++t) v[t] = cmulc<float>(v[t], __ldg(&a.tw[(t * j) * 2]));
                dft_ct<float, -1, R>(v);
                float* out = a.out_real + (long long)(r0 + l) * a.in_pitch;
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    const int n = j + t * NS;
                    if (2 * n + 1 < a.nx) {
                        if (vec2) *reinterpret_cast<float2*>(out + 2 * n) = v[t];
                        else { out[2 * n] = v[t].x; out[2 * n + 1] = v[t].y; }
                    } else if (2 * n < a.nx) {
                        out[2 * n] = v[t].x;
                    }
                }
            }
        }
    }
}

// FP32 X passes for rows of half length 64 ... 512: one row per warp, eight
// warps per CTA, no CTA-wide barrier.  R2C: packed pairs straight from global memory
// into the first pass, later passes in warp-private shared memory, then the
// split to the Lh+1 spectrum.  C2R: the rebuild of Z' from X[k] and
// X[M-k] (both read from global memory) feeds the first pass; the last pass
// writes the real row.
constexpr int kXW = 8;   // warps (rows) per CTA

// Slot of stage j's slope under the first-same-as-last rotation (slots 0
// and 6 swap roles between steps).
__device__ __forceinline__ int stage_slot(int j, int k_first) {
    return j == 0 ? k_first : j == 6 ? 6 - k_first : j;
}

// m_s = m0 + sum_{j<S} (dt a_sj) k_j at the float2 pair starting at q
template <int S>
__device__ __forceinline__ float2 stage_pair(const XArgs<float>& a, const float* cf, int kf, long long q) {
    float2 acc = __ldg(reinterpret_cast<const float2*>(a.m0 + q));
#pragma unroll
    for (int j = 0; j < S; ++j) {
        if (j == 1 && S == 6) continue;             // a_7,2 = 0
        const float2 k = __ldg(reinterpret_cast<const float2*>(a.kptr[stage_slot(j, kf)] + q));
        acc.x += cf[j] * k.x;
        acc.y += cf[j] * k.y;
    }
    return acc;
}

// S = 0: rows of a.in.  S >= 1 (RK45 stage S, nx even): rows of the stage
// state formed from m0 and the slopes, which is also stored to a.ms; the
// whole launch is a no-op when the attempt is inactive.
// (at most 64 registers: four CTAs of 8 warps per SM; 512x512x64 stage
// transform 412 -> 385 us against the unconstrained 80)
template <int LT, int S>
__global__ void __launch_bounds__(32 * kXW, 4) fft_x_r2c_warp_kernel(XArgs<float> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (S > 0 && !a.st->active) return;
    // a group of GW lanes per row (a warp takes 32 / GW rows of a short line)
    constexpr int GW = warp_group(LT), RPW = 32 / GW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & (GW - 1);
    const int wrow = (blockIdx.x * kXW + warp) * RPW;
    if (wrow >= a.rows) return;                 // whole warp: no CTA barrier below
    const int slot = warp * RPW + (threadIdx.x & 31) / GW;
    const bool rvalid = wrow + (threadIdx.x & 31) / GW < a.rows;
    const int row = rvalid ? wrow + (threadIdx.x & 31) / GW : wrow;   // a spare group repeats the first row
    float2* sm = reinterpret_cast<float2*>(smem_raw) + slot * wline(LT);
    constexpr int NP = ct_npass(LT);
    const int nin = (a.nx + 1) / 2;
    const long long g0 = (long long)row * a.in_pitch;
    const bool vec2 = (a.nx % 2 == 0) && (a.in_pitch % 2 == 0);
    const float* cf = S > 0 ? a.st->cf32[S] : nullptr;
    const int kf = S > 0 ? a.st->k_first : 0;
    auto load_in = [&](int n) {
        float2 z = make_float2(0.f, 0.f);
        if (n < nin) {
            const long long q = g0 + 2 * n;
            const bool has_y = 2 * n + 1 < a.nx;
            if constexpr (S > 0) {
                z = stage_pair<S>(a, cf, kf, q);
                if (rvalid) *reinterpret_cast<float2*>(a.ms + q) = z;
            } else if (vec2) {
                z = *reinterpret_cast<const float2*>(a.in + q);
            } else {
                z.x = a.in[q];
                z.y = has_y ? a.in[q + 1] : 0.f;
            }
            if (a.region) {
                z.x *= a.lut[a.region[q % a.cells_per_comp]].Ms;
                z.y = has_y ? z.y * a.lut[a.region[(q + 1) % a.cells_per_comp]].Ms : 0.f;
            } else {
                z.x *= a.ms_uniform;
                z.y *= a.ms_uniform;
            }
        }
        return z;
    };
    warp_pass<float, 1, LT, ct_radix(LT, 0), 1, GW>(a.tw, 2, load_in, [&](int i, float2 v) { sm[wpad(i)] = v; });
    warp_fft_smem<float, 1, LT, 1, NP, GW>(sm, a.tw, 2);
    constexpr int M = LT, Kx = LT + 1;
    float2* out = a.spec + spec_row(a, row) * a.Wk;
    for (int k = lane; k < Kx; k += GW) {
        const float2 zk = sm[wpad(k == M ? 0 : k)];
        const float2 zc = cconj<float>(sm[wpad(k == 0 ? 0 : M - k)]);
        const float2 E = cscale<float>(cadd<float>(zk, zc), 0.5f);
        const float2 O = cscale<float>(mul_mi<float, 1>(csub<float>(zk, zc)), 0.5f);
        if (rvalid) out[k] = cadd<float>(E, cmul<float>(__ldg(&a.tw[k]), O));
    }
}

template <int LT>
__global__ void __launch_bounds__(32 * kXW) fft_x_c2r_warp_kernel(XArgs<float> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int GW = warp_group(LT), RPW = 32 / GW;
    const int warp = threadIdx.x >> 5;
    const int wrow = (blockIdx.x * kXW + warp) * RPW;
    if (wrow >= a.rows) return;                 // whole warp
    const int slot = warp * RPW + (threadIdx.x & 31) / GW;
    const bool rvalid = wrow + (threadIdx.x & 31) / GW < a.rows;
    const int row = rvalid ? wrow + (threadIdx.x & 31) / GW : wrow;   // a spare group repeats the first row
    float2* sm = reinterpret_cast<float2*>(smem_raw) + slot * wline(LT);
    float* out = a.out_real + (long long)row * a.in_pitch;
    const bool vec2 = (a.nx % 2 == 0) && (a.in_pitch % 2 == 0);
    const int nx = a.nx;
    warp_c2r<LT, GW>(a.spec + spec_row(a, row) * a.Wk, a.tw, sm, [&](int n, float2 v) {
        if (!rvalid) return;
        if (2 * n + 1 < nx) {
            if (vec2) *reinterpret_cast<float2*>(out + 2 * n) = v;
            else { out[2 * n] = v.x; out[2 * n + 1] = v.y; }
        } else if (2 * n < nx) {
            out[2 * n] = v.x;
        }
    });
}

// C2R with the spectrum rows prefetched: persistent warps, each with two
// line buffers in shared memory.  While a warp transforms one row (in place
// in one buffer), cp.async brings its next row into the other, so the
// global-memory latency of a row hides behind the transform of the previous
// one instead of stalling the first pass.
__device__ __forceinline__ void cpa16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// float2 per line buffer: the padded line, rounded to 16 bytes
template <int LT> constexpr int xpipe_buf() { return (wline(LT) + 1) & ~1; }
template <int LT> constexpr size_t xpipe_smem() { return (size_t)kXW * 2 * xpipe_buf<LT>() * sizeof(float2); }

template <int LT>
__global__ void __launch_bounds__(32 * kXW, 3) fft_x_c2r_pipe_kernel(XArgs<float> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int BS = xpipe_buf<LT>();
    static_assert(LT % 2 == 0, "16-byte pieces of the half spectrum");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* buf = reinterpret_cast<float2*>(smem_raw) + warp * 2 * BS;
    const int nw = gridDim.x * kXW;
    float* const out0 = a.out_real;
    const bool vec2 = (a.nx % 2 == 0) && (a.in_pitch % 2 == 0);
    const int nx = a.nx;
    // row r's LT + 1 spectrum values (16-byte aligned: the pitch Wk is even)
    auto fetch = [&](int r, float2* dst) {
        const float2* src = a.spec + spec_row(a, r) * a.Wk;
        for (int q = lane; q < LT / 2; q += 32) cpa16(dst + 2 * q, src + 2 * q);
        if (lane == 0) cpa8(dst + LT, src + LT);
        cpa_commit();
    };
    int row = blockIdx.x * kXW + warp;
    if (row < a.rows) fetch(row, buf);
    for (int it = 0; row < a.rows; ++it, row += nw) {
        float2* cur = buf + (it & 1) * BS;
        if (row + nw < a.rows) {
            fetch(row + nw, buf + ((it + 1) & 1) * BS);
            cpa_wait<1>();
        } else {
            cpa_wait<0>();
        }
        __syncwarp();
        float* out = out0 + (long long)row * a.in_pitch;
        warp_c2r_inplace<LT>(cur, a.tw, [&](int n, float2 v) {
            if (2 * n + 1 < nx) {
                if (vec2) *reinterpret_cast<float2*>(out + 2 * n) = v;
                else { out[2 * n] = v.x; out[2 * n + 1] = v.y; }
            } else if (2 * n < nx) {
                out[2 * n] = v.x;
            }
        });
    }
}

// ---------------------------------------------------------------------------
// Column passes (strided axes), optionally with the tensor multiply
// ---------------------------------------------------------------------------
template <typename T>
struct ColArgs {
    cplx<T>* base;
    long long comp_stride;   // between the three components
    long long line_stride;   // between consecutive points of the axis
    long long other_stride;  // between consecutive values of blockIdx.y
    int nc;                  // components per CTA (1 or 3)
    int Kx, TK;
    int L, n_in, n_out;
    Plan plan;
    const cplx<T>* tw;       // exp(-2 pi i q / L)
    // tensor multiply (middle pass only)
    const T* khat;
    long long kc_stride;     // elements per tensor component
    long long kk_stride;     // tensor stride for the transform-axis frequency
    long long ko_stride;     // tensor stride for the other-axis frequency
    int ncomp;               // 6 or 4
    int L_other;             // padded length of the other axis (Py in 3-D), 1 in 2-D
    int axis_is_y;           // 1: transform axis is y (2-D), 0: z (3-D)
};

template <typename T>
__device__ __forceinline__ void tensor_multiply(const ColArgs<T>& a, cplx<T>* sm, int pitch, int kx0, int L, int tks) {
    const int other = blockIdx.y;
    // fold the other-axis frequency (3-D: ky) to the stored half range
    int ko = 0, so = 1;
    if (!a.axis_is_y) {
        ko = other <= a.L_other / 2 ? other : a.L_other - other;
        so = other <= a.L_other / 2 ? 1 : -1;
    }
    for (int e = threadIdx.x; e < (L << tks); e += blockDim.x) {
        const int kxl = e & (a.TK - 1), kk = e >> tks;
        const int kx = kx0 + kxl;
        if (kx >= a.Kx) continue;
        const int kkf = kk <= L / 2 ? kk : L - kk;
        const int sk = kk <= L / 2 ? 1 : -1;
        const T* K = a.khat + (long long)kkf * a.kk_stride + (long long)ko * a.ko_stride + kx;
        const T kxx = __ldg(K), kyy = __ldg(K + a.kc_stride), kzz = __ldg(K + 2 * a.kc_stride);
        T kxy = __ldg(K + 3 * a.kc_stride);
        T kxz = 0, kyz = 0;
        // parity: xy odd in y, xz odd in z, yz odd in y and z
        const int sy = a.axis_is_y ? sk : so;
        const int sz = a.axis_is_y ? 1 : sk;
        kxy *= (T)sy;
        if (a.ncomp == 6) {
            kxz = __ldg(K + 4 * a.kc_stride) * (T)sz;
            kyz = __ldg(K + 5 * a.kc_stride) * (T)(sy * sz);
        }
        cplx<T>* px = &sm[(0 * a.TK + kxl) * pitch + kk];
        cplx<T>* py = &sm[(1 * a.TK + kxl) * pitch + kk];
        cplx<T>* pz = &sm[(2 * a.TK + kxl) * pitch + kk];
        const cplx<T> mx = *px, my = *py, mz = *pz;
        *px = mkc<T>(kxx * mx.x + kxy * my.x + kxz * mz.x, kxx * mx.y + kxy * my.y + kxz * mz.y);
        *py = mkc<T>(kxy * mx.x + kyy * my.x + kyz * mz.x, kxy * mx.y + kyy * my.y + kyz * mz.y);
        *pz = mkc<T>(kxz * mx.x + kyz * my.x + kzz * mz.x, kxz * mx.y + kyz * my.y + kzz * mz.y);
    }
    __syncthreads();
}

template <typename T, int MODE, int LT>  // MODE: +1 forward, -1 inverse, 0 convolution
__global__ void __launch_bounds__(512) fft_col_kernel(ColArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int L = LT > 0 ? LT : a.L;
    const int pitch = L + 1;
    const int kx0 = blockIdx.x * a.TK;
    const long long obase = (long long)blockIdx.y * a.other_stride;
    const int nl = a.nc * a.TK;
    const int tks = __ffs(a.TK) - 1;            // TK is a power of two
    const int tkm = a.TK - 1;
    // load: consecutive threads take consecutive kx (coalesced rows of TK)
    for (int c = 0; c < a.nc; ++c) {
        const cplx<T>* src = a.base + c * a.comp_stride + obase + kx0;
        for (int e = threadIdx.x; e < (a.n_in << tks); e += blockDim.x) {
            const int kxl = e & tkm, pt = e >> tks;
            cplx<T> v = mkc<T>(0, 0);
            if (kx0 + kxl < a.Kx) v = src[pt * a.line_stride + kxl];
            sm[((c << tks) + kxl) * pitch + pt] = v;
        }
    }
    __syncthreads();
    constexpr int NT = LT >= 512 ? 512 : 256;
    if constexpr (LT > 0) {
        if (MODE >= 0) ct_fft<T, 1, LT, LT + 1, NT, kMaxV>(sm, nl, a.n_in, a.tw, 1);
        else ct_fft<T, -1, LT, LT + 1, NT, kMaxV>(sm, nl, a.n_in, a.tw, 1);
    } else {
        if (MODE >= 0) fft_lines<T, 1>(sm, nl, pitch, a.plan, a.n_in, a.tw, 1);
        else fft_lines<T, -1>(sm, nl, pitch, a.plan, a.n_in, a.tw, 1);
    }
    if (MODE == 0) {
        tensor_multiply<T>(a, sm, pitch, kx0, L, tks);
        if constexpr (LT > 0) ct_fft<T, -1, LT, LT + 1, NT, kMaxV>(sm, nl, LT, a.tw, 1);
        else fft_lines<T, -1>(sm, nl, pitch, a.plan, L, a.tw, 1);
    }
    for (int c = 0; c < a.nc; ++c) {
        cplx<T>* dst = a.base + c * a.comp_stride + obase + kx0;
        for (int e = threadIdx.x; e < (a.n_out << tks); e += blockDim.x) {
            const int kxl = e & tkm, pt = e >> tks;
            if (kx0 + kxl < a.Kx) dst[pt * a.line_stride + kxl] = sm[((c << tks) + kxl) * pitch + pt];
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 3-D fast paths
// ---------------------------------------------------------------------------
// Y passes: TK = 16 columns per CTA taken from the flattened (component, z,
// kx) column list, so no CTA is left with a ragged handful of columns; the
// first Stockham pass reads global memory straight into registers and the
// last one writes its outputs straight back (128-byte row segments).
template <typename T>
struct YArgs {
    cplx<T>* base;        // spectrum [3][nz][Py][Wk]
    long long plane;      // Py * Wk: between consecutive (component, z) planes
    int Kx, Wk;
    int ncols;            // 3 * nz * Kx
    int n_in, n_out;
    const cplx<T>* tw;    // exp(-2 pi i q / Py)
};

// Columns per CTA and threads: 16 columns, except at L >= 1024 where 8
// columns of 256 threads (64 KB of shared memory) let three CTAs share an SM.
__host__ __device__ constexpr int y_direct_tk(int L) { return L >= 1024 ? 8 : 16; }
__host__ __device__ constexpr int y_direct_threads(int L) { return L >= 1024 ? 256 : L >= 512 ? 512 : 256; }

template <typename T, int DIR, int L>
__global__ void __launch_bounds__(y_direct_threads(L)) fft_y_direct_kernel(YArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    constexpr int TK = y_direct_tk(L);
    const int col = blockIdx.x * TK + (int)(threadIdx.x % TK);
    long long gcol = -1;
    if (col < a.ncols) {
        const int q = col / a.Kx, kx = col - q * a.Kx;
        gcol = (long long)q * a.plane + kx;
    }
    cd_fft<T, DIR, L, y_direct_threads(L), TK>(sm, a.base, a.base, gcol, a.Wk, a.n_in, a.n_out, a.tw);
}

// Middle (z) pass for Pz a power of two <= 32: one thread per (component,
// column) keeps its whole z line in registers.  Forward by decimation in
// frequency (bit-reversed spectrum), the three components exchanged once
// through shared memory for H^ = K^ M^ (row c of the symmetric tensor), then
// the inverse by decimation in time straight back to natural order; only the
// nz un-padded outputs are stored.  Columns are the flattened (ky, kx)
// positions of a z-plane, kZT per CTA, so loads are contiguous 256-byte runs.
template <typename T>
struct ZArgs {
    cplx<T>* base;          // spectrum [3][nz][Py][Wk]
    long long comp_stride;  // nz * Py * Wk
    long long plane;        // Py * Wk: between consecutive z
    int nz, Py, Kx, Wk;
    const cplx<T>* tw;      // exp(-2 pi i q / Pz)
    const T* khat;          // [6][Pz/2+1][Py/2+1][Wk]
    long long kc_stride;    // per tensor component
    long long kk_stride;    // per kz: (Py/2+1) * Wk
};

constexpr int kZT = 32;

// v[i] (bit-reversed kz = bitrev(i)) = sum_j K_cj(kx, ky, kz) M_j, the three
// spectra M_j read from shared memory.  Tensor components xx yy zz xy xz yz
// = 0..5 stored for ky, kz <= P/2; xy is odd in ky, xz odd in kz, yz odd in
// both, so row C needs the signs (1, sy, sz), (sy, 1, sy sz), (sz, sy sz, 1).
template <typename T, int L, int C, bool YF>
__device__ __forceinline__ void zconv_multiply(cplx<T> (&v)[L], const cplx<T>* sm, int tx, const T* K,
                                               long long kcs, long long kks) {
    constexpr int LOG = ilog2_c(L);
    constexpr int j0 = C == 0 ? 0 : C == 1 ? 3 : 4;
    constexpr int j1 = C == 0 ? 3 : C == 1 ? 1 : 5;
    constexpr int j2 = C == 0 ? 4 : C == 1 ? 5 : 2;
    constexpr T sy = YF ? (T)-1 : (T)1;
    const T* K0 = K + j0 * kcs;
    const T* K1 = K + j1 * kcs;
    const T* K2 = K + j2 * kcs;
    // kz and L - kz share the stored entries kzf (signs flip with sz): each
    // tensor value is loaded once and used for both
#pragma unroll
    for (int kzf = 0; kzf <= L / 2; ++kzf) {
        const T a0 = __ldg(K0 + kzf * kks);
        const T a1 = __ldg(K1 + kzf * kks);
        const T a2 = __ldg(K2 + kzf * kks);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && (kzf == 0 || kzf == L / 2)) continue;
            const int kz = h == 0 ? kzf : L - kzf;
            const int i = bitrev_c(kz, LOG);             // register slot of kz (bit-reversed order)
            const T sz = h == 0 ? (T)1 : (T)-1;
            const T s0 = C == 0 ? (T)1 : C == 1 ? sy : sz;
            const T s1 = C == 0 ? sy : C == 1 ? (T)1 : sy * sz;
            const T s2 = C == 0 ? sz : C == 1 ? sy * sz : (T)1;
            const T k0 = s0 * a0, k1 = s1 * a1, k2 = s2 * a2;
            const cplx<T> m0 = sm[(0 * L + i) * kZT + tx];
            const cplx<T> m1 = sm[(1 * L + i) * kZT + tx];
            const cplx<T> m2 = sm[(2 * L + i) * kZT + tx];
            v[i] = mkc<T>(k0 * m0.x + k1 * m1.x + k2 * m2.x, k0 * m0.y + k1 * m1.y + k2 * m2.y);
        }
    }
}

template <typename T, int L, bool HALF>
__global__ void __launch_bounds__(3 * kZT, HALF ? 5 : 4) fft_zconv_reg_kernel(ZArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw) + L;  // [3][L][kZT]
    const cplx<T>* tws = nullptr;                            // twiddles from c_tw32
    const int tx = threadIdx.x % kZT, c = threadIdx.x / kZT;
    const long long p = (long long)blockIdx.x * kZT + tx;
    const int ky = (int)(p / a.Wk), kx = (int)(p - (long long)ky * a.Wk);
    const bool valid = ky < a.Py && kx < a.Kx;
    cplx<T>* col = a.base + c * a.comp_stride + (valid ? p : 0);
    cplx<T> v[L];
#pragma unroll
    for (int z = 0; z < L; ++z) v[z] = (valid && z < a.nz && (!HALF || z < L / 2)) ? col[z * a.plane] : mkc<T>(0, 0);
    reg_dif<T, L, HALF>(v, tws);
#pragma unroll
    for (int i = 0; i < L; ++i) sm[(c * L + i) * kZT + tx] = v[i];
    __syncthreads();
    // row c of the tensor times the three spectra; c is uniform over a warp
    // (kZT is a multiple of 32) and the ky fold nearly so, which makes every
    // parity sign a compile-time constant
    const bool yfold = ky > a.Py / 2;
    const int kyf = yfold ? a.Py - ky : ky;
    const T* K = a.khat + (valid ? (long long)kyf * a.Wk + kx : 0);
    if (c == 0) {
        if (yfold) zconv_multiply<T, L, 0, true>(v, sm, tx, K, a.kc_stride, a.kk_stride);
        else zconv_multiply<T, L, 0, false>(v, sm, tx, K, a.kc_stride, a.kk_stride);
    } else if (c == 1) {
        if (yfold) zconv_multiply<T, L, 1, true>(v, sm, tx, K, a.kc_stride, a.kk_stride);
        else zconv_multiply<T, L, 1, false>(v, sm, tx, K, a.kc_stride, a.kk_stride);
    } else {
        if (yfold) zconv_multiply<T, L, 2, true>(v, sm, tx, K, a.kc_stride, a.kk_stride);
        else zconv_multiply<T, L, 2, false>(v, sm, tx, K, a.kc_stride, a.kk_stride);
    }
    reg_dit_inv<T, L, HALF>(v, tws);
    if (valid) {
#pragma unroll
        for (int z = 0; z < (HALF ? L / 2 : L); ++z)
            if (z < a.nz) col[z * a.plane] = v[z];
    }
}

// ---------------------------------------------------------------------------
// FP64 Newell tensor
// ---------------------------------------------------------------------------
struct GLTable {
    // nodes/weights on [-1,1] for the orders used: 16, 12, 6, 4, 3
    double x[41], w[41];
    int off[5], n[5];
};

__device__ double newell_f_dev(double x, double y, double z) {
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z, R = sqrt(xx + yy + zz);
    double r = (2.0 * xx - yy - zz) * R * (1.0 / 6.0);
    if (y > 0.0 && xx + zz > 0.0) r += 0.5 * y * (zz - xx) * asinh(y / sqrt(xx + zz));
    if (z > 0.0 && xx + yy > 0.0) r += 0.5 * z * (yy - xx) * asinh(z / sqrt(xx + yy));
    if (x > 0.0 && y > 0.0 && z > 0.0) r -= x * y * z * atan(y * z / (x * R));
    return r;
}

__device__ double newell_g_dev(double x, double y, double z) {
    double sg = 1.0;
    if (x < 0.0) { sg = -sg; x = -x; }
    if (y < 0.0) { sg = -sg; y = -y; }
    z = fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z, R = sqrt(xx + yy + zz);
    double r = -x * y * R * (1.0 / 3.0);
    if (z > 0.0 && xx + yy > 0.0) r += x * y * z * asinh(z / sqrt(xx + yy));
    if (x > 0.0 && yy + zz > 0.0) r += y * (3.0 * zz - yy) * asinh(x / sqrt(yy + zz)) * (1.0 / 6.0);
    if (y > 0.0 && xx + zz > 0.0) r += x * (3.0 * zz - xx) * asinh(y / sqrt(xx + zz)) * (1.0 / 6.0);
    if (x > 0.0 && y > 0.0 && z > 0.0) {
        r -= zz * z * atan(x * y / (z * R)) * (1.0 / 6.0);
        r -= 0.5 * z * yy * atan(x * z / (y * R));
        r -= 0.5 * z * xx * atan(y * z / (x * R));
    }
    return sg * r;
}

// N at displacement (X,Y,Z) for cell (hx,hy,hz), all lengths already divided
// by the largest cell edge.  out: xx yy zz xy xz yz.
__device__ void newell_eval(double X, double Y, double Z, double hx, double hy, double hz,
                            const GLTable& gl, double* out) {
    const double d = sqrt(X * X + Y * Y + Z * Z);
    if (d <= 2.0) {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int i = -1; i <= 1; ++i)
            for (int j = -1; j <= 1; ++j)
                for (int k = -1; k <= 1; ++k) {
                    const double w = (i ? -1.0 : 2.0) * (j ? -1.0 : 2.0) * (k ? -1.0 : 2.0);
                    const double x = X + i * hx, y = Y + j * hy, z = Z + k * hz;
                    s[0] += w * newell_f_dev(x, y, z);
                    s[1] += w * newell_f_dev(y, x, z);
                    s[2] += w * newell_f_dev(z, y, x);
                    s[3] += w * newell_g_dev(x, y, z);
                    s[4] += w * newell_g_dev(x, z, y);
                    s[5] += w * newell_g_dev(y, z, x);
                }
        const double c = 1.0 / (4.0 * kPi * hx * hy * hz);
        for (int a = 0; a < 6; ++a) out[a] = c * s[a];
        return;
    }
    const int band = d <= 3.0 ? 0 : d <= 8.0 ? 1 : d <= 32.0 ? 2 : d <= 128.0 ? 3 : 4;
    const int n = gl.n[band], o = gl.off[band];
    // tent per axis: nodes t = +-h (1 + xi)/2, weights w h^2 (1 - xi)/4
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 2 * n; ++i) {
        const double xi = gl.x[o + (i >> 1)];
        const double tx = ((i & 1) ? -0.5 : 0.5) * hx * (1.0 + xi);
        const double wx = gl.w[o + (i >> 1)] * 0.25 * hx * hx * (1.0 - xi);
        const double rx = X + tx;
        for (int j = 0; j < 2 * n; ++j) {
            const double yj = gl.x[o + (j >> 1)];
            const double ty = ((j & 1) ? -0.5 : 0.5) * hy * (1.0 + yj);
            const double wy = wx * gl.w[o + (j >> 1)] * 0.25 * hy * hy * (1.0 - yj);
            const double ry = Y + ty;
            for (int k = 0; k < 2 * n; ++k) {
                const double zk = gl.x[o + (k >> 1)];
                const double tz = ((k & 1) ? -0.5 : 0.5) * hz * (1.0 + zk);
                const double w = wy * gl.w[o + (k >> 1)] * 0.25 * hz * hz * (1.0 - zk);
                const double rz = Z + tz;
                const double r2 = rx * rx + ry * ry + rz * rz;
                const double ir2 = 1.0 / r2;
                const double ir3 = ir2 * rsqrt(r2);
                const double w5 = 3.0 * w * ir3 * ir2;
                acc[0] += w5 * rx * rx - w * ir3;
                acc[1] += w5 * ry * ry - w * ir3;
                acc[2] += w5 * rz * rz - w * ir3;
                acc[3] += w5 * rx * ry;
                acc[4] += w5 * rx * rz;
                acc[5] += w5 * ry * rz;
            }
        }
    }
    const double c = -1.0 / (4.0 * kPi * hx * hy * hz);
    for (int a = 0; a < 6; ++a) out[a] = c * acc[a];
}

__global__ void newell_list_kernel(long count, const int* __restrict__ ijk, double hx, double hy,
                                   double hz, GLTable gl, double* __restrict__ out) {
    const long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (q >= count) return;
    const double s = fmax(hx, fmax(hy, hz));
    double v[6];
    newell_eval(ijk[3 * q] * hx / s, ijk[3 * q + 1] * hy / s, ijk[3 * q + 2] * hz / s, hx / s, hy / s,
                hz / s, gl, v);
    for (int a = 0; a < 6; ++a) out[6 * q + a] = v[a];
}

// Tensor on the octant displacements 0 <= i < nx, ... ; with periodic
// images (Methods: periodic-boundary demagnetisation by an image-sum
// kernel) the sum over a in [-Rx, Rx], b in [-Ry, Ry], c in [-Rz, Rz] of
// N(i + a nx, j + b ny, k + c nz): the field of the sample and its shifted
// copies, seen from the central copy.
__global__ void newell_octant_kernel(int nx, int ny, int nz, double hx, double hy, double hz, GLTable gl,
                                     int Rx, int Ry, int Rz, double* __restrict__ out) {
    const long long n = (long long)nx * ny * nz;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long long)nx * ny));
    const double s = fmax(hx, fmax(hy, hz));
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int a = -Rx; a <= Rx; ++a)
        for (int b = -Ry; b <= Ry; ++b)
            for (int c = -Rz; c <= Rz; ++c) {
                double w[6];
                newell_eval((double)(i + (long long)a * nx) * hx / s, (double)(j + (long long)b * ny) * hy / s,
                            (double)(k + (long long)c * nz) * hz / s, hx / s, hy / s, hz / s, gl, w);
                for (int e = 0; e < 6; ++e) v[e] += w[e];
            }
    for (int e = 0; e < 6; ++e) out[e * n + q] = v[e];
}

// padded real array of one component from the octant (parity per component)
__global__ void padded_component_kernel(const double* __restrict__ oct, int comp, int nx, int ny, int nz,
                                        int Px, int Py, int Pz, double* __restrict__ dst) {
    const long long P = (long long)Px * Py * Pz;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= P) return;
    const int X = (int)(q % Px), Y = (int)((q / Px) % Py), Z = (int)(q / ((long long)Px * Py));
    const int i = X <= Px / 2 ? X : X - Px;
    const int j = Y <= Py / 2 ? Y : Y - Py;
    const int k = Z <= Pz / 2 ? Z : Z - Pz;
    double v = 0.0;
    if (abs(i) < nx && abs(j) < ny && abs(k) < nz) {
        const long long n = (long long)nx * ny * nz;
        v = oct[comp * n + ((long long)abs(k) * ny + abs(j)) * nx + abs(i)];
        const int sx = i < 0 ? -1 : 1, sy = j < 0 ? -1 : 1, sz = k < 0 ? -1 : 1;
        if (comp == 3) v *= sx * sy;
        else if (comp == 4) v *= sx * sz;
        else if (comp == 5) v *= sy * sz;
    }
    dst[q] = v;
}

template <typename T>
__global__ void extract_khat_kernel(const double2* __restrict__ spec, int Wk, int Kx, int Py, int Pz,
                                    int Ky, int Kz, double scale, T* __restrict__ khat) {
    const long long n = (long long)Kz * Ky * Wk;
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int kx = (int)(q % Wk), ky = (int)((q / Wk) % Ky), kz = (int)(q / ((long long)Wk * Ky));
    T v = 0;
    if (kx < Kx) v = (T)(scale * spec[((long long)kz * Py + ky) * Wk + kx].x);
    khat[q] = v;
}

template <typename T>
__global__ void khat_to_double_kernel(const T* __restrict__ k, long long n, double* __restrict__ out) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q < n) out[q] = (double)k[q];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static void gauss_legendre_host(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double t = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double step = p1 / dp;
            t -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

static GLTable make_gl() {
    GLTable g{};
    const int orders[5] = {16, 12, 6, 4, 3};
    int o = 0;
    for (int b = 0; b < 5; ++b) {
        g.off[b] = o;
        g.n[b] = orders[b];
        gauss_legendre_host(orders[b], g.x + o, g.w + o);
        o += orders[b];
    }
    return g;
}

template <typename T>
static void* make_twiddles(int L) {
    std::vector<cplx<T>> h(L);
    for (int q = 0; q < L; ++q) {
        const double a = -2.0 * kPi * (double)q / (double)L;
        h[q] = mkc<T>((T)std::cos(a), (T)std::sin(a));
    }
    void* d = nullptr;
    if (cudaMalloc(&d, sizeof(cplx<T>) * L) != cudaSuccess) return nullptr;
    cudaMemcpy(d, h.data(), sizeof(cplx<T>) * L, cudaMemcpyHostToDevice);
    return d;
}

static int col_threads(int L) { return L >= 512 ? 512 : 256; }

// multiprocessors of the current device (cached per device)
static int sm_count() {
    static int cache[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 152;
    }
    return cache[dev];
}

static int col_tk(int L, int nc) {
    const int cap = kMaxV * col_threads(L) / (L * nc);
    int tk = 1;
    while (tk * 2 <= cap && tk * 2 <= 16) tk *= 2;
    return tk;
}

// Lengths with a compile-time FFT (FP32): every half-length and column
// length of the benchmark workloads; other lengths and FP64 take the
// runtime-planned path.
#define MM_CT_LENGTHS(X) \
    X(16) X(32) X(48) X(64) X(81) X(96) X(108) X(128) X(162) X(192) X(216) X(256) X(324) X(432) X(512) X(1024)

template <typename T> using XKern = void (*)(XArgs<T>);
template <typename T> using CKern = void (*)(ColArgs<T>);

template <typename T>
static XKern<T> x_kernel(bool fwd, int Lh) {
    if constexpr (sizeof(T) == 4) {
        switch (Lh) {
#define MM_CASE(n) case n: return fwd ? fft_x_r2c_direct_kernel<n> : fft_x_c2r_direct_kernel<n>;
            MM_CT_LENGTHS(MM_CASE)
#undef MM_CASE
            default: break;
        }
    }
    return fwd ? fft_x_r2c_kernel<T, 0> : fft_x_c2r_kernel<T, 0>;
}

template <typename T, int MODE>
static CKern<T> col_kernel(int L) {
    if constexpr (sizeof(T) == 4) {
        switch (L) {
#define MM_CASE(n) case n: return fft_col_kernel<T, MODE, n>;
            MM_CT_LENGTHS(MM_CASE)
#undef MM_CASE
            default: break;
        }
    }
    return fft_col_kernel<T, MODE, 0>;
}

// lanes per row of the one-row-per-warp kernels (warp_group of the length)
static int x_warp_group(int Lh) {
    switch (Lh) {
#define MM_CASE(n) case n: return warp_group(n);
        MM_CASE(32) MM_CASE(48) MM_CASE(64) MM_CASE(96) MM_CASE(128) MM_CASE(192) MM_CASE(216) MM_CASE(256) MM_CASE(324) MM_CASE(432)
        MM_CASE(512)
#undef MM_CASE
        default: return 32;
    }
}

static XKern<float> x_warp_kernel(bool fwd, int Lh) {
    switch (Lh) {
#define MM_CASE(n) case n: return fwd ? fft_x_r2c_warp_kernel<n, 0> : fft_x_c2r_warp_kernel<n>;
        MM_CASE(32) MM_CASE(48) MM_CASE(64) MM_CASE(96) MM_CASE(128) MM_CASE(192) MM_CASE(216) MM_CASE(256) MM_CASE(324) MM_CASE(432)
        MM_CASE(512)
#undef MM_CASE
        default: return nullptr;
    }
}

// prefetching C2R (persistent warps); null where the plain warp kernel is used
#define MM_XPIPE_LENGTHS(X) X(256) X(512)
static XKern<float> x_c2r_pipe_kernel(int Lh) {
    switch (Lh) {
#define MM_CASE(n) case n: return fft_x_c2r_pipe_kernel<n>;
        MM_XPIPE_LENGTHS(MM_CASE)
#undef MM_CASE
        default: return nullptr;
    }
}
static size_t x_c2r_pipe_smem(int Lh) {
    switch (Lh) {
#define MM_CASE(n) case n: return xpipe_smem<n>();
        MM_XPIPE_LENGTHS(MM_CASE)
#undef MM_CASE
        default: return 0;
    }
}

// R2C fused with RK45 stage s (1..6); null where the warp path does not apply
static XKern<float> x_stage_kernel(int s, int Lh) {
#define MM_ST(n) \
    case n: { \
        static XKern<float> const t[7] = {nullptr, fft_x_r2c_warp_kernel<n, 1>, fft_x_r2c_warp_kernel<n, 2>, \
                                          fft_x_r2c_warp_kernel<n, 3>, fft_x_r2c_warp_kernel<n, 4>, \
                                          fft_x_r2c_warp_kernel<n, 5>, fft_x_r2c_warp_kernel<n, 6>}; \
        return (s >= 1 && s <= 6) ? t[s] : nullptr; \
    }
    switch (Lh) {
        MM_ST(192) MM_ST(216) MM_ST(256) MM_ST(324) MM_ST(432) MM_ST(512)
        default: return nullptr;
    }
#undef MM_ST
}

using YKern = void (*)(YArgs<float>);
using ZKern = void (*)(ZArgs<float>);

static YKern y_direct_kernel(bool fwd, int L) {
    switch (L) {
#define MM_CASE(n) case n: return fwd ? fft_y_direct_kernel<float, 1, n> : fft_y_direct_kernel<float, -1, n>;
        MM_CT_LENGTHS(MM_CASE)
#undef MM_CASE
        default: return nullptr;
    }
}

// half: nz <= Pz/2 (the zero-padded upper half of every z line is known)
static ZKern zconv_reg_kernel(int L, bool half) {
    switch (L) {
#define MM_CASE(n) case n: return half ? fft_zconv_reg_kernel<float, n, true> : fft_zconv_reg_kernel<float, n, false>;
        MM_CASE(4) MM_CASE(8) MM_CASE(16) MM_CASE(32)
#undef MM_CASE
        default: return nullptr;
    }
}

static size_t y_direct_smem(int L) { return (size_t)L * y_direct_tk(L) * sizeof(cplx<float>); }
static size_t zconv_reg_smem(int L) { return (size_t)(L + 3 * L * kZT) * sizeof(cplx<float>); }

template <typename T>
static void launch_x(mm_ctx* c, bool forward, const T* in, T* out_real, cplx<T>* spec, int rows,
                     int rows_per_plane, int spec_rows_per_plane, int nx, long long in_pitch, int Lh,
                     const cplx<T>* tw, bool scale_ms, long long cells_per_comp, int stage = 0) {
    XArgs<T> a{};
    if (stage > 0) {
        a.st = c->d_state;
        a.kptr = (T* const*)c->d_kslot;
        a.m0 = (const T*)c->d_m;
        a.ms = (T*)c->d_mtmp;
    }
    a.in = in;
    a.out_real = out_real;
    a.spec = spec;
    a.in_pitch = in_pitch;
    a.rows = rows;
    a.rows_per_plane = rows_per_plane;
    a.spec_rows_per_plane = spec_rows_per_plane;
    a.nx = nx;
    a.Lh = Lh;
    a.Kx = Lh + 1;
    a.Wk = c->dm.Wk;
    make_plan(Lh, &a.plan);
    a.tw = tw;
    a.ms_uniform = (T)1;
    if (scale_ms) {
        if (c->uniform) a.ms_uniform = (T)c->regions[0].Ms;
        else {
            a.region = (const uint8_t*)c->d_region;
            a.lut = (const Region<T>*)c->d_lut;
        }
    }
    a.cells_per_comp = cells_per_comp;
    a.stage = stage;
    if constexpr (sizeof(T) == 4) {
        if (stage > 0 && x_stage_kernel(stage, Lh)) {
            // stage s reads m0 and the s slopes (s - 1 at stage 7), writes m_s and the spectrum
            const double reads = (double)(1 + stage - (stage == 6 ? 1 : 0));
            const size_t smem = (size_t)kXW * wline(Lh) * sizeof(float2);
            LaunchScope ls(c, "fft_x_r2c_stage",
                           (double)rows * ((reads + 1.0) * nx * sizeof(T) + (Lh + 1) * sizeof(cplx<T>)));
            x_stage_kernel(stage, Lh)<<<(rows + kXW - 1) / kXW, 32 * kXW, smem, c->stream>>>(a);
            return;
        }
        if (!forward && stage == 0 && x_c2r_pipe_kernel(Lh) && c->dm.Wk % 2 == 0) {
            static int occ_by_len[2] = {0, 0};     // Lh = 256, 512
            int& occ = occ_by_len[Lh == 512 ? 1 : 0];
            if (!occ) {
                int o = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, x_c2r_pipe_kernel(Lh), 32 * kXW,
                                                              x_c2r_pipe_smem(Lh));
                occ = std::max(1, o);
            }
            const int grid = std::max(1, std::min((rows + kXW - 1) / kXW, occ * sm_count()));
            LaunchScope ls(c, "fft_x_c2r", (double)rows * (nx * sizeof(T) + (Lh + 1) * sizeof(cplx<T>)));
            x_c2r_pipe_kernel(Lh)<<<grid, 32 * kXW, x_c2r_pipe_smem(Lh), c->stream>>>(a);
            return;
        }
        // the plain one-row-per-warp kernels take no stage combine: with a
        // stage to form they are only used through x_stage_kernel above
        XKern<float> wk = stage == 0 ? x_warp_kernel(forward, Lh) : nullptr;
        if (wk) {
            const int rpc = kXW * (32 / x_warp_group(Lh));      // rows per CTA
            const size_t smem = (size_t)rpc * wline(Lh) * sizeof(float2);
            LaunchScope ls(c, forward ? "fft_x_r2c" : "fft_x_c2r",
                           (double)rows * (nx * sizeof(T) + (Lh + 1) * sizeof(cplx<T>)));
            wk<<<(rows + rpc - 1) / rpc, 32 * kXW, smem, c->stream>>>(a);
            return;
        }
    }
    int rpc = std::max(1, kMaxV * 256 / Lh);
    rpc = std::min(rpc, 16);
    const size_t smem = (size_t)rpc * (Lh + 1) * sizeof(cplx<T>);
    // small grids: fewer rows per CTA so that at least two CTAs per SM run
    rpc = std::max(1, std::min(rpc, (rows + 2 * sm_count() - 1) / (2 * sm_count())));
    a.rpc = rpc;
    const int grid = (rows + rpc - 1) / rpc;
    const double reads = stage > 0 ? (double)(1 + stage - (stage == 6 ? 1 : 0)) + 1.0 : 1.0;
    LaunchScope ls(c, stage > 0 ? "fft_x_r2c_stage" : forward ? "fft_x_r2c" : "fft_x_c2r",
                   (double)rows * (reads * nx * sizeof(T) + (Lh + 1) * sizeof(cplx<T>)));
    x_kernel<T>(forward, Lh)<<<grid, 256, smem, c->stream>>>(a);
}

template <typename T, int MODE>
static void launch_col(mm_ctx* c, ColArgs<T> a, int n_other, const char* name, double bytes) {
    make_plan(a.L, &a.plan);
    const int thr = col_threads(a.L);
    a.TK = col_tk(a.L, a.nc);
    // small grids: narrower column groups so that at least two CTAs per SM run
    while (a.TK > 1 && (long long)((a.Kx + a.TK - 1) / a.TK) * n_other < 2LL * sm_count()) a.TK /= 2;
    const size_t smem = (size_t)a.nc * a.TK * (a.L + 1) * sizeof(cplx<T>);
    dim3 grid((a.Kx + a.TK - 1) / a.TK, n_other);
    LaunchScope ls(c, name, bytes);
    col_kernel<T, MODE>(a.L)<<<grid, thr, smem, c->stream>>>(a);
}

static void launch_y_direct(mm_ctx* c, bool fwd, cplx<float>* S, long long plane, int n_in, int n_out,
                            const char* name, double bytes) {
    const DemagPlan& d = c->dm;
    YArgs<float> a{};
    a.base = S; a.plane = plane; a.Kx = d.Kx; a.Wk = d.Wk;
    a.ncols = 3 * c->grid.nz * d.Kx;
    a.n_in = n_in; a.n_out = n_out;
    a.tw = (const cplx<float>*)d.tw_y;
    LaunchScope ls(c, name, bytes);
    const int tk = y_direct_tk(d.Py);
    y_direct_kernel(fwd, d.Py)<<<(unsigned)((a.ncols + tk - 1) / tk), y_direct_threads(d.Py), y_direct_smem(d.Py),
                                 c->stream>>>(a);
}

// c2r = false: every pass but the inverse X pass (which the fused inverse-X +
// field kernel then runs); Hd is not written.
template <typename T>
static void demag_apply_t(mm_ctx* c, const T* m, T* Hd, int stage = 0, bool c2r = true) {
    DemagPlan& d = c->dm;
    const mm_grid& g = c->grid;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    cplx<T>* S = (cplx<T>*)d.spec;
    const long long plane = (long long)d.PyA * d.Wk;        // one z-plane of one component
    const long long comp = (long long)nz * plane;
    const long long N = c->N;
    const double cplxb = sizeof(cplx<T>), realb = sizeof(T);
    // X forward: rows (c, z, y) of Ms*m
    launch_x<T>(c, true, m, nullptr, S, 3 * nz * ny, ny, d.PyA, nx, nx, d.Lh, (const cplx<T>*)d.tw_x, true, N,
                stage);
    const bool three_d = nz > 1;
    const bool fast_y = sizeof(T) == 4 && three_d && y_direct_kernel(true, d.Py) != nullptr;
    const bool fast_z = sizeof(T) == 4 && three_d && zconv_reg_kernel(d.Pz, false) != nullptr;
    const bool split_y = sizeof(T) == 4 && three_d && ysplit_supported(d.Py);
    if (three_d && d.Py > 1 && split_y) {
        ysplit_launch(c, true, S, nz, d.Py, d.Kx, d.Wk, ny, d.Py, "fft_y_fwd", 3.0 * nz * d.Kx * (ny + d.Py) * cplxb);
    } else if (three_d && d.Py > 1 && fast_y) {
        launch_y_direct(c, true, (cplx<float>*)S, plane, ny, d.Py, "fft_y_fwd",
                        3.0 * nz * d.Kx * (ny + d.Py) * cplxb);
    } else if (three_d && d.Py > 1) {
        ColArgs<T> a{};
        a.base = S; a.comp_stride = comp; a.line_stride = d.Wk; a.other_stride = plane;
        a.nc = 3; a.Kx = d.Kx; a.L = d.Py; a.n_in = ny; a.n_out = d.Py;
        a.tw = (const cplx<T>*)d.tw_y;
        launch_col<T, 1>(c, a, nz, "fft_y_fwd", 3.0 * nz * d.Kx * (ny + d.Py) * cplxb);
    }
    {
        ColArgs<T> a{};
        a.base = S; a.comp_stride = comp; a.nc = 3; a.Kx = d.Kx;
        a.khat = (const T*)d.khat;
        a.ncomp = d.ncomp;
        const long long Ky = d.Py / 2 + 1, Kz = d.Pz / 2 + 1;
        a.kc_stride = Kz * Ky * d.Wk;
        if (three_d && fast_z) {
            ZArgs<float> z{};
            z.base = (cplx<float>*)S; z.comp_stride = comp; z.plane = plane;
            z.nz = nz; z.Py = d.Py; z.Kx = d.Kx; z.Wk = d.Wk;
            z.tw = (const cplx<float>*)d.tw_z;
            z.khat = (const float*)d.khat;
            z.kc_stride = a.kc_stride; z.kk_stride = Ky * d.Wk;
            const long long cols = (long long)d.Py * d.Wk;
            LaunchScope ls(c, "fft_conv",
                           3.0 * d.Py * d.Kx * 2 * nz * cplxb + (double)d.ncomp * Kz * Ky * d.Kx * realb);
            zconv_reg_kernel(d.Pz, 2 * nz <= d.Pz)<<<(unsigned)((cols + kZT - 1) / kZT), 3 * kZT, zconv_reg_smem(d.Pz),
                                                      c->stream>>>(z);
        } else if (three_d && sizeof(T) == 4 && split_conv_supported(d.Pz)) {
            split_conv_launch_3d(c, S, d.khat, nz, d.Py, d.Pz, d.Kx, d.Wk,
                                 3.0 * d.Py * d.Kx * 2 * nz * cplxb + (double)d.ncomp * Kz * Ky * d.Kx * realb);
        } else if (three_d) {
            a.line_stride = plane; a.other_stride = d.Wk;
            a.L = d.Pz; a.n_in = nz; a.n_out = nz;
            a.tw = (const cplx<T>*)d.tw_z;
            a.kk_stride = Ky * d.Wk; a.ko_stride = d.Wk;
            a.L_other = d.Py; a.axis_is_y = 0;
            launch_col<T, 0>(c, a, d.Py, "fft_conv",
                             3.0 * d.Py * d.Kx * 2 * nz * cplxb + (double)d.ncomp * Kz * Ky * d.Kx * realb);
        } else if (sizeof(T) == 4 && split_conv_supported(d.Py)) {
            split_conv_launch_2d(c, S, d.khat, ny, d.Py, d.Kx, d.Wk, comp, 3 * comp, 1, "fft_conv",
                                 3.0 * d.Kx * 2 * ny * cplxb + (double)d.ncomp * Ky * d.Kx * realb);
        } else {
            a.line_stride = d.Wk; a.other_stride = plane;
            a.L = d.Py; a.n_in = ny; a.n_out = ny;
            a.tw = (const cplx<T>*)d.tw_y;
            a.kk_stride = d.Wk; a.ko_stride = 0;
            a.L_other = 1; a.axis_is_y = 1;
            launch_col<T, 0>(c, a, 1, "fft_conv",
                             3.0 * d.Kx * 2 * ny * cplxb + (double)d.ncomp * Ky * d.Kx * realb);
        }
    }
    if (three_d && d.Py > 1 && split_y) {
        ysplit_launch(c, false, S, nz, d.Py, d.Kx, d.Wk, d.Py, ny, "fft_y_inv", 3.0 * nz * d.Kx * (ny + d.Py) * cplxb);
    } else if (three_d && d.Py > 1 && fast_y) {
        launch_y_direct(c, false, (cplx<float>*)S, plane, d.Py, ny, "fft_y_inv",
                        3.0 * nz * d.Kx * (ny + d.Py) * cplxb);
    } else if (three_d && d.Py > 1) {
        ColArgs<T> a{};
        a.base = S; a.comp_stride = comp; a.line_stride = d.Wk; a.other_stride = plane;
        a.nc = 3; a.Kx = d.Kx; a.L = d.Py; a.n_in = d.Py; a.n_out = ny;
        a.tw = (const cplx<T>*)d.tw_y;
        launch_col<T, -1>(c, a, nz, "fft_y_inv", 3.0 * nz * d.Kx * (ny + d.Py) * cplxb);
    }
    if (c2r)
        launch_x<T>(c, false, nullptr, Hd, S, 3 * nz * ny, ny, d.PyA, nx, nx, d.Lh, (const cplx<T>*)d.tw_x, false, N);
}

// Demag of Rc equal thin films stored back to back ([replica][component][y]
// [x], FP32): the 2-D passes of one film run over all of them at once -- the
// X pass over 3 ny Rc rows, the column convolution over Rc film planes with
// the shared tensor spectrum (it does not depend on the plane), the inverse
// X pass -- with the spectrum S laid out [replica][component][PyA][Wk].
void demag_apply_stacked2d(mm_ctx* c, const DemagPlan& p, const float* m, float* Hd, void* S, int nx, int ny,
                           int Rc) {
    const DemagPlan saved = c->dm;
    c->dm = p;                                   // launch_x reads the plan's row pitch
    cplx<float>* Sp = (cplx<float>*)S;
    const long long plane = (long long)p.PyA * p.Wk;
    const long long N = (long long)nx * ny;
    const double cplxb = sizeof(cplx<float>), realb = sizeof(float);
    launch_x<float>(c, true, m, nullptr, Sp, 3 * ny * Rc, ny, p.PyA, nx, nx, p.Lh, (const cplx<float>*)p.tw_x, true,
                    N);
    if (split_conv_supported(p.Py)) {
        split_conv_launch_2d(c, Sp, p.khat, ny, p.Py, p.Kx, p.Wk, plane, 3 * plane, Rc, "fft_conv_stacked",
                             Rc * (3.0 * p.Kx * 2 * ny * cplxb) + (double)p.ncomp * (p.Py / 2 + 1) * p.Kx * realb);
    } else {
        ColArgs<float> a{};
        a.base = Sp; a.comp_stride = plane; a.nc = 3; a.Kx = p.Kx;
        a.khat = (const float*)p.khat;
        a.ncomp = p.ncomp;
        const long long Ky = p.Py / 2 + 1;
        a.kc_stride = Ky * p.Wk;
        a.line_stride = p.Wk; a.other_stride = 3 * plane;
        a.L = p.Py; a.n_in = ny; a.n_out = ny;
        a.tw = (const cplx<float>*)p.tw_y;
        a.kk_stride = p.Wk; a.ko_stride = 0;
        a.L_other = 1; a.axis_is_y = 1;
        launch_col<float, 0>(c, a, Rc, "fft_conv_stacked",
                             Rc * (3.0 * p.Kx * 2 * ny * cplxb) + (double)p.ncomp * Ky * p.Kx * realb);
    }
    launch_x<float>(c, false, nullptr, Hd, Sp, 3 * ny * Rc, ny, p.PyA, nx, nx, p.Lh, (const cplx<float>*)p.tw_x,
                    false, N);
    c->dm = saved;
}

void demag_apply(mm_ctx* c, const void* m, void* Hd) {
    if (c->prec == 32) demag_apply_t<float>(c, (const float*)m, (float*)Hd);
    else demag_apply_t<double>(c, (const double*)m, (double*)Hd);
}

// The one-row-per-warp X pass takes the stage combine at no cost; the
// CTA-wide R2C kernels read the slopes with scalar loads, which only pays
// on small grids where launches, not bandwidth, set the time (measured:
// 10 K cells faster, 540 K cells 10 % slower fused).
bool demag_stage_fusable(const mm_ctx* c) {
    if (c->prec != 32 || !c->dm.on || c->grid.nx % 2 != 0) return false;
    return x_stage_kernel(1, c->dm.Lh) != nullptr || c->N <= 131072;
}

void demag_apply_stage(mm_ctx* c, int stage, void* Hd) {
    demag_apply_t<float>(c, (const float*)c->d_mtmp, (float*)Hd, stage);
}

void demag_apply_partial(mm_ctx* c, const void* m, int stage) {
    demag_apply_t<float>(c, (const float*)(stage > 0 ? c->d_mtmp : m), nullptr, stage, false);
}

template <typename T>
static mm_status demag_setup_t(mm_ctx* c) {
    DemagPlan& d = c->dm;
    const mm_grid& g = c->grid;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    d.Px = nice_length(std::max(2, 2 * nx - 1), true);
    d.Py = ny > 1 ? nice_length(2 * ny - 1, false) : 1;
    d.Pz = nz > 1 ? nice_length(2 * nz - 1, false) : 1;
    if (d.Px > 8192 || d.Py > 4096 || d.Pz > 4096)
        return set_error(c, MM_ERR_ARG, "demag supports padded lengths up to 8192 (x) and 4096 (y, z)");
    d.Lh = d.Px / 2;
    d.Kx = d.Lh + 1;
    d.Wk = (d.Kx + 3) / 4 * 4;
    d.PyA = nz > 1 ? d.Py : ny;
    d.ncomp = nz > 1 ? 6 : 4;
    const int Ky = d.Py / 2 + 1, Kz = d.Pz / 2 + 1;
    Plan tmp;
    if (!make_plan(d.Lh, &tmp) || !make_plan(d.Py, &tmp) || !make_plan(d.Pz, &tmp))
        return set_error(c, MM_ERR_ARG, "internal: padded length is not 2^a 3^b");

    // twiddles in working precision, and FP64 twiddles for the setup FFTs
    d.tw_x = make_twiddles<T>(d.Px);
    d.tw_y = make_twiddles<T>(d.Py);
    d.tw_z = make_twiddles<T>(d.Pz);
    void* tw64x = make_twiddles<double>(d.Px);
    void* tw64y = make_twiddles<double>(d.Py);
    void* tw64z = make_twiddles<double>(d.Pz);
    auto free_tw64 = [&] {   // the FP64 setup twiddles live until the tensor is built
        cudaFree(tw64x);
        cudaFree(tw64y);
        cudaFree(tw64z);
    };
    if (!d.tw_x || !d.tw_y || !d.tw_z || !tw64x || !tw64y || !tw64z) {
        free_tw64();
        return set_error(c, MM_ERR_OOM, "twiddles");
    }

    const size_t spec_bytes = (size_t)3 * nz * d.PyA * d.Wk * sizeof(cplx<T>);
    const size_t khat_bytes = (size_t)d.ncomp * Kz * Ky * d.Wk * sizeof(T);
    if (cudaMalloc(&d.spec, spec_bytes) != cudaSuccess) {
        free_tw64();
        return set_error(c, MM_ERR_OOM, "demag spectrum");
    }
    if (cudaMalloc(&d.khat, khat_bytes) != cudaSuccess) {
        free_tw64();
        return set_error(c, MM_ERR_OOM, "demag kernel");
    }
    cudaMemsetAsync(d.spec, 0, spec_bytes, c->stream);

    // FP64 Newell tensor on the non-negative octant
    const long long noct = (long long)nx * ny * nz;
    double* oct = nullptr;
    double* pad = nullptr;
    double2* sp = nullptr;
    const long long P = (long long)d.Px * d.Py * d.Pz;
    const size_t sp_elems = (size_t)d.Pz * d.Py * d.Wk;
    if (cudaMalloc(&oct, sizeof(double) * 6 * noct) != cudaSuccess ||
        cudaMalloc(&pad, sizeof(double) * P) != cudaSuccess ||
        cudaMalloc(&sp, sizeof(double2) * sp_elems) != cudaSuccess) {
        cudaFree(oct); cudaFree(pad); cudaFree(sp);
        free_tw64();
        return set_error(c, MM_ERR_OOM, "demag setup scratch");
    }
    GLTable gl = make_gl();
    {
        LaunchScope ls(c, "newell_octant", 48.0 * noct);
        newell_octant_kernel<<<(unsigned)((noct + 127) / 128), 128, 0, c->stream>>>(
            nx, ny, nz, g.dx, g.dy, g.dz, gl, std::max(0, g.pbc[0]), std::max(0, g.pbc[1]), std::max(0, g.pbc[2]),
            oct);
    }
    // temporarily point the X-pass geometry at the padded tensor
    const int saveWk = d.Wk;
    for (int comp = 0; comp < d.ncomp; ++comp) {
        // nz = 1 stores xx, yy, zz, xy (xz = yz = 0)
        const int src = comp;
        {
            LaunchScope ls(c, "newell_pad", 8.0 * P);
            padded_component_kernel<<<(unsigned)((P + 255) / 256), 256, 0, c->stream>>>(oct, src, nx, ny, nz, d.Px,
                                                                                        d.Py, d.Pz, pad);
        }
        cudaMemsetAsync(sp, 0, sizeof(double2) * sp_elems, c->stream);
        // X: rows (z, y) of the padded real tensor, all Px entries nonzero
        launch_x<double>(c, true, pad, nullptr, (cplx<double>*)sp, d.Py * d.Pz, d.Py * d.Pz, d.Py * d.Pz, d.Px,
                         d.Px, d.Lh, (const cplx<double>*)tw64x, false, P);
        if (d.Py > 1) {
            ColArgs<double> a{};
            a.base = (cplx<double>*)sp; a.comp_stride = 0; a.line_stride = d.Wk;
            a.other_stride = (long long)d.Py * d.Wk; a.nc = 1; a.Kx = d.Kx;
            a.L = d.Py; a.n_in = d.Py; a.n_out = d.Py; a.tw = (const cplx<double>*)tw64y;
            launch_col<double, 1>(c, a, d.Pz, "newell_fft_y", 0.0);
        }
        if (d.Pz > 1) {
            ColArgs<double> a{};
            a.base = (cplx<double>*)sp; a.comp_stride = 0; a.line_stride = (long long)d.Py * d.Wk;
            a.other_stride = d.Wk; a.nc = 1; a.Kx = d.Kx;
            a.L = d.Pz; a.n_in = d.Pz; a.n_out = d.Pz; a.tw = (const cplx<double>*)tw64z;
            launch_col<double, 1>(c, a, d.Py, "newell_fft_z", 0.0);
        }
        const long long nk = (long long)Kz * Ky * saveWk;
        const double scale = -1.0 / ((double)d.Px * d.Py * d.Pz);
        LaunchScope ls(c, "newell_extract", 0.0);
        extract_khat_kernel<T><<<(unsigned)((nk + 255) / 256), 256, 0, c->stream>>>(
            sp, saveWk, d.Kx, d.Py, d.Pz, Ky, Kz, scale, (T*)d.khat + comp * nk);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    cudaFree(oct);
    cudaFree(pad);
    cudaFree(sp);
    free_tw64();
    if (e != cudaSuccess) return cuda_check(c, e, "demag setup");
    d.on = 1;
    return MM_OK;
}

// Opt every FFT kernel into the full 227 KB of dynamic shared memory once,
// outside any stream capture.
template <typename K>
static cudaError_t smem_attr(K k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

template <typename T>
static cudaError_t fft_attributes() {
    static const int lengths[] = {0, 16, 32, 48, 64, 81, 96, 108, 128, 162, 192, 216, 256, 324, 432, 512, 1024};
    cudaError_t e = cudaSuccess;
    for (int L : lengths) {
        if (L != 0 && sizeof(T) != 4) continue;
        const int n = L == 0 ? 7 : L;
        if (e == cudaSuccess) e = smem_attr(x_kernel<T>(true, n));
        if (e == cudaSuccess) e = smem_attr(x_kernel<T>(false, n));
        if (e == cudaSuccess) e = smem_attr(col_kernel<T, 1>(n));
        if (e == cudaSuccess) e = smem_attr(col_kernel<T, -1>(n));
        if (e == cudaSuccess) e = smem_attr(col_kernel<T, 0>(n));
    }
    return e;
}

static cudaError_t fast_attributes() {
    cudaError_t e = cudaSuccess;
    for (int L : {16, 32, 48, 64, 81, 96, 108, 128, 162, 192, 216, 256, 324, 432, 512, 1024}) {
        if (e == cudaSuccess) e = smem_attr(y_direct_kernel(true, L));
        if (e == cudaSuccess) e = smem_attr(y_direct_kernel(false, L));
    }
    for (int L : {4, 8, 16, 32}) {
        if (e == cudaSuccess) e = smem_attr(zconv_reg_kernel(L, false));
        if (e == cudaSuccess) e = smem_attr(zconv_reg_kernel(L, true));
    }
    for (int L : {256, 512})
        if (e == cudaSuccess) e = smem_attr(x_c2r_pipe_kernel(L));
    for (int L : {192, 216, 256, 324, 432, 512}) {
        if (e == cudaSuccess) e = smem_attr(x_warp_kernel(true, L));
        if (e == cudaSuccess) e = smem_attr(x_warp_kernel(false, L));
        for (int st = 1; st <= 6; ++st)
            if (e == cudaSuccess) e = smem_attr(x_stage_kernel(st, L));
    }
    return e;
}

mm_status demag_setup(mm_ctx* c) {
    // length-32 twiddles of the register z pass (per device; cheap to repeat)
    float2 tw32[32];
    for (int q = 0; q < 32; ++q) {
        const double ang = -2.0 * kPi * (double)q / 32.0;
        tw32[q] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_tw32, tw32, sizeof tw32);
    if (e == cudaSuccess) e = split_conv_setup();
    if (e == cudaSuccess) e = field_c2r_setup();
    if (e != cudaSuccess) return cuda_check(c, e, "twiddle table");
    e = fft_attributes<float>();
    if (e == cudaSuccess) e = fast_attributes();
    if (e == cudaSuccess) e = fft_attributes<double>();
    if (e != cudaSuccess) return cuda_check(c, e, "FFT kernel attributes");
    return c->prec == 32 ? demag_setup_t<float>(c) : demag_setup_t<double>(c);
}

// Tensor spectrum and twiddles of one grid (a replica size class), built
// with the context's precision without touching the context's own plan.
mm_status demag_setup_for(mm_ctx* c, const mm_grid& g, DemagPlan* out) {
    const mm_grid sg = c->grid;
    const long long sN = c->N;
    const DemagPlan sd = c->dm;
    c->grid = g;
    c->N = (long long)g.nx * g.ny * g.nz;
    c->dm = DemagPlan{};
    mm_status s = demag_setup(c);
    *out = c->dm;
    c->grid = sg;
    c->N = sN;
    c->dm = sd;
    return s;
}

void demag_free_plan(DemagPlan& d) {
    cudaFree(d.spec);
    cudaFree(d.khat);
    cudaFree(d.tw_x);
    cudaFree(d.tw_y);
    cudaFree(d.tw_z);
    d = DemagPlan{};
}

void demag_free(mm_ctx* c) {
    DemagPlan& d = c->dm;
    cudaFree(d.spec);
    cudaFree(d.khat);
    cudaFree(d.tw_x);
    cudaFree(d.tw_y);
    cudaFree(d.tw_z);
    d = DemagPlan{};
}

mm_status newell_gpu(long count, const int* ijk, double dx, double dy, double dz, double* out_host) {
    int* d_ijk = nullptr;
    double* d_out = nullptr;
    if (count <= 0) return MM_OK;
    if (cudaMalloc(&d_ijk, sizeof(int) * 3 * count) != cudaSuccess) return MM_ERR_OOM;
    if (cudaMalloc(&d_out, sizeof(double) * 6 * count) != cudaSuccess) {
        cudaFree(d_ijk);
        return MM_ERR_OOM;
    }
    cudaMemcpy(d_ijk, ijk, sizeof(int) * 3 * count, cudaMemcpyHostToDevice);
    GLTable gl = make_gl();
    newell_list_kernel<<<(unsigned)((count + 127) / 128), 128>>>(count, d_ijk, dx, dy, dz, gl, d_out);
    cudaError_t e = cudaMemcpy(out_host, d_out, sizeof(double) * 6 * count, cudaMemcpyDeviceToHost);
    cudaFree(d_ijk);
    cudaFree(d_out);
    return e == cudaSuccess ? MM_OK : MM_ERR_CUDA;
}

// Stored tensor spectrum -> host doubles (test access).
mm_status demag_kernel_copy(mm_ctx* c, double* out, size_t n_out, int* dims) {
    DemagPlan& d = c->dm;
    if (!d.on) return set_error(c, MM_ERR_STATE, "demag is off");
    const int Ky = d.Py / 2 + 1, Kz = d.Pz / 2 + 1;
    const size_t need = (size_t)d.ncomp * Kz * Ky * d.Kx;
    if (dims) { dims[0] = d.ncomp; dims[1] = d.Px; dims[2] = d.Py; dims[3] = d.Pz; }
    if (!out) return MM_OK;
    if (n_out < need) return set_error(c, MM_ERR_ARG, "output too small for the tensor spectrum");
    const long long nk = (long long)d.ncomp * Kz * Ky * d.Wk;
    double* tmp = nullptr;
    if (cudaMalloc(&tmp, sizeof(double) * nk) != cudaSuccess) return set_error(c, MM_ERR_OOM, "copy");
    if (c->prec == 32) khat_to_double_kernel<float><<<(unsigned)((nk + 255) / 256), 256, 0, c->stream>>>((const float*)d.khat, nk, tmp);
    else khat_to_double_kernel<double><<<(unsigned)((nk + 255) / 256), 256, 0, c->stream>>>((const double*)d.khat, nk, tmp);
    std::vector<double> h(nk);
    cudaError_t e = cudaMemcpyAsync(h.data(), tmp, sizeof(double) * nk, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_check(c, e, "tensor copy");
    size_t o = 0;
    for (long long r = 0; r < nk / d.Wk; ++r)
        for (int kx = 0; kx < d.Kx; ++kx) out[o++] = h[r * d.Wk + kx];
    return MM_OK;
}

}  // namespace mm
