// Middle pass of the demag convolution (Methods, "Physics and discretization":
// the zero-padded FFT convolution with the Newell tensor) for line lengths
// too long to keep in one thread's registers: L = G * Q, each line split over
// G threads of Q values (the four-step factorisation of the DFT).
//
//   X[k1 + Q k2] = sum_t W_G^(t k2) [ W_L^(t k1) sum_q x[q G + t] W_Q^(q k1) ]
//
// Phase 1 (thread t of a column, all three components): its Q strided inputs
// x[q G + t] straight from global memory into registers, Q-point FFT, twiddle
// W_L^(t k1), one store of the line part to shared memory.
// Phase 2 (item (k1, column)): the G values of every component, G-point DFT,
// H^ = K^ M^ with the real symmetry-compressed tensor (row folding and parity
// signs as in the stored half range), inverse G-point DFT, stored back in
// place -- an item's slots belong to it alone, so no barrier inside.
// Phase 3: the inverse of phase 1, keeping only the n_in un-padded outputs.
// Inputs beyond the un-padded n_in of a line are compile-time zeros (q >=
// QIN), so the compiler drops the additions they would feed; outputs past
// QIN are never formed.  Every twiddle with a compile-time exponent is a
// constant-bank operand of its multiply (tables filled once per process).
//
// Columns are flattened (other-axis index, kx) positions, TC consecutive per
// CTA.  In 3-D (line axis z, other axis y) CTA 2j takes columns at ky and CTA
// 2j + 1 the mirrored ky' = Py - ky: both read the same stored tensor rows
// (ky folds to the half range), so the second read hits L2 and the tensor
// crosses the HBM bus once per evaluation.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "ctx.h"
#include "fft_ct.cuh"

namespace mm {

// exp(-2 pi i q / L), q < L, per supported line length
__constant__ float2 c_tw_16[16], c_tw_32[32], c_tw_48[48], c_tw_64[64], c_tw_81[81], c_tw_96[96],
    c_tw_108[108], c_tw_128[128], c_tw_192[192], c_tw_256[256], c_tw_512[512];

template <int L>
__device__ __forceinline__ float2 twc(int q) {
    if constexpr (L == 16) return c_tw_16[q];
    else if constexpr (L == 32) return c_tw_32[q];
    else if constexpr (L == 48) return c_tw_48[q];
    else if constexpr (L == 64) return c_tw_64[q];
    else if constexpr (L == 81) return c_tw_81[q];
    else if constexpr (L == 96) return c_tw_96[q];
    else if constexpr (L == 108) return c_tw_108[q];
    else if constexpr (L == 128) return c_tw_128[q];
    else if constexpr (L == 192) return c_tw_192[q];
    else if constexpr (L == 256) return c_tw_256[q];
    else return c_tw_512[q];
}

// v * W_L^q (DIR > 0) or v * conj(W_L^q); q is a compile-time constant after
// unrolling, so the exact quarter-turn cases cost no multiplication.
template <int DIR, int L>
__device__ __forceinline__ float2 twq(float2 v, int q) {
    if (q == 0) return v;
    if (2 * q == L) return make_float2(-v.x, -v.y);
    if (4 * q == L) return mul_mi<float, DIR>(v);
    if (4 * q == 3 * L) return mul_mi<float, -DIR>(v);
    const float2 w = twc<L>(q);
    return DIR > 0 ? cmul<float>(v, w) : cmulc<float>(v, w);
}

// In-register DFT of length N (natural order in and out), mixed radix
// 8/4/2/3 Stockham passes with every index a compile-time constant; the
// twiddles W_N^m are taken from the length-L table (N divides L).
template <int DIR, int N, int L, int P = 0>
__device__ __forceinline__ void rfft(float2 (&v)[N]) {
    if constexpr (P < ct_npass(N)) {
        constexpr int R = ct_radix(N, P), NS = ct_ns(N, P), NB = N / R, SPAN = N / (NS * R);
        float2 w[N];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            float2 u[R];
#pragma unroll
            for (int t = 0; t < R; ++t) u[t] = v[j + t * NB];
            const int k = j % NS;
            if constexpr (NS > 1) {
#pragma unroll
                for (int t = 1; t < R; ++t) u[t] = twq<DIR, L>(u[t], (t * k * SPAN) * (L / N));
            }
            dft_ct<float, DIR, R>(u);
            const int dst = (j / NS) * NS * R + k;
#pragma unroll
            for (int t = 0; t < R; ++t) w[dst + t * NS] = u[t];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = w[i];
        rfft<DIR, N, L, P + 1>(v);
    }
}

struct SplitArgs {
    float2* base;             // spectrum
    long long comp_stride;    // between the three components
    long long line_stride;    // between consecutive points of a line
    long long o_stride;       // between consecutive other-axis indices
    int Wk, Kx;               // columns per other-axis index (row pitch), valid ones
    int n_o;                  // 3-D: Py (other-axis length); 2-D: number of film planes
    long long n_cols;         // flattened columns enumerated by side 0
    int n_in;                 // un-padded points per line (inputs read, outputs kept)
    const float* khat;        // [ncomp][L/2+1][n_o/2+1 (3-D) or 1][Wk]
    long long kc, kk, ko;     // tensor strides: component, line frequency, other-axis frequency
};

// Tensor components xx yy zz xy xz yz = 0..5.  3-D (line z, other y): xy odd in
// y, xz odd in z, yz odd in both.  2-D (line y): xy odd in y; xz = yz = 0.
template <int L, int G, int Q, int TC, bool THREE_D>
__global__ void __launch_bounds__(G * TC) fft_conv_split_kernel(SplitArgs a) {
    static_assert(L == G * Q, "line length");
    constexpr int NT = G * TC;
    constexpr int NMAX = (L + 1) / 2;                 // 2 n_in - 1 <= L
    constexpr int QIN = (NMAX + G - 1) / G;           // register slots that can hold inputs
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);   // [3][G][Q][TC]
    const int col = threadIdx.x % TC, t = threadIdx.x / TC;

    // column of this thread
    int side = 0;
    long long p = (long long)blockIdx.x * TC + col;
    if constexpr (THREE_D) {
        side = blockIdx.x & 1;
        p = (long long)(blockIdx.x >> 1) * TC + col;
    }
    int o = (int)(p / a.Wk), kx = (int)(p - (long long)o * a.Wk);
    bool valid = p < a.n_cols && kx < a.Kx;
    int om = o;                                        // other-axis index of the data
    float so = 1.f;                                    // parity sign of the other axis
    if constexpr (THREE_D) {
        if (side) {
            valid = valid && o != 0 && 2 * o != a.n_o;
            om = a.n_o - o;
            so = -1.f;
        }
    }
    if (!valid) { o = 0; om = 0; kx = 0; }
    const long long gcol = (long long)om * a.o_stride + kx;
    const float* K = a.khat + (THREE_D ? (long long)o * a.ko : 0) + kx;

    // ---- phase 1: forward Q-point transforms of the strided line parts
    {
        float2 x[3][QIN];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < QIN; ++q) {
                const int n = q * G + t;
                x[c][q] = (valid && n < a.n_in) ? a.base[c * a.comp_stride + gcol + n * a.line_stride]
                                                 : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 v[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) v[q] = q < QIN ? x[c][q] : make_float2(0.f, 0.f);
            rfft<1, Q, L>(v);
#pragma unroll
            for (int k1 = 0; k1 < Q; ++k1) {
                float2 r = v[k1];
                if (G > 1 && k1 > 0) r = cmul<float>(r, twc<L>(t * k1));   // W_L^0 = 1 exactly
                sm[((c * G + t) * Q + k1) * TC + col] = r;
            }
        }
    }
    __syncthreads();

    // ---- phase 2: G-point DFTs across the line parts, tensor multiply, inverse
#pragma unroll 1
    for (int k1 = t; k1 < Q; k1 += G) {
        float2 m[3][G];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int u = 0; u < G; ++u) m[c][u] = sm[((c * G + u) * Q + k1) * TC + col];
#pragma unroll
        for (int c = 0; c < 3; ++c) rfft<1, G, L>(m[c]);
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) {
            const int kz = k1 + Q * k2;
            const bool fold = 2 * kz > L;
            const int kzf = fold ? L - kz : kz;
            const float st = fold ? -1.f : 1.f;
            const float* Kp = K + (long long)kzf * a.kk;
            const float kxx = __ldg(Kp), kyy = __ldg(Kp + a.kc), kzz = __ldg(Kp + 2 * a.kc);
            float kxy, kxz = 0.f, kyz = 0.f;
            if constexpr (THREE_D) {
                kxy = __ldg(Kp + 3 * a.kc) * so;
                kxz = __ldg(Kp + 4 * a.kc) * st;
                kyz = __ldg(Kp + 5 * a.kc) * (so * st);
            } else {
                kxy = __ldg(Kp + 3 * a.kc) * st;
            }
            const float2 mx = m[0][k2], my = m[1][k2], mz = m[2][k2];
            m[0][k2] = make_float2(kxx * mx.x + kxy * my.x + kxz * mz.x, kxx * mx.y + kxy * my.y + kxz * mz.y);
            m[1][k2] = make_float2(kxy * mx.x + kyy * my.x + kyz * mz.x, kxy * mx.y + kyy * my.y + kyz * mz.y);
            m[2][k2] = make_float2(kxz * mx.x + kyz * my.x + kzz * mz.x, kxz * mx.y + kyz * my.y + kzz * mz.y);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) rfft<-1, G, L>(m[c]);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int u = 0; u < G; ++u) sm[((c * G + u) * Q + k1) * TC + col] = m[c][u];
    }
    __syncthreads();

    // ---- phase 3: inverse Q-point transforms, the un-padded outputs only
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 v[Q];
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) {
            float2 r = sm[((c * G + t) * Q + k1) * TC + col];
            if (G > 1 && k1 > 0) r = cmulc<float>(r, twc<L>(t * k1));
            v[k1] = r;
        }
        rfft<-1, Q, L>(v);
        if (valid) {
#pragma unroll
            for (int q = 0; q < QIN; ++q) {
                const int n = q * G + t;
                if (n < a.n_in) a.base[c * a.comp_stride + gcol + n * a.line_stride] = v[q];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using SplitKern = void (*)(SplitArgs);

struct SplitShape {
    SplitKern k3, k2;   // 3-D and 2-D variants
    int G, TC;
};

// (L, G, Q, TC): TC columns per CTA so that G * TC is a whole number of warps
// and the exchange buffer 3 L TC complex values stays within 72 KB.
#define MM_SPLIT_SHAPES(X) \
    X(16, 1, 16, 64) X(32, 1, 32, 64) X(48, 3, 16, 32) X(64, 2, 32, 32) X(81, 3, 27, 32) X(96, 3, 32, 32) \
    X(108, 4, 27, 16) X(128, 4, 32, 16) X(192, 6, 32, 16) X(256, 8, 32, 8) X(512, 16, 32, 4)

static SplitShape split_shape(int L) {
    switch (L) {
#define MM_CASE(L_, G_, Q_, TC_) \
    case L_: return {fft_conv_split_kernel<L_, G_, Q_, TC_, true>, fft_conv_split_kernel<L_, G_, Q_, TC_, false>, G_, TC_};
        MM_SPLIT_SHAPES(MM_CASE)
#undef MM_CASE
        default: return {nullptr, nullptr, 0, 0};
    }
}

static size_t split_smem(int L, int TC) { return (size_t)3 * L * TC * sizeof(float2); }

bool split_conv_supported(int L) { return split_shape(L).k3 != nullptr; }

// Twiddle tables and shared-memory opt-in (per device, outside any capture).
cudaError_t split_conv_setup() {
    cudaError_t e = cudaSuccess;
#define MM_TW(L_)                                                                                  \
    if (e == cudaSuccess) {                                                                        \
        float2 tw[L_];                                                                             \
        for (int q = 0; q < L_; ++q) {                                                             \
            const double ang = -2.0 * kPi * (double)q / (double)L_;                                \
            tw[q] = make_float2((float)std::cos(ang), (float)std::sin(ang));                       \
        }                                                                                          \
        e = cudaMemcpyToSymbol(c_tw_##L_, tw, sizeof tw);                                          \
    }
    MM_TW(16) MM_TW(32) MM_TW(48) MM_TW(64) MM_TW(81) MM_TW(96) MM_TW(108) MM_TW(128) MM_TW(192) MM_TW(256)
    MM_TW(512)
#undef MM_TW
    for (int L : {16, 32, 48, 64, 81, 96, 108, 128, 192, 256, 512}) {
        const SplitShape s = split_shape(L);
        const int smem = (int)split_smem(L, s.TC);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(s.k3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(s.k2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    return e;
}

// 3-D middle pass along z of the spectrum [3][nz][Py][Wk] (FP32).
void split_conv_launch_3d(mm_ctx* c, void* spec, const void* khat, int nz, int Py, int Pz, int Kx, int Wk,
                          double bytes) {
    const SplitShape s = split_shape(Pz);
    SplitArgs a{};
    a.base = (float2*)spec;
    const long long plane = (long long)Py * Wk;
    a.comp_stride = (long long)nz * plane;
    a.line_stride = plane;
    a.o_stride = Wk;
    a.Wk = Wk;
    a.Kx = Kx;
    a.n_o = Py;
    const long long Ky = Py / 2 + 1, Kz = Pz / 2 + 1;
    a.n_cols = Ky * Wk;
    a.n_in = nz;
    a.khat = (const float*)khat;
    a.kc = Kz * Ky * Wk;
    a.kk = Ky * Wk;
    a.ko = Wk;
    const unsigned half_blocks = (unsigned)((a.n_cols + s.TC - 1) / s.TC);
    LaunchScope ls(c, "fft_conv", bytes);
    s.k3<<<2 * half_blocks, s.G * s.TC, split_smem(Pz, s.TC), c->stream>>>(a);
}

// 2-D middle pass along y over n_planes film planes; plane r, component q at
// spec + r * plane_stride + q * comp_stride, rows of pitch Wk.
void split_conv_launch_2d(mm_ctx* c, void* spec, const void* khat, int ny, int Py, int Kx, int Wk,
                          long long comp_stride, long long plane_stride, int n_planes, const char* name,
                          double bytes) {
    const SplitShape s = split_shape(Py);
    SplitArgs a{};
    a.base = (float2*)spec;
    a.comp_stride = comp_stride;
    a.line_stride = Wk;
    a.o_stride = plane_stride;
    a.Wk = Wk;
    a.Kx = Kx;
    a.n_o = n_planes;
    a.n_cols = (long long)n_planes * Wk;
    a.n_in = ny;
    a.khat = (const float*)khat;
    const long long Ky = Py / 2 + 1;
    a.kc = Ky * Wk;
    a.kk = Wk;
    a.ko = 0;
    LaunchScope ls(c, name, bytes);
    s.k2<<<(unsigned)((a.n_cols + s.TC - 1) / s.TC), s.G * s.TC, split_smem(Py, s.TC), c->stream>>>(a);
}

}  // namespace mm
