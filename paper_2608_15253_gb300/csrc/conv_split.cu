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

// Packed two-lane FP32 arithmetic (one instruction for both parts of a
// complex value).  `z` flags an operand known to be zero at compile time
// (after unrolling): the operation then folds away, which the packed
// builtins would not do by themselves.
__device__ __forceinline__ float2 add2(float2 a, float2 b, bool zb = false) {
    return zb ? a : __fadd2_rn(a, b);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b, bool zb = false) {
    return zb ? a : __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
// a + (-i)^DIR t and a - (-i)^DIR t (the rotation is a swap, so scalar)
template <int DIR> __device__ __forceinline__ float2 add_rot(float2 a, float2 t) {
    return DIR > 0 ? make_float2(a.x + t.y, a.y - t.x) : make_float2(a.x - t.y, a.y + t.x);
}
template <int DIR> __device__ __forceinline__ float2 sub_rot(float2 a, float2 t) {
    return DIR > 0 ? make_float2(a.x - t.y, a.y + t.x) : make_float2(a.x + t.y, a.y - t.x);
}

// 4-point DFT of (a, b, c, d); zc / zd: c / d known zero
template <int DIR>
__device__ __forceinline__ void dft4x(float2& a, float2& b, float2& c, float2& d, bool zc, bool zd) {
    const float2 a0 = add2(a, c, zc), a1 = sub2(a, c, zc);
    const float2 a2 = add2(b, d, zd), t = sub2(b, d, zd);
    a = add2(a0, a2);
    c = sub2(a0, a2);
    b = add_rot<DIR>(a1, t);
    d = sub_rot<DIR>(a1, t);
}

// R-point DFT in place; zu[t]: input t known zero (only the upper half of a
// radix-2/4/8 group is ever flagged: the zero-padded half of a line)
template <int DIR, int R>
__device__ __forceinline__ void dftx(float2* v, const bool* zu) {
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = add2(a, b, zu[1]);
        v[1] = sub2(a, b, zu[1]);
    } else if constexpr (R == 4) {
        dft4x<DIR>(v[0], v[1], v[2], v[3], zu[2], zu[3]);
    } else if constexpr (R == 8) {
        const float h = 0.70710678118654752440f;
        float2 b0 = add2(v[0], v[4], zu[4]), c0 = sub2(v[0], v[4], zu[4]);
        float2 b1 = add2(v[1], v[5], zu[5]), c1 = sub2(v[1], v[5], zu[5]);
        float2 b2 = add2(v[2], v[6], zu[6]), t2 = sub2(v[2], v[6], zu[6]);   // c2 = (-i)^DIR t2
        float2 b3 = add2(v[3], v[7], zu[7]), c3 = sub2(v[3], v[7], zu[7]);
        // c1 *= W8, c3 *= W8^3 (W8 = exp(-+ i pi/4))
        c1 = DIR > 0 ? make_float2(c1.x + c1.y, c1.y - c1.x) : make_float2(c1.x - c1.y, c1.y + c1.x);
        c3 = DIR > 0 ? make_float2(c3.y - c3.x, -(c3.x + c3.y)) : make_float2(-(c3.x + c3.y), c3.x - c3.y);
        c1 = __fmul2_rn(c1, make_float2(h, h));
        c3 = __fmul2_rn(c3, make_float2(h, h));
        dft4x<DIR>(b0, b1, b2, b3, false, false);
        // 4-point DFT of (c0, c1, (-i)^DIR t2, c3)
        const float2 a0 = add_rot<DIR>(c0, t2), a1 = sub_rot<DIR>(c0, t2);
        const float2 a2 = add2(c1, c3), t = sub2(c1, c3);
        v[0] = b0; v[2] = b1; v[4] = b2; v[6] = b3;
        v[1] = add2(a0, a2);
        v[5] = sub2(a0, a2);
        v[3] = add_rot<DIR>(a1, t);
        v[7] = sub_rot<DIR>(a1, t);
    } else {  // R == 3: scalar arithmetic (its zero inputs fold by themselves)
        dft_ct<float, DIR, 3>(v);
    }
}

// In-register DFT of length N (natural order in and out), mixed radix
// 8/4/2/3 Stockham passes with every index a compile-time constant; the
// twiddles W_N^m are taken from the length-L table (N divides L).  Inputs
// at index >= NZ are known zeros (the zero-padded part of a line).
template <int DIR, int N, int L, int NZ = N, int P = 0>
__device__ __forceinline__ void rfft(float2 (&v)[N]) {
    if constexpr (P < ct_npass(N)) {
        constexpr int R = ct_radix(N, P), NS = ct_ns(N, P), NB = N / R, SPAN = N / (NS * R);
        float2 w[N];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            float2 u[R];
            bool zu[R];
#pragma unroll
            for (int t = 0; t < R; ++t) {
                u[t] = v[j + t * NB];
                zu[t] = P == 0 && j + t * NB >= NZ;
            }
            const int k = j % NS;
            if constexpr (NS > 1) {
#pragma unroll
                for (int t = 1; t < R; ++t) u[t] = twq<DIR, L>(u[t], (t * k * SPAN) * (L / N));
            }
            dftx<DIR, R>(u, zu);
            const int dst = (j / NS) * NS * R + k;
#pragma unroll
            for (int t = 0; t < R; ++t) w[dst + t * NS] = u[t];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = w[i];
        rfft<DIR, N, L, N, P + 1>(v);
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
//
// Shared memory: the exchange buffer [3][G][Q][TC] complex, then the CTA's
// tensor tile [NC][L/2+1][TC] real.  The tile is fetched with cp.async at
// kernel start (16-byte pieces: four consecutive columns share one tensor row
// because the row pitch Wk is a multiple of 4), so its latency hides behind
// phase 1 and phase 2 reads the tensor from shared memory.
template <int L, bool THREE_D> constexpr int split_nc() { return THREE_D ? 6 : 4; }

template <int L, int G, int Q, int TC, bool THREE_D>
constexpr size_t split_smem_bytes() {
    return (size_t)3 * L * TC * sizeof(float2) + (size_t)split_nc<L, THREE_D>() * (L / 2 + 1) * TC * sizeof(float);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One phase-2 item (k1, column): the G line-part values of every component,
// G-point DFT, H^ = K^ M^ at kz = k1 + Q k2 (k2 < G), inverse DFT, stored
// back in place.  SO is the parity sign of the other axis (3-D: -1 for the
// mirrored ky' = Py - ky).  The fold of kz into the stored half range is a
// compile-time constant except on the one k2 where it depends on k1.
template <int L, int G, int Q, int TC, bool THREE_D, int SO>
__device__ __forceinline__ void split_item(float2* sm, const float* sk, int k1, int col) {
    constexpr int KZ = L / 2 + 1;
    float2 m[3][G];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int u = 0; u < G; ++u) m[c][u] = sm[((c * G + u) * Q + k1) * TC + col];
#pragma unroll
    for (int c = 0; c < 3; ++c) rfft<1, G, L>(m[c]);
#pragma unroll
    for (int k2 = 0; k2 < G; ++k2) {
        const int lo = 2 * Q * k2;                   // 2 kz - 2 k1, 0 <= k1 < Q
        const bool fold = lo > L ? true : (lo + 2 * (Q - 1) <= L ? false : 2 * k1 + lo > L);
        const int kz = k1 + Q * k2;
        const int kzf = fold ? L - kz : kz;
        const float st = fold ? -1.f : 1.f;
        const float* Kp = sk + kzf * TC + col;
        const float kxx = Kp[0], kyy = Kp[KZ * TC], kzz = Kp[2 * KZ * TC];
        float kxy, kxz = 0.f, kyz = 0.f;
        if constexpr (THREE_D) {
            kxy = Kp[3 * KZ * TC] * (float)SO;
            kxz = Kp[4 * KZ * TC] * st;
            kyz = Kp[5 * KZ * TC] * ((float)SO * st);
        } else {
            kxy = Kp[3 * KZ * TC] * st;
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

template <int L, int G, int Q, int TC, bool THREE_D>
__global__ void __launch_bounds__(G * TC, (228 * 1024) / (split_smem_bytes<L, G, Q, TC, THREE_D>() + 1024) < 1
                                              ? 1
                                              : (228 * 1024) / (split_smem_bytes<L, G, Q, TC, THREE_D>() + 1024))
    fft_conv_split_kernel(SplitArgs a) {
    static_assert(L == G * Q, "line length");
    static_assert(TC % 4 == 0, "tensor tile pieces of four columns");
    constexpr int NT = G * TC;
    constexpr int NC = split_nc<L, THREE_D>();
    constexpr int KZ = L / 2 + 1;
    constexpr int NMAX = (L + 1) / 2;                 // 2 n_in - 1 <= L
    constexpr int QIN = (NMAX + G - 1) / G;           // register slots that can hold inputs
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);                      // [3][G][Q][TC]
    float* sk = reinterpret_cast<float*>(smem_raw + (size_t)3 * L * TC * sizeof(float2));   // [NC][KZ][TC]
    const int col = threadIdx.x % TC, t = threadIdx.x / TC;

    // column of this thread
    int side = 0;
    long long pblk = (long long)blockIdx.x * TC;
    if constexpr (THREE_D) {
        side = blockIdx.x & 1;
        pblk = (long long)(blockIdx.x >> 1) * TC;
    }

    // tensor tile: piece (j, kzf, group of four columns) -> 16 bytes
    {
        constexpr int NG = TC / 4;
        for (int e = threadIdx.x; e < NC * KZ * NG; e += NT) {
            const int grp = e % NG, row = e / NG;                 // row = j * KZ + kzf
            const int j = row / KZ, kzf = row - j * KZ;
            long long pg = pblk + 4 * grp;
            if (pg >= a.n_cols) pg = 0;                          // whole group past the end: any valid row
            const int og = (int)(pg / a.Wk), kxg = (int)(pg - (long long)og * a.Wk);
            const float* src = a.khat + j * a.kc + (long long)kzf * a.kk + (THREE_D ? (long long)og * a.ko : 0) + kxg;
            cp_async16(sk + (size_t)row * TC + 4 * grp, src);
        }
    }

    const long long p = pblk + col;
    int o = (int)(p / a.Wk), kx = (int)(p - (long long)o * a.Wk);
    bool valid = p < a.n_cols && kx < a.Kx;
    int om = o;                                        // other-axis index of the data
    if constexpr (THREE_D) {
        if (side) {
            valid = valid && o != 0 && 2 * o != a.n_o;
            om = a.n_o - o;
        }
    }
    if (!valid) { om = 0; kx = 0; }
    const long long gcol = (long long)om * a.o_stride + kx;

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
            rfft<1, Q, L, QIN>(v);
#pragma unroll
            for (int k1 = 0; k1 < Q; ++k1) {
                float2 r = v[k1];
                if (G > 1 && k1 > 0) r = cmul<float>(r, twc<L>(t * k1));   // W_L^0 = 1 exactly
                sm[((c * G + t) * Q + k1) * TC + col] = r;
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // ---- phase 2: G-point DFTs across the line parts, tensor multiply, inverse
    // (the other-axis parity sign is CTA-uniform: both signs are compiled)
    if (THREE_D && side) {
#pragma unroll 1
        for (int k1 = t; k1 < Q; k1 += G) split_item<L, G, Q, TC, THREE_D, -1>(sm, sk, k1, col);
    } else {
#pragma unroll 1
        for (int k1 = t; k1 < Q; k1 += G) split_item<L, G, Q, TC, THREE_D, 1>(sm, sk, k1, col);
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
// Y passes of 3-D grids (forward: ny inputs -> Py outputs; inverse: Py
// inputs -> ny outputs) by the same four-step split, without a tensor: one
// shared-memory exchange per transform instead of a barrier per Stockham
// pass.  Columns are the flattened (component, z, kx) list, TC per CTA.
//  forward  phase 1: thread t, Q-point FFTs of x[q G + t] (zero past n_in),
//                    twiddle W_L^(t k1), to shared memory;
//           phase 2: item k1, G-point DFT over t -> X[k1 + Q k2], to global.
//  inverse  phase 1: item k1, inverse G-point DFT of H[k1 + Q k2] over k2,
//                    twiddle conj W_L^(u k1), to shared memory;
//           phase 2: thread t, inverse Q-point FFT -> y[q G + t], the first
//                    n_out rows to global.
// In place: every element a CTA writes belongs to its own columns and was
// read before the barrier.
// ---------------------------------------------------------------------------
struct ColSplitArgs {
    float2* base;          // spectrum [3][nz][Py][Wk]
    long long plane;       // Py * Wk
    int Kx, Wk;
    int ncols;             // 3 * nz * Kx
    int n_in, n_out;       // forward: ny, Py; inverse: Py, ny
};

template <int L, int G, int Q, int TC, int DIR>
__global__ void __launch_bounds__(G * TC, 2) fft_ysplit_kernel(ColSplitArgs a) {
    static_assert(L == G * Q, "line length");
    constexpr int NMAX = (L + 1) / 2;
    constexpr int QIN = (NMAX + G - 1) / G;       // forward inputs / inverse outputs per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);   // [G][Q][TC]
    const int col = threadIdx.x % TC, t = threadIdx.x / TC;
    const int p = blockIdx.x * TC + col;
    const bool valid = p < a.ncols;
    long long gcol = 0;
    if (valid) {
        const int q = p / a.Kx, kx = p - q * a.Kx;
        gcol = (long long)q * a.plane + kx;
    }
    float2* g = a.base + gcol;
    const long long W = a.Wk;
    if constexpr (DIR > 0) {
        float2 v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int n = q * G + t;
            v[q] = (q < QIN && valid && n < a.n_in) ? g[n * W] : make_float2(0.f, 0.f);
        }
        rfft<1, Q, L>(v);
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) {
            float2 r = v[k1];
            if (G > 1 && k1 > 0) r = cmul<float>(r, twc<L>(t * k1));
            sm[(t * Q + k1) * TC + col] = r;
        }
        __syncthreads();
#pragma unroll 1
        for (int k1 = t; k1 < Q; k1 += G) {
            float2 m[G];
#pragma unroll
            for (int u = 0; u < G; ++u) m[u] = sm[(u * Q + k1) * TC + col];
            rfft<1, G, L>(m);
            if (valid) {
#pragma unroll
                for (int k2 = 0; k2 < G; ++k2) g[(k1 + Q * k2) * W] = m[k2];
            }
        }
    } else {
#pragma unroll 1
        for (int k1 = t; k1 < Q; k1 += G) {
            float2 m[G];
#pragma unroll
            for (int k2 = 0; k2 < G; ++k2) m[k2] = valid ? g[(k1 + Q * k2) * W] : make_float2(0.f, 0.f);
            rfft<-1, G, L>(m);
#pragma unroll
            for (int u = 0; u < G; ++u) {
                float2 r = m[u];
                if (G > 1 && u > 0) r = cmulc<float>(r, twc<L>(u * k1));
                sm[(u * Q + k1) * TC + col] = r;
            }
        }
        __syncthreads();
        float2 v[Q];
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) v[k1] = sm[(t * Q + k1) * TC + col];
        rfft<-1, Q, L>(v);
        if (valid) {
#pragma unroll
            for (int q = 0; q < QIN; ++q) {
                const int n = q * G + t;
                if (n < a.n_out) g[n * W] = v[q];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using SplitKern = void (*)(SplitArgs);

// (L, G, Q, TC): Q = 16 register values per thread where the line allows it
// (more resident warps per shared-memory byte), TC columns per CTA so that
// G * TC is a whole number of warps.
#define MM_SPLIT_SHAPES(X) \
    X(16, 1, 16, 64) X(32, 1, 32, 64) X(48, 3, 16, 32) X(64, 4, 16, 16) X(81, 3, 27, 32) X(96, 6, 16, 16) \
    X(108, 4, 27, 16) X(128, 8, 16, 16) X(192, 12, 16, 8) X(256, 16, 16, 8) X(512, 16, 32, 4)

struct SplitShape {
    SplitKern k3, k2;   // 3-D and 2-D variants
    int G, TC;
    size_t smem3, smem2;
};

static SplitShape split_shape(int L) {
    switch (L) {
#define MM_CASE(L_, G_, Q_, TC_)                                                                              \
    case L_:                                                                                                 \
        return {fft_conv_split_kernel<L_, G_, Q_, TC_, true>, fft_conv_split_kernel<L_, G_, Q_, TC_, false>, \
                G_, TC_, split_smem_bytes<L_, G_, Q_, TC_, true>(), split_smem_bytes<L_, G_, Q_, TC_, false>()};
        MM_SPLIT_SHAPES(MM_CASE)
#undef MM_CASE
        default: return {nullptr, nullptr, 0, 0, 0, 0};
    }
}


using YSplitKern = void (*)(ColSplitArgs);
struct YSplitShape {
    YSplitKern fwd, inv;
    int G, TC;
};

// (L, G, Q, TC) of the Y passes: G * TC = 256 threads, exchange L TC values.
// At L = 1024 the shared-memory Stockham kernel (fft_y_direct_kernel) was
// measured faster (383 against 411 us on 512x512x64): only 512 splits.
#define MM_YSPLIT_SHAPES(X) X(512, 16, 32, 16)

static YSplitShape ysplit_shape(int L) {
    switch (L) {
#define MM_CASE(L_, G_, Q_, TC_) \
    case L_: return {fft_ysplit_kernel<L_, G_, Q_, TC_, 1>, fft_ysplit_kernel<L_, G_, Q_, TC_, -1>, G_, TC_};
        MM_YSPLIT_SHAPES(MM_CASE)
#undef MM_CASE
        default: return {nullptr, nullptr, 0, 0};
    }
}

bool ysplit_supported(int L) { return ysplit_shape(L).fwd != nullptr; }

void ysplit_launch(mm_ctx* c, bool fwd, void* spec, int nz, int Py, int Kx, int Wk, int n_in, int n_out,
                   const char* name, double bytes) {
    const YSplitShape s = ysplit_shape(Py);
    ColSplitArgs a{};
    a.base = (float2*)spec;
    a.plane = (long long)Py * Wk;
    a.Kx = Kx;
    a.Wk = Wk;
    a.ncols = 3 * nz * Kx;
    a.n_in = n_in;
    a.n_out = n_out;
    const size_t smem = (size_t)Py * s.TC * sizeof(float2);
    LaunchScope ls(c, name, bytes);
    (fwd ? s.fwd : s.inv)<<<(unsigned)((a.ncols + s.TC - 1) / s.TC), s.G * s.TC, smem, c->stream>>>(a);
}

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
        if (e == cudaSuccess) e = cudaFuncSetAttribute(s.k3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem3);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(s.k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem2);
    }
    for (int L : {512}) {
        const YSplitShape s = ysplit_shape(L);
        const int smem = (int)((size_t)L * s.TC * sizeof(float2));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(s.fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(s.inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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
    s.k3<<<2 * half_blocks, s.G * s.TC, s.smem3, c->stream>>>(a);
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
    s.k2<<<(unsigned)((a.n_cols + s.TC - 1) / s.TC), s.G * s.TC, s.smem2, c->stream>>>(a);
}

}  // namespace mm
