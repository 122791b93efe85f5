// FFT building blocks that keep data in registers between global memory and
// the transform, used by the FP32 demag passes of 3-D grids:
//  * reg_dif / reg_dit: a whole power-of-two line in one thread's registers.
//    The forward transform (decimation in frequency) leaves the spectrum in
//    bit-reversed order and the inverse (decimation in time) takes it back
//    in that order, so a pointwise product between them needs no reordering.
//  * cd_pass: one Stockham pass over TK interleaved columns held in shared
//    memory as [index][column]; its first pass may read straight from global
//    memory and its last pass may write straight to global memory.
#pragma once

#include "common.cuh"
#include "fft_ct.cuh"

namespace mm {

__host__ __device__ constexpr int ilog2_c(int n) {
    int b = 0;
    while ((1 << b) < n) ++b;
    return b;
}
__host__ __device__ constexpr int bitrev_c(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b)
        if ((i >> b) & 1) r |= 1 << (bits - 1 - b);
    return r;
}

// exp(-2 pi i q / 32), q < 32, in constant memory (filled by the demag
// setup of the including translation unit): with a compile-time index it is
// read as an instruction operand.
static __constant__ float2 c_tw32[32];

// Multiply by the twiddle tw[q] = exp(-2 pi i q / L) (DIR > 0) or its
// conjugate; q is a compile-time constant after unrolling, so the exact
// cases q = 0 and q = L/4 (a swap and a sign) cost no multiplication.
// tw == nullptr (FP32, L dividing 32): the constant table c_tw32.
template <typename T, int DIR, int L, int TS = 1>
__device__ __forceinline__ cplx<T> twiddle_mul(cplx<T> v, int q, const cplx<T>* tw) {
    if (q == 0) return v;
    if (4 * q == L) return mul_mi<T, DIR>(v);
    cplx<T> w;
    if constexpr (sizeof(T) == 4 && 32 % (L * TS) == 0) {
        if (tw == nullptr) {
            const float2 c = c_tw32[q * TS * (32 / (L * TS))];
            w = mkc<T>(c.x, c.y);
        } else {
            w = tw[q * TS];
        }
    } else {
        w = tw[q * TS];
    }
    return DIR > 0 ? cmul<T>(v, w) : cmulc<T>(v, w);
}

// In-register forward DFT of length L (a power of two), natural order in,
// bit-reversed order out.  tw[q] = exp(-2 pi i q / L).  One template level
// per stage so that every register index is a compile-time constant.
// HALF: the upper half of the input is known to be zero (a zero-padded
// line), which removes the first stage's additions.
// TS: stride of tw (the table may belong to a length TS * L).
template <typename T, int L, bool HALF = false, int TS = 1, int S = 0>
__device__ __forceinline__ void reg_dif(cplx<T> (&v)[L], const cplx<T>* tw) {
    if constexpr ((L >> S) >= 2) {
        constexpr int len = L >> S, h = len >> 1;
#pragma unroll
        for (int q = 0; q < L / 2; ++q) {
            const int b = (q / h) * len, j = q % h;
            const cplx<T> u = v[b + j];
            if (HALF && S == 0) {
                v[b + j + h] = twiddle_mul<T, 1, L, TS>(u, j * (L / len), tw);
            } else {
                const cplx<T> t = v[b + j + h];
                v[b + j] = cadd<T>(u, t);
                v[b + j + h] = twiddle_mul<T, 1, L, TS>(csub<T>(u, t), j * (L / len), tw);
            }
        }
        reg_dif<T, L, HALF, TS, S + 1>(v, tw);
    }
}

// In-register inverse DFT (unnormalised, exp(+2 pi i k n / L)), bit-reversed
// order in, natural order out.  HALF: only the lower half of the output is
// used (the last stage skips the upper half).
template <typename T, int L, bool HALF = false, int TS = 1, int S = 0>
__device__ __forceinline__ void reg_dit_inv(cplx<T> (&v)[L], const cplx<T>* tw) {
    if constexpr ((2 << S) <= L) {
        constexpr int len = 2 << S, h = len >> 1;
        constexpr bool last = (2 << S) == L;
#pragma unroll
        for (int q = 0; q < L / 2; ++q) {
            const int b = (q / h) * len, j = q % h;
            const cplx<T> u = v[b + j];
            const cplx<T> t = twiddle_mul<T, -1, L, TS>(v[b + j + h], j * (L / len), tw);
            v[b + j] = cadd<T>(u, t);
            if (!(HALF && last)) v[b + j + h] = csub<T>(u, t);
        }
        reg_dit_inv<T, L, HALF, TS, S + 1>(v, tw);
    }
}

// Where a column pass reads its input from / writes its output to.
enum { CD_SMEM = 0, CD_GLOBAL = 1 };

// One Stockham pass (radix R, current sub-length NS) over TK columns of
// length L.  Butterfly b of NT threads: column l = b % TK, butterfly j =
// b / TK, so a warp touches consecutive columns (one contiguous row segment
// in global memory, consecutive words in shared memory).  Shared layout:
// element idx of column l at sm[idx * TK + l].  Global: element idx of
// column l at g[l] + idx * gstride (g[l] < 0: the column is absent).
// Reads at idx >= nin are zero; global writes at idx >= nout are dropped.
// gin and gout may be the same buffer: every element a CTA writes was read
// by the same CTA in its first pass.
template <typename T, int DIR, int L, int R, int NS, int NT, int TK, int SRC, int DST>
__device__ __forceinline__ void cd_pass(cplx<T>* sm, const cplx<T>* gin, cplx<T>* gout, long long gcol,
                                        long long gstride, int nin, int nout, const cplx<T>* __restrict__ tw) {
    constexpr int NB = L / R;
    constexpr int SPAN = L / (NS * R);
    constexpr int TOT = TK * NB;                 // butterflies in the pass
    constexpr int NBT = (TOT + NT - 1) / NT;     // per thread
    static_assert(NT % TK == 0, "a thread keeps one column");
    const int l = threadIdx.x % TK;
    cplx<T> v[NBT][R];
#pragma unroll
    for (int i = 0; i < NBT; ++i) {
        const int b = threadIdx.x + i * NT;
        if (TOT % NT == 0 || b < TOT) {
            const int j = b / TK;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int idx = j + t * NB;
                if constexpr (SRC == CD_GLOBAL) {
                    v[i][t] = (gcol >= 0 && idx < nin) ? gin[gcol + idx * gstride] : mkc<T>(0, 0);
                } else {
                    v[i][t] = sm[idx * TK + l];
                }
            }
        }
    }
    if constexpr (SRC == CD_SMEM && DST == CD_SMEM) __syncthreads();
#pragma unroll
    for (int i = 0; i < NBT; ++i) {
        const int b = threadIdx.x + i * NT;
        if (TOT % NT != 0 && b >= TOT) continue;
        const int j = b / TK;
        const int k = j % NS;
        if constexpr (NS > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                const cplx<T> w = __ldg(&tw[t * k * SPAN]);
                v[i][t] = DIR > 0 ? cmul<T>(v[i][t], w) : cmulc<T>(v[i][t], w);
            }
        }
        dft_ct<T, DIR, R>(v[i]);
        const int dst = (j / NS) * NS * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int idx = dst + t * NS;
            if constexpr (DST == CD_GLOBAL) {
                if (gcol >= 0 && idx < nout) gout[gcol + idx * gstride] = v[i][t];
            } else {
                sm[idx * TK + l] = v[i][t];
            }
        }
    }
    if constexpr (DST == CD_SMEM) __syncthreads();
}

// Whole column transform: global -> registers -> (shared passes) -> global.
template <typename T, int DIR, int L, int NT, int TK, int P = 0>
__device__ __forceinline__ void cd_fft(cplx<T>* sm, const cplx<T>* gin, cplx<T>* gout,
                                       long long gcol, long long gstride, int nin, int nout,
                                       const cplx<T>* __restrict__ tw) {
    constexpr int NP = ct_npass(L);
    if constexpr (P < NP) {
        constexpr int R = ct_radix(L, P);
        constexpr int NS = ct_ns(L, P);
        constexpr int SRC = P == 0 ? CD_GLOBAL : CD_SMEM;
        constexpr int DST = P == NP - 1 ? CD_GLOBAL : CD_SMEM;
        cd_pass<T, DIR, L, R, NS, NT, TK, SRC, DST>(sm, gin, gout, gcol, gstride, nin, nout, tw);
        cd_fft<T, DIR, L, NT, TK, P + 1>(sm, gin, gout, gcol, gstride, nin, nout, tw);
    }
}

// ---------------------------------------------------------------------------
// One line per warp, or per group of GW lanes when the line is short (a
// warp then transforms 32 / GW lines at once, so that the passes' NB
// butterflies fill its lanes).  The line lives in warp-private shared memory
// with one pad slot every 8 entries (index i at wpad(i)), which keeps the
// stride-R writes of the early Stockham passes free of bank conflicts;
// passes are separated by __syncwarp only, so warps never wait on each
// other.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int wpad(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int wline(int L) { return wpad(L) + 1; }

// lanes per line: the smallest power of two that covers the narrowest pass
// of the plan (at most 32)
__host__ __device__ constexpr int warp_group(int L) {
    int nb = L;
    for (int p = 0; p < ct_npass(L); ++p) nb = L / ct_radix(L, p) < nb ? L / ct_radix(L, p) : nb;
    int g = 1;
    while (g < nb && g < 32) g *= 2;
    return g;
}

template <typename T, int DIR, int L, int R, int NS, int GW = 32, typename Load, typename Store>
__device__ __forceinline__ void warp_pass(const cplx<T>* __restrict__ tw, int tws, Load load, Store store) {
    constexpr int NB = L / R;
    constexpr int SPAN = L / (NS * R);
    constexpr int NBL = (NB + GW - 1) / GW;
    const int lane = threadIdx.x & (GW - 1);
    cplx<T> v[NBL][R];
#pragma unroll
    for (int i = 0; i < NBL; ++i) {
        const int j = lane + GW * i;
        if (NB % GW == 0 || j < NB) {
#pragma unroll
            for (int t = 0; t < R; ++t) v[i][t] = load(j + t * NB);
        }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NBL; ++i) {
        const int j = lane + GW * i;
        if (NB % GW != 0 && j >= NB) continue;
        const int k = j % NS;
        if constexpr (NS > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                const cplx<T> w = __ldg(&tw[(t * k * SPAN) * tws]);
                v[i][t] = DIR > 0 ? cmul<T>(v[i][t], w) : cmulc<T>(v[i][t], w);
            }
        }
        dft_ct<T, DIR, R>(v[i]);
        const int dst = (j / NS) * NS * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) store(dst + t * NS, v[i][t]);
    }
    __syncwarp();
}

// Passes P .. PEND-1 of a warp's (or lane group's) line, all shared memory
// -> shared memory.
template <typename T, int DIR, int L, int P, int PEND, int GW = 32>
__device__ __forceinline__ void warp_fft_smem(cplx<T>* sm, const cplx<T>* __restrict__ tw, int tws) {
    if constexpr (P < PEND) {
        constexpr int R = ct_radix(L, P);
        constexpr int NS = ct_ns(L, P);
        warp_pass<T, DIR, L, R, NS, GW>(tw, tws, [&](int i) { return sm[wpad(i)]; },
                                        [&](int i, cplx<T> v) { sm[wpad(i)] = v; });
        warp_fft_smem<T, DIR, L, P + 1, PEND, GW>(sm, tw, tws);
    }
}

// Inverse real transform of one row on one warp: the half spectrum X[0..M]
// (M = LT, global memory) to 2M real values, of which the caller's store
// keeps what it needs: store(n, v) receives the pair (2n, 2n+1).  The
// rebuild Z'[k] = (X[k] + conj X[M-k]) + i (X[k] - conj X[M-k]) conj(W^k)
// feeds the first pass; the last pass goes straight to the store.  sm is
// the warp's line of wline(LT) values; tw = exp(-2 pi i q / 2M).
template <int LT, int GW = 32, typename Store>
__device__ __forceinline__ void warp_c2r(const float2* __restrict__ X, const float2* __restrict__ tw, float2* sm,
                                         Store store) {
    constexpr int NP = ct_npass(LT), M = LT;
    static_assert(NP >= 2, "first and last pass must differ");
    auto load_rebuild = [&](int k) {
        const float2 xk = X[k];
        const float2 xc = cconj<float>(X[M - k]);
        const float2 E = cadd<float>(xk, xc);
        const float2 O = cmulc<float>(csub<float>(xk, xc), __ldg(&tw[k]));
        return cadd<float>(E, mul_mi<float, -1>(O));
    };
    auto to_smem = [&](int i, float2 v) { sm[wpad(i)] = v; };
    warp_pass<float, -1, LT, ct_radix(LT, 0), 1, GW>(tw, 2, load_rebuild, to_smem);
    warp_fft_smem<float, -1, LT, 1, NP - 1, GW>(sm, tw, 2);
    warp_pass<float, -1, LT, ct_radix(LT, NP - 1), ct_ns(LT, NP - 1), GW>(tw, 2,
                                                                          [&](int i) { return sm[wpad(i)]; }, store);
}

// The same inverse real transform with the half spectrum already in the
// warp's line: sm[0 .. M] holds X[k] at plain index k.  The first pass reads
// every value it needs before its __syncwarp and writes its outputs to the
// padded positions afterwards, so it runs in place.
template <int LT, typename Store>
__device__ __forceinline__ void warp_c2r_inplace(float2* sm, const float2* __restrict__ tw, Store store) {
    constexpr int NP = ct_npass(LT), M = LT;
    static_assert(NP >= 2, "first and last pass must differ");
    auto load_rebuild = [&](int k) {
        const float2 xk = sm[k];
        const float2 xc = cconj<float>(sm[M - k]);
        const float2 E = cadd<float>(xk, xc);
        const float2 O = cmulc<float>(csub<float>(xk, xc), __ldg(&tw[k]));
        return cadd<float>(E, mul_mi<float, -1>(O));
    };
    auto to_smem = [&](int i, float2 v) { sm[wpad(i)] = v; };
    warp_pass<float, -1, LT, ct_radix(LT, 0), 1>(tw, 2, load_rebuild, to_smem);
    warp_fft_smem<float, -1, LT, 1, NP - 1>(sm, tw, 2);
    warp_pass<float, -1, LT, ct_radix(LT, NP - 1), ct_ns(LT, NP - 1)>(tw, 2, [&](int i) { return sm[wpad(i)]; },
                                                                      store);
}

}  // namespace mm
