// Runtime-planned in-shared-memory FFT (any length 2^a 3^b): the generic
// path behind the compile-time specialised one in fft_ct.cuh.
#pragma once

#include "common.cuh"

namespace mm {

// ---------------------------------------------------------------------------
// FFT plan and in-shared-memory Stockham passes
// ---------------------------------------------------------------------------
constexpr int kMaxPasses = 16;
constexpr int kMaxV = 24;   // complex values held in registers per thread per pass

struct Plan {
    int L;
    int npass;
    int radix[kMaxPasses];
};

inline bool make_plan(int L, Plan* p) {
    p->L = L;
    p->npass = 0;
    int n = L;
    while (n % 4 == 0) { p->radix[p->npass++] = 4; n /= 4; }
    while (n % 2 == 0) { p->radix[p->npass++] = 2; n /= 2; }
    while (n % 3 == 0) { p->radix[p->npass++] = 3; n /= 3; }
    return n == 1 && p->npass <= kMaxPasses;
}

// smallest 2^a 3^b >= n (even when want_even)
inline int nice_length(int n, bool want_even) {
    int best = 1 << 30;
    for (long long p2 = 1; p2 < (1LL << 31); p2 *= 2)
        for (long long p3 = p2; p3 < (1LL << 31); p3 *= 3) {
            if (p3 >= n && p3 < best && (!want_even || p3 % 2 == 0)) best = (int)p3;
            if (p3 >= n) break;
        }
    return best;
}

template <typename T, int DIR, int R>
__device__ __forceinline__ void dft(cplx<T>* v) {
    if (R == 2) {
        cplx<T> a = v[0], b = v[1];
        v[0] = cadd<T>(a, b);
        v[1] = csub<T>(a, b);
    } else if (R == 4) {
        cplx<T> a0 = cadd<T>(v[0], v[2]), a1 = csub<T>(v[0], v[2]);
        cplx<T> a2 = cadd<T>(v[1], v[3]), a3 = mul_mi<T, DIR>(csub<T>(v[1], v[3]));
        v[0] = cadd<T>(a0, a2);
        v[2] = csub<T>(a0, a2);
        v[1] = cadd<T>(a1, a3);
        v[3] = csub<T>(a1, a3);
    } else {  // R == 3
        const T s3 = (T)0.86602540378443864676;
        cplx<T> t1 = cadd<T>(v[1], v[2]);
        cplx<T> t2 = csub<T>(v[0], cscale<T>(t1, (T)0.5));
        cplx<T> t3 = cscale<T>(mul_mi<T, DIR>(csub<T>(v[1], v[2])), s3);
        v[0] = cadd<T>(v[0], t1);
        v[1] = cadd<T>(t2, t3);
        v[2] = csub<T>(t2, t3);
    }
}

// One in-place Stockham pass over nl lines of length L stored at `pitch`
// (complex elements) in shared memory.  Every thread first loads all the
// butterflies it owns into registers, the block synchronises, then the
// results are written to their autosorted positions.  Inputs at index
// >= nin are zero (pruned, only meaningful on the first pass).
template <typename T, int DIR, int R>
__device__ void stockham_pass(cplx<T>* sm, int nl, int pitch, int L, int Ns, int nin,
                              const cplx<T>* __restrict__ tw, int tw_stride) {
    constexpr int MAXB = kMaxV / R;
    const int nb = L / R;
    const int total = nl * nb;
    cplx<T> v[MAXB][R];
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int b = threadIdx.x + i * blockDim.x;
        if (b < total) {
            const int l = b / nb, j = b - l * nb;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int idx = j + t * nb;
                v[i][t] = idx < nin ? sm[l * pitch + idx] : mkc<T>(0, 0);
            }
        }
    }
    __syncthreads();
    const int span = L / (Ns * R);
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int b = threadIdx.x + i * blockDim.x;
        if (b < total) {
            const int l = b / nb, j = b - l * nb;
            const int k = j % Ns;
            if (Ns > 1) {
#pragma unroll
                for (int t = 1; t < R; ++t) {
                    cplx<T> w = __ldg(&tw[(t * k * span) * tw_stride]);
                    v[i][t] = DIR > 0 ? cmul<T>(v[i][t], w) : cmulc<T>(v[i][t], w);
                }
            }
            dft<T, DIR, R>(v[i]);
            const int dst = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int t = 0; t < R; ++t) sm[l * pitch + dst + t * Ns] = v[i][t];
        }
    }
    __syncthreads();
}

// Full FFT of nl lines; twiddle table tw holds exp(-2 pi i q / (L*tw_stride)).
template <typename T, int DIR>
__device__ void fft_lines(cplx<T>* sm, int nl, int pitch, const Plan& p, int nin,
                          const cplx<T>* __restrict__ tw, int tw_stride) {
    int Ns = 1;
    for (int s = 0; s < p.npass; ++s) {
        const int r = p.radix[s];
        const int ni = s == 0 ? nin : p.L;
        if (r == 4) stockham_pass<T, DIR, 4>(sm, nl, pitch, p.L, Ns, ni, tw, tw_stride);
        else if (r == 2) stockham_pass<T, DIR, 2>(sm, nl, pitch, p.L, Ns, ni, tw, tw_stride);
        else stockham_pass<T, DIR, 3>(sm, nl, pitch, p.L, Ns, ni, tw, tw_stride);
        Ns *= r;
    }
}

}  // namespace mm
