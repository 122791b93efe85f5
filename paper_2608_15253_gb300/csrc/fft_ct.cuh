// Compile-time specialised in-shared-memory FFT: the length L, every radix,
// every Stockham stride and the line pitch are template constants, so the
// butterfly index arithmetic reduces to shifts, masks and constant
// multiplies.  Radix order: 8s first, then one 4 or 2, then 3s.
#pragma once

#include "common.cuh"

namespace mm {

__host__ __device__ constexpr int ct_radix(int L, int p) {
    int n = L;
    for (int q = 0;; ++q) {
        int r = n % 8 == 0 ? 8 : n % 4 == 0 ? 4 : n % 2 == 0 ? 2 : n % 3 == 0 ? 3 : 1;
        if (q == p) return r;
        n /= r;
    }
}
__host__ __device__ constexpr int ct_npass(int L) {
    int n = L, p = 0;
    while (n > 1) { n /= ct_radix(L, p); ++p; }
    return p;
}
__host__ __device__ constexpr int ct_ns(int L, int p) {
    int ns = 1;
    for (int q = 0; q < p; ++q) ns *= ct_radix(L, q);
    return ns;
}

template <typename T, int DIR>
__device__ __forceinline__ void dft4v(cplx<T>& a, cplx<T>& b, cplx<T>& c, cplx<T>& d) {
    const cplx<T> a0 = cadd<T>(a, c), a1 = csub<T>(a, c);
    const cplx<T> a2 = cadd<T>(b, d), a3 = mul_mi<T, DIR>(csub<T>(b, d));
    a = cadd<T>(a0, a2);
    c = csub<T>(a0, a2);
    b = cadd<T>(a1, a3);
    d = csub<T>(a1, a3);
}

template <typename T, int DIR, int R>
__device__ __forceinline__ void dft_ct(cplx<T>* v) {
    if constexpr (R == 2) {
        const cplx<T> a = v[0], b = v[1];
        v[0] = cadd<T>(a, b);
        v[1] = csub<T>(a, b);
    } else if constexpr (R == 4) {
        dft4v<T, DIR>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 3) {
        const T s3 = (T)0.86602540378443864676;
        const cplx<T> t1 = cadd<T>(v[1], v[2]);
        const cplx<T> t2 = csub<T>(v[0], cscale<T>(t1, (T)0.5));
        const cplx<T> t3 = cscale<T>(mul_mi<T, DIR>(csub<T>(v[1], v[2])), s3);
        v[0] = cadd<T>(v[0], t1);
        v[1] = cadd<T>(t2, t3);
        v[2] = csub<T>(t2, t3);
    } else {  // R == 8: radix-2 split into two DFT-4s
        const T h = (T)0.70710678118654752440;
        cplx<T> b0 = cadd<T>(v[0], v[4]), c0 = csub<T>(v[0], v[4]);
        cplx<T> b1 = cadd<T>(v[1], v[5]), c1 = csub<T>(v[1], v[5]);
        cplx<T> b2 = cadd<T>(v[2], v[6]), c2 = mul_mi<T, DIR>(csub<T>(v[2], v[6]));
        cplx<T> b3 = cadd<T>(v[3], v[7]), c3 = csub<T>(v[3], v[7]);
        // c1 *= W8, c3 *= W8^3 (W8 = exp(-+ i pi/4))
        c1 = DIR > 0 ? mkc<T>(h * (c1.x + c1.y), h * (c1.y - c1.x)) : mkc<T>(h * (c1.x - c1.y), h * (c1.y + c1.x));
        c3 = DIR > 0 ? mkc<T>(h * (c3.y - c3.x), -h * (c3.x + c3.y)) : mkc<T>(-h * (c3.x + c3.y), h * (c3.x - c3.y));
        dft4v<T, DIR>(b0, b1, b2, b3);
        dft4v<T, DIR>(c0, c1, c2, c3);
        v[0] = b0; v[2] = b1; v[4] = b2; v[6] = b3;
        v[1] = c0; v[3] = c1; v[5] = c2; v[7] = c3;
    }
}

// One in-place pass over nl lines of length L at pitch LP.  NT threads,
// each holding up to MAXV complex values in registers across the barrier.
template <typename T, int DIR, int L, int LP, int R, int NS, int NT, int MAXV>
__device__ __forceinline__ void ct_pass(cplx<T>* sm, int nl, int nin, const cplx<T>* __restrict__ tw, int tws) {
    constexpr int NB = L / R;
    constexpr int MAXB = MAXV / R;
    constexpr int SPAN = L / (NS * R);
    const int total = nl * NB;
    cplx<T> v[MAXB][R];
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < total) {
            const int l = b / NB, j = b % NB;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int idx = j + t * NB;
                v[i][t] = (NS > 1 || idx < nin) ? sm[l * LP + idx] : mkc<T>(0, 0);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXB; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < total) {
            const int l = b / NB, j = b % NB;
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
            for (int t = 0; t < R; ++t) sm[l * LP + dst + t * NS] = v[i][t];
        }
    }
    __syncthreads();
}

// Passes P .. PEND-1 (PEND = -1: through the last pass).
template <typename T, int DIR, int L, int LP, int NT, int MAXV, int P = 0, int PEND = -1>
__device__ __forceinline__ void ct_fft(cplx<T>* sm, int nl, int nin, const cplx<T>* __restrict__ tw, int tws) {
    if constexpr (P < (PEND < 0 ? ct_npass(L) : PEND)) {
        constexpr int R = ct_radix(L, P);
        constexpr int NS = ct_ns(L, P);
        ct_pass<T, DIR, L, LP, R, NS, NT, (MAXV / R) * R>(sm, nl, P == 0 ? nin : L, tw, tws);
        ct_fft<T, DIR, L, LP, NT, MAXV, P + 1, PEND>(sm, nl, nin, tw, tws);
    }
}

}  // namespace mm
