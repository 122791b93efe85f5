// Device-side helpers shared by the kernels of libmm: SI constants, complex
// and 3-vector arithmetic in the working precision, warp reductions, and
// the compensated (Neumaier) FP64 accumulator used by the observables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mm {

// SI constants (gamma0 in rad/(s T): the mumax3 value, which the paper says
// its conventions follow).
constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4e-7 * kPi;
constexpr double kGamma0 = 1.7595e11;
constexpr double kKB = 1.380649e-23;
constexpr double kHbar = 1.054571817e-34;
constexpr double kQe = 1.602176634e-19;
constexpr double kMuB = 9.2740100783e-24;

template <typename T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename T> using cplx = typename cvec<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mkc(T x, T y) { cplx<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
    return mkc<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return mkc<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return mkc<T>(a.x * s, a.y * s); }
// multiply by -i (forward) / +i (inverse)
template <typename T, int DIR> __device__ __forceinline__ cplx<T> mul_mi(cplx<T> a) {
    return DIR > 0 ? mkc<T>(a.y, -a.x) : mkc<T>(-a.y, a.x);
}

template <typename T> struct v3 { T x, y, z; };
template <typename T> __device__ __forceinline__ v3<T> mk3(T x, T y, T z) { v3<T> r; r.x = x; r.y = y; r.z = z; return r; }
template <typename T> __device__ __forceinline__ v3<T> operator+(v3<T> a, v3<T> b) { return mk3<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <typename T> __device__ __forceinline__ v3<T> operator-(v3<T> a, v3<T> b) { return mk3<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <typename T> __device__ __forceinline__ v3<T> operator*(T s, v3<T> a) { return mk3<T>(s * a.x, s * a.y, s * a.z); }
template <typename T> __device__ __forceinline__ T dot(v3<T> a, v3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T> __device__ __forceinline__ v3<T> cross(v3<T> a, v3<T> b) {
    return mk3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Neumaier-compensated FP64 sum: value = s + c.
struct CompSum {
    double s, c;
    __device__ __forceinline__ void add(double v) {
        double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ void add(const CompSum& o) { add(o.s); add(o.c); }
};

__device__ __forceinline__ CompSum warp_sum(CompSum v) {
    for (int o = 16; o > 0; o >>= 1) {
        CompSum w;
        w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
        w.c = __shfl_xor_sync(0xffffffffu, v.c, o);
        v.add(w);
    }
    return v;
}

// Non-negative floating-point atomic max through the integer ordering of
// IEEE bit patterns (valid for values >= 0; a positive NaN would order above
// +inf, but warp_max's fmax drops NaN operands before it gets here, so
// callers that must see a NaN map it to +inf themselves).
__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
    atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace mm
