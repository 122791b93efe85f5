// Integrators (Methods, "Integrators"): Dormand-Prince RK45 (adaptive,
// first-same-as-last) with the step controller on the device, and Heun
// (Stratonovich: one thermal draw per step, shared by predictor and
// corrector).  Every kernel of an attempt reads the device state (dt,
// active flag), so chunks of attempts are captured once in a CUDA graph and
// replayed without host round trips.
//
// Controller (the paper says only "adaptive, FSAL"): err = max over cells
// of |dt sum_j e_j k_j|_2; accept when err <= rtol; factor =
// clamp(0.9 (rtol/err)^(1/5), 0.2, 5), capped at 1 right after a rejection;
// on accept m <- m5/|m5| and k7 becomes k1 (slot rotation, no copy).
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "ctx.h"

namespace mm {

// Dormand & Prince (1980) RK5(4)7FSAL coefficients.
__constant__ double c_dp_a[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84},
};
// e_j = b5_j - b4_j
__constant__ double c_dp_e[7] = {35.0 / 384 - 5179.0 / 57600, 0.0, 500.0 / 1113 - 7571.0 / 16695,
                                 125.0 / 192 - 393.0 / 640, -2187.0 / 6784 + 92097.0 / 339200,
                                 11.0 / 84 - 187.0 / 2100, -1.0 / 40};

// k slot of stage j (0-based) under FSAL rotation: slot 0 and 6 swap roles
__device__ __forceinline__ int kslot_of(int j, int k_first) {
    if (j == 0) return k_first;
    if (j == 6) return 6 - k_first;
    return j;
}

template <typename T> __device__ __forceinline__ const T* stage_coef(const DevState* st, int s);
template <> __device__ __forceinline__ const float* stage_coef<float>(const DevState* st, int s) { return st->cf32[s]; }
template <> __device__ __forceinline__ const double* stage_coef<double>(const DevState* st, int s) { return st->cf64[s]; }
template <typename T> __device__ __forceinline__ const T* err_coef(const DevState* st);
template <> __device__ __forceinline__ const float* err_coef<float>(const DevState* st) { return st->ce32; }
template <> __device__ __forceinline__ const double* err_coef<double>(const DevState* st) { return st->ce64; }

// m_s = m0 + sum_j (dt a_sj) k_j, S = stage index (compile time)
template <typename T, int S>
__global__ void __launch_bounds__(256) combine_kernel(const DevState* __restrict__ st, T* const* __restrict__ kptr,
                                                      const T* __restrict__ m0, T* __restrict__ ms, long long n3) {
    if (!st->active) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const int kf = st->k_first;
    const T* cf = stage_coef<T>(st, S);
    T acc = m0[i];
#pragma unroll
    for (int j = 0; j < S; ++j) {
        if (j == 1 && S == 6) continue;             // a_7,2 = 0
        acc += cf[j] * __ldg(&kptr[kslot_of(j, kf)][i]);
    }
    ms[i] = acc;
}

// FP32, 3N a multiple of 4: four elements per thread as 16-byte vectors.
template <int S>
__global__ void __launch_bounds__(256) combine_vec4_kernel(const DevState* __restrict__ st,
                                                           float* const* __restrict__ kptr,
                                                           const float* __restrict__ m0, float* __restrict__ ms,
                                                           long long n4) {
    if (!st->active) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n4) return;
    const int kf = st->k_first;
    const float* cf = st->cf32[S];
    float4 acc = __ldg(reinterpret_cast<const float4*>(m0) + i);
#pragma unroll
    for (int j = 0; j < S; ++j) {
        if (j == 1 && S == 6) continue;             // a_7,2 = 0
        const float c = cf[j];
        const float4 k = __ldg(reinterpret_cast<const float4*>(kptr[kslot_of(j, kf)]) + i);
        acc.x += c * k.x; acc.y += c * k.y; acc.z += c * k.z; acc.w += c * k.w;
    }
    reinterpret_cast<float4*>(ms)[i] = acc;
}

// per-cell error |dt sum e_j k_j|, block max, atomic max into st->err(_f)
template <typename T>
__global__ void error_kernel(DevState* st, T* const* __restrict__ kptr, long long N) {
    if (!st->active) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int kf = st->k_first;
    const T* ce = err_coef<T>(st);
    T e2 = 0;
    if (i < N) {
        T ex = 0, ey = 0, ez = 0;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            if (j == 1) continue;                   // e_2 = 0
            const T* k = kptr[kslot_of(j, kf)];
            const T w = ce[j];
            ex += w * k[i];
            ey += w * k[N + i];
            ez += w * k[2 * N + i];
        }
        e2 = sqrt(ex * ex + ey * ey + ez * ez);
        if (!(e2 == e2)) e2 = (T)INFINITY;   // NaN -> inf: forces a rejection, then underflow status
    }
    T bm = warp_max(e2);
    __shared__ T red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bm;
    __syncthreads();
    if (threadIdx.x < 32) {
        T v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : (T)0;
        v = warp_max(v);
        if (threadIdx.x == 0) {
            if (sizeof(T) == 4) atomic_max_nonneg(&st->err_f, (float)v);
            else atomic_max_nonneg(&st->err, (double)v);
        }
    }
}

// Start of an attempt: decide whether it runs, pick dt_eff, clear the error.
__global__ void attempt_begin_kernel(DevState* st) {
    const bool more = st->accepted < st->target && st->t < st->t_end && st->status == 0;
    st->active = more ? 1 : 0;
    if (!more) return;
    double dt = st->dt;
    if (st->replay) {
        const long long q = st->accepted;
        dt = q < st->replay_n ? st->replay_dts[q] : 0.0;
    }
    if (st->t + dt > st->t_end) dt = st->t_end - st->t;
    st->dt_eff = dt;
    for (int s = 0; s < 7; ++s) {
        for (int j = 0; j < 6; ++j) {
            st->cf64[s][j] = dt * c_dp_a[s][j];
            st->cf32[s][j] = (float)(dt * c_dp_a[s][j]);
        }
        st->ce64[s] = dt * c_dp_e[s];
        st->ce32[s] = (float)(dt * c_dp_e[s]);
    }
    st->err = 0.0;
    st->err_f = 0.0f;
    st->attempts += 1;
}

// After the error reduction: accept / reject and the next step size.
__global__ void controller_kernel(DevState* st, int prec) {
    st->accept = 0;
    if (!st->active) return;
    const double err = prec == 32 ? (double)st->err_f : st->err;
    const double dt = st->dt_eff;
    if (st->replay) {
        st->accept = 1;
    } else {
        double fac = err > 0.0 ? 0.9 * pow(st->rtol / err, st->ctrl_exp) : 5.0;
        if (!(fac == fac)) fac = 0.2;
        fac = fmin(fmax(fac, 0.2), 5.0);
        if (err <= st->rtol) {
            if (st->last_rejected) fac = fmin(fac, 1.0);
            st->accept = 1;
            st->last_rejected = 0;
            // a step clipped to land on t_end keeps the unclipped size
            const double base = dt < st->dt ? st->dt : dt;
            st->dt = fmin(base * fac, st->dt_max);
        } else {
            st->last_rejected = 1;
            st->rejected += 1;
            const double nd = dt * fac;
            if (nd < st->dt_min || !(err < INFINITY)) {
                st->status = !(err < INFINITY) ? MM_ERR_NONFINITE : MM_ERR_DT_UNDERFLOW;
            }
            st->dt = fmax(nd, st->dt_min);
        }
    }
    if (st->accept) {
        st->t += dt;
        st->accepted += 1;
        st->step += 1;
        if (st->fsal) st->k_first = 6 - st->k_first;   // FSAL: k7 becomes k1
    }
}

template <typename T>
__global__ void accept_kernel(const DevState* __restrict__ st, const T* __restrict__ m5, T* __restrict__ m0,
                              long long N) {
    if (!st->active || !st->accept) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T x = m5[i], y = m5[N + i], z = m5[2 * N + i];
    const T n2 = x * x + y * y + z * z;
    const T inv = n2 > (T)0 ? (T)1 / sqrt(n2) : (T)0;
    m0[i] = x * inv;
    m0[N + i] = y * inv;
    m0[2 * N + i] = z * inv;
}

// Heun step bookkeeping (fixed dt): t += dt, step += 1.
__global__ void heun_advance_kernel(DevState* st) {
    if (!st->active) return;
    st->t += st->dt;
    st->step += 1;
    st->accepted += 1;
    st->attempts += 1;
}

__global__ void heun_begin_kernel(DevState* st) {
    st->active = (st->accepted < st->target && st->t < st->t_end && st->status == 0) ? 1 : 0;
    st->dt_eff = st->dt;
}

void demag_eval(mm_ctx* c, const void* m, void* Hd) {
    if (surrogate_active(c)) surrogate_apply(c, m, Hd);
    else demag_apply(c, m, Hd);
}

// H_demag(m) followed by the field kernel of `mode`.  With exact demag on a
// grid that allows it, the last demag pass (inverse X) runs inside the
// field kernel and H_demag never goes through global memory.
static void demag_and_field(mm_ctx* c, bool demag, int mode, unsigned terms, const void* m, void* out, void* out2,
                            const void* m0, const void* k1, int gate, int kstage) {
    if (demag && !surrogate_active(c) && field_c2r_fusable(c)) {
        demag_apply_partial(c, m, 0);
        field_c2r_launch(c, mode, terms, m, out, out2, m0, k1, -1, gate, kstage);
        return;
    }
    if (demag) demag_eval(c, m, c->d_hd);
    field_launch(c, mode, terms, m, demag ? c->d_hd : nullptr, out, out2, m0, k1, -1, gate, kstage);
}

template <typename T>
static void rk45_attempt_t(mm_ctx* c) {
    const long long N = c->N, n3 = 3 * N;
    const unsigned tb = 256, nb3 = (unsigned)((n3 + tb - 1) / tb), nb = (unsigned)((N + tb - 1) / tb);
    {
        LaunchScope ls(c, "rk_begin", 0.0);
        attempt_begin_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
    }
    T* const* kp = (T* const*)c->d_kslot;
    const unsigned terms = c->terms;
    const bool demag = c->dm.on && (terms & MM_TERM_DEMAG);
    const bool fused = demag && sizeof(T) == 4 && !surrogate_active(c) && demag_stage_fusable(c);
    const bool fused_c2r = fused && field_c2r_fusable(c);
    for (int s = 1; s < 7; ++s) {
        if (fused_c2r) {
            // stage combine inside the forward X pass, inverse X pass inside the field kernel
            demag_apply_partial(c, nullptr, s);
            field_c2r_launch(c, MODE_K, terms, c->d_mtmp, s < 6 ? c->d_k[s] : nullptr, nullptr, nullptr, nullptr,
                             -1, 1, 6);
            continue;
        }
        if (fused) {
            demag_apply_stage(c, s, c->d_hd);
        } else {
            LaunchScope ls(c, "rk_combine", (double)sizeof(T) * n3 * (1 + s + (s == 6 ? 0 : 1)));
            static void (*const kern[7])(const DevState*, T* const*, const T*, T*, long long) = {
                nullptr, combine_kernel<T, 1>, combine_kernel<T, 2>, combine_kernel<T, 3>,
                combine_kernel<T, 4>, combine_kernel<T, 5>, combine_kernel<T, 6>};
            if constexpr (sizeof(T) == 4) {
                if (n3 % 4 == 0) {
                    static void (*const k4[7])(const DevState*, float* const*, const float*, float*, long long) = {
                        nullptr, combine_vec4_kernel<1>, combine_vec4_kernel<2>, combine_vec4_kernel<3>,
                        combine_vec4_kernel<4>, combine_vec4_kernel<5>, combine_vec4_kernel<6>};
                    const long long n4 = n3 / 4;
                    k4[s]<<<(unsigned)((n4 + tb - 1) / tb), tb, 0, c->stream>>>(
                        c->d_state, (float* const*)kp, (const float*)c->d_m, (float*)c->d_mtmp, n4);
                } else {
                    kern[s]<<<nb3, tb, 0, c->stream>>>(c->d_state, kp, (const T*)c->d_m, (T*)c->d_mtmp, n3);
                }
            } else {
                kern[s]<<<nb3, tb, 0, c->stream>>>(c->d_state, kp, (const T*)c->d_m, (T*)c->d_mtmp, n3);
            }
        }
        if (demag && !fused) demag_eval(c, c->d_mtmp, c->d_hd);
        // stages 2..6 own fixed slots; the FSAL stage 7 slope goes to the slot
        // that does not hold k1 (resolved on the device)
        field_launch(c, MODE_K, terms, c->d_mtmp, demag ? c->d_hd : nullptr, s < 6 ? c->d_k[s] : nullptr, nullptr,
                     nullptr, nullptr, -1, 1, 6);
    }
    {
        LaunchScope ls(c, "rk_error", (double)sizeof(T) * 3 * N * 6);
        error_kernel<T><<<nb, tb, 0, c->stream>>>(c->d_state, kp, N);
    }
    {
        LaunchScope ls(c, "rk_control", 0.0);
        controller_kernel<<<1, 1, 0, c->stream>>>(c->d_state, c->prec);
    }
    {
        LaunchScope ls(c, "rk_accept", (double)sizeof(T) * 6 * N);
        accept_kernel<T><<<nb, tb, 0, c->stream>>>(c->d_state, (const T*)c->d_mtmp, (T*)c->d_m, N);
    }
}

void rk45_attempt(mm_ctx* c) {
    if (c->prec == 32) rk45_attempt_t<float>(c);
    else rk45_attempt_t<double>(c);
}

void rk45_first_slope(mm_ctx* c) {
    const unsigned terms = c->terms;
    const bool demag = c->dm.on && (terms & MM_TERM_DEMAG);
    demag_and_field(c, demag, MODE_K, terms, c->d_m, nullptr, nullptr, nullptr, nullptr, 0, 0);
}

void heun_batch_begin(mm_ctx* c) {
    LaunchScope ls(c, "heun_begin", 0.0);
    heun_begin_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
}

void heun_batch_advance(mm_ctx* c) {
    LaunchScope ls(c, "heun_advance", 0.0);
    heun_advance_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
}

// Classical RK4 (Methods, "Integrators": fixed step): stage states
// m0 + c dt k with c = 1/2, 1/2, 1, then m0 <- normalise(m0 + dt/6 (k1 +
// 2 k2 + 2 k3 + k4)); dt from the device state (fixed per context).
template <typename T>
__global__ void __launch_bounds__(256) rk4_stage_kernel(const DevState* __restrict__ st, const T* __restrict__ m0,
                                                        const T* __restrict__ k, double c, T* __restrict__ out,
                                                        long long n3) {
    if (!st->active) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const T h = (T)(c * st->dt);
    out[i] = m0[i] + h * __ldg(k + i);
}

template <typename T>
__global__ void __launch_bounds__(256) rk4_final_kernel(const DevState* __restrict__ st, T* __restrict__ m0,
                                                        const T* __restrict__ k1, const T* __restrict__ k2,
                                                        const T* __restrict__ k3, const T* __restrict__ k4,
                                                        long long N) {
    if (!st->active) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T h6 = (T)(st->dt / 6.0);
    T v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long j = c * N + i;
        v[c] = m0[j] + h6 * (k1[j] + (T)2 * k2[j] + (T)2 * k3[j] + k4[j]);
    }
    const T n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const T inv = n2 > (T)0 ? (T)1 / sqrt(n2) : (T)0;
#pragma unroll
    for (int c = 0; c < 3; ++c) m0[c * N + i] = v[c] * inv;
}

template <typename T>
static void rk4_step_t(mm_ctx* c) {
    const unsigned terms = c->terms;
    const bool demag = c->dm.on && (terms & MM_TERM_DEMAG);
    const long long N = c->N, n3 = 3 * N;
    const unsigned tb = 256, nb3 = (unsigned)((n3 + tb - 1) / tb), nb = (unsigned)((N + tb - 1) / tb);
    {
        LaunchScope ls(c, "rk4_begin", 0.0);
        heun_begin_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
    }
    static const double cs[4] = {0.0, 0.5, 0.5, 1.0};
    for (int s = 0; s < 4; ++s) {
        const void* ms = c->d_m;
        if (s > 0) {
            LaunchScope ls(c, "rk4_stage", (double)sizeof(T) * n3 * 3);
            rk4_stage_kernel<T><<<nb3, tb, 0, c->stream>>>(c->d_state, (const T*)c->d_m, (const T*)c->d_k[s - 1],
                                                            cs[s], (T*)c->d_mtmp, n3);
            ms = c->d_mtmp;
        }
        demag_and_field(c, demag, MODE_K, terms, ms, c->d_k[s], nullptr, nullptr, nullptr, 1, 0);
    }
    {
        LaunchScope ls(c, "rk4_final", (double)sizeof(T) * N * 18);
        rk4_final_kernel<T><<<nb, tb, 0, c->stream>>>(c->d_state, (T*)c->d_m, (const T*)c->d_k[0], (const T*)c->d_k[1],
                                                       (const T*)c->d_k[2], (const T*)c->d_k[3], N);
    }
    LaunchScope ls(c, "rk4_advance", 0.0);
    heun_advance_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
}

void rk4_step(mm_ctx* c) {
    if (c->prec == 32) rk4_step_t<float>(c);
    else rk4_step_t<double>(c);
}

void heun_step(mm_ctx* c) {
    const unsigned terms = c->terms;
    const bool demag = c->dm.on && (terms & MM_TERM_DEMAG);
    {
        LaunchScope ls(c, "heun_begin", 0.0);
        heun_begin_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
    }
    // predictor: k1 = f(m, H(m) + H_th); m* = m + dt k1
    demag_and_field(c, demag, MODE_HEUN1, terms, c->d_m, c->d_mtmp, c->d_k[0], nullptr, nullptr, 1, 0);
    // corrector: m' = normalise(m + dt/2 (k1 + f(m*, H(m*) + H_th))), same noise
    demag_and_field(c, demag, MODE_HEUN2, terms, c->d_mtmp, c->d_m, nullptr, c->d_m, c->d_k[0], 1, 0);
    LaunchScope ls(c, "heun_advance", 0.0);
    heun_advance_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
}

// Depondt-Mertens (Methods, "Integrators"): Omega_1 = Omega(m) and the
// predictor m* = R(Omega_1 dt) m in one launch, then Omega_2 = Omega(m*) and
// m <- R((Omega_1 + Omega_2) dt / 2) m in the next; one thermal draw per step
// (the step counter advances after the corrector).  The rotation keeps |m|;
// the corrector also rescales by 1/|m|, a round-off-level change that keeps
// long FP32 runs from drifting.
void dm_step(mm_ctx* c) {
    const unsigned terms = c->terms;
    const bool demag = c->dm.on && (terms & MM_TERM_DEMAG);
    {
        LaunchScope ls(c, "dm_begin", 0.0);
        heun_begin_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
    }
    demag_and_field(c, demag, MODE_DM1, terms, c->d_m, c->d_mtmp, c->d_k[0], nullptr, nullptr, 1, 0);
    demag_and_field(c, demag, MODE_DM2, terms, c->d_mtmp, c->d_m, nullptr, c->d_m, c->d_k[0], 1, 0);
    LaunchScope ls(c, "dm_advance", 0.0);
    heun_advance_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
}

// Adaptive Depondt-Mertens: err = max over cells |cand - m*| (the corrector
// against the first-order predictor), block max, atomic max into st->err(_f).
template <typename T>
__global__ void dm_error_kernel(DevState* st, const T* __restrict__ cand, const T* __restrict__ mstar, long long N) {
    if (!st->active) return;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    T e2 = 0;
    if (i < N) {
        const T dx = cand[i] - mstar[i], dy = cand[N + i] - mstar[N + i], dz = cand[2 * N + i] - mstar[2 * N + i];
        e2 = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(e2 == e2)) e2 = (T)INFINITY;
    }
    T bm = warp_max(e2);
    __shared__ T red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bm;
    __syncthreads();
    if (threadIdx.x < 32) {
        T v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : (T)0;
        v = warp_max(v);
        if (threadIdx.x == 0) {
            if (sizeof(T) == 4) atomic_max_nonneg(&st->err_f, (float)v);
            else atomic_max_nonneg(&st->err, (double)v);
        }
    }
}

// One attempted adaptive step: begin (dt_eff, active, error cleared),
// predictor (Omega_1 -> k[0], m* -> mtmp), corrector into the candidate
// buffer k[1], the embedded error, the device controller, and the accept copy.
template <typename T>
static void dm_adaptive_attempt_t(mm_ctx* c) {
    const unsigned terms = c->terms;
    const bool demag = c->dm.on && (terms & MM_TERM_DEMAG);
    const long long N = c->N;
    const unsigned tb = 256, nb = (unsigned)((N + tb - 1) / tb);
    {
        LaunchScope ls(c, "dm_begin", 0.0);
        attempt_begin_kernel<<<1, 1, 0, c->stream>>>(c->d_state);
    }
    demag_and_field(c, demag, MODE_DM1, terms, c->d_m, c->d_mtmp, c->d_k[0], nullptr, nullptr, 1, 0);
    demag_and_field(c, demag, MODE_DM2, terms, c->d_mtmp, c->d_k[1], nullptr, c->d_m, c->d_k[0], 1, 0);
    {
        LaunchScope ls(c, "dm_error", (double)sizeof(T) * 6 * N);
        dm_error_kernel<T><<<nb, tb, 0, c->stream>>>(c->d_state, (const T*)c->d_k[1], (const T*)c->d_mtmp, N);
    }
    {
        LaunchScope ls(c, "dm_control", 0.0);
        controller_kernel<<<1, 1, 0, c->stream>>>(c->d_state, c->prec);
    }
    LaunchScope ls(c, "dm_accept", (double)sizeof(T) * 6 * N);
    accept_kernel<T><<<nb, tb, 0, c->stream>>>(c->d_state, (const T*)c->d_k[1], (T*)c->d_m, N);
}

void dm_adaptive_attempt(mm_ctx* c) {
    if (c->prec == 32) dm_adaptive_attempt_t<float>(c);
    else dm_adaptive_attempt_t<double>(c);
}

}  // namespace mm
