// Replica batching (Methods, "Replica batching"): R independent thin-film
// replicas (nz = 1) of possibly different sizes advance together, each with
// its own Philox key, temperature and current density.  One persistent
// launch per stage of the Heun or Depondt-Mertens step: every CTA takes whole replicas, one after another,
// from a shared work counter over a size-mixed order and runs, for each, the
// three demag phases
// (row R2C, column convolution with the size class's tensor spectrum,
// row C2R) and the fused field + torque + stage update.  The replica's
// half spectrum lives in a CTA-private scratch slab (small enough to stay
// in L2); every transform runs in shared memory.  No grid-wide
// synchronisation is needed: a CTA owns its replica for the whole stage.
//
// Device side: descriptors, the per-replica stage and the persistent kernel
// template.  Each thread-count variant of the kernel is instantiated in its
// own translation unit (batch_k256.cu, batch_k512.cu) so they compile in
// parallel.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "fft_ct.cuh"
#include "fft_rt.cuh"
#include "field_dev.cuh"

namespace mm {

// complex values a thread holds per Stockham pass of a compile-time plan
// (the runtime-planned path holds kMaxV); a pass of radix R can use
// (kMaxVB / R) R of them, so the lines per pass are sized by ct_cap.  24
// (every radix divides it) measured faster than 8: fewer spills did not
// pay for three times the passes and barriers.
constexpr int kMaxVB = 24;

struct RepDev {
    int nx, ny, cls;
    int active;             // 0: an idle slot (retire/refill ran out of trials)
    long long off;          // element offset of the replica's [3][ny][nx] block
    uint32_t key0, key1;    // Philox key
    float th_scale;         // sqrt(T / (V dt))
    float tq_base;          // hbar J / (e mu0 t_F)
    long long trial;        // trial running in this slot (retire/refill), else -1
    long long step0;        // global step at which that trial started: the noise
                            // counter is the trial's own step, step - step0
};

// Retire/refill of batched trials (Results, "Replica batching"): trial q has
// its own current J[q], temperature T[q] and Philox key splitmix64(base + q)
// and starts from m_init; after every step a slot whose trial has
// mean(m . axis) <= threshold, or has taken max_steps steps, records the
// outcome and, with refill, starts the next trial not yet started.
struct TrialDev {
    long long n_trials, max_steps;
    const float* J;                 // [n_trials]
    const float* T;                 // [n_trials]
    const float* m_init;            // [3][N] of the common replica grid
    float axis[3];
    float threshold;
    unsigned long long base_seed;
    float tq_per_J;                 // hbar / (e mu0 t_F)
    float th_per_sqrtT;             // 1 / sqrt(V dt)
    int refill;
    unsigned long long* next;       // next trial to start
    unsigned long long* done;       // trials finished
    long long* steps;               // per trial: steps taken (-1 until finished)
    int* stopped;                   // per trial: 1 if the stop condition ended it
};

// splitmix64 (Steele, Lea and Flood, 2014): the trial key schedule
__host__ __device__ __forceinline__ unsigned long long splitmix64_dev(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// End-of-step check of one slot (one thread): records a finished trial and
// loads the next one into rp (and into the slot's descriptor in global
// memory).  Returns 1 when a new trial starts (the caller resets m to
// m_init), 0 otherwise.  steps_taken counts the trial's steps including the
// one just finished; step_next is the global step the next trial starts at.
__device__ __forceinline__ int trial_check(const TrialDev& tr, RepDev& rp, RepDev* rp_glob, float mean_proj,
                                           long long steps_taken, long long step_next) {
    const bool stop = mean_proj <= tr.threshold;
    if (!stop && steps_taken < tr.max_steps) return 0;
    const long long q = rp.trial;
    tr.steps[q] = steps_taken;
    tr.stopped[q] = stop ? 1 : 0;
    atomicAdd(tr.done, 1ull);
    const unsigned long long qn = tr.refill ? atomicAdd(tr.next, 1ull) : (unsigned long long)tr.n_trials;
    if (qn >= (unsigned long long)tr.n_trials) {
        rp.active = 0;
        rp.trial = -1;
        rp_glob->active = 0;
        rp_glob->trial = -1;
        return 0;
    }
    const unsigned long long key = splitmix64_dev(tr.base_seed + qn);
    rp.trial = (long long)qn;
    rp.step0 = step_next;
    rp.key0 = (uint32_t)(key & 0xFFFFFFFFull);
    rp.key1 = (uint32_t)(key >> 32);
    const float T = tr.T[qn];
    rp.th_scale = T > 0.f ? sqrtf(T) * tr.th_per_sqrtT : 0.f;
    rp.tq_base = tr.J[qn] * tr.tq_per_J;
    rp_glob->trial = rp.trial;
    rp_glob->step0 = rp.step0;
    rp_glob->key0 = rp.key0;
    rp_glob->key1 = rp.key1;
    rp_glob->th_scale = rp.th_scale;
    rp_glob->tq_base = rp.tq_base;
    return 1;
}

struct ClsDev {
    int nx, ny, Lh, Py, Kx, Wk, Ky;
    const float* khat;      // [4][Ky][Wk]: xx, yy, zz, xy
    const float2* twx;      // exp(-2 pi i q / (2 Lh))
    const float2* twy;      // exp(-2 pi i q / Py)
    Plan ph, py;            // runtime plans (generic path)
};

struct BatchArgs {
    RepDev* rep;
    const ClsDev* cls;
    const int* order;
    int* next;              // work counter of this stage (zeroed before the launch)
    int R;
    float* m0;              // state
    float* ms;              // predictor state
    float* k1;              // predictor slope
    float2* scratch;
    long long scratch_stride;
    FieldArgs<float> fa;    // shared field parameters (per-replica fields set in-kernel)
    int demag;
    int stage;              // 1: predictor, 2: corrector
    int dm;                 // 1: Depondt-Mertens rotation, 0: Heun
    int trials;             // 1: retire/refill is on (tr is valid)
    TrialDev tr;
    const DevState* st;
};

// values per thread every pass of the compile-time plan of length L can hold
__host__ __device__ constexpr int ct_cap(int L, int maxv) {
    int cap = maxv;
    for (int p = 0; p < ct_npass(L); ++p) {
        const int r = ct_radix(L, p), c = (maxv / r) * r;
        if (c < cap) cap = c;
    }
    return cap;
}
// size classes with compile-time plans (half length, column length): the
// cases of batch_stage_kernel's dispatch
__host__ __device__ inline bool b_compiled(int Lh, int Py) {
    return (Lh == 16 && Py == 32) || (Lh == 32 && Py == 64) || (Lh == 48 && Py == 96) || (Lh == 64 && Py == 128) ||
           (Lh == 96 && Py == 192) || (Lh == 128 && Py == 256) || (Lh == 256 && Py == 512);
}
__host__ __device__ inline int b_cap(int L, bool ct) { return ct ? ct_cap(L, kMaxVB) : kMaxV; }
__host__ __device__ inline int b_rows_x(int Lh, int NT, bool ct) { return b_cap(Lh, ct) * NT / Lh; }
__host__ __device__ inline int b_tk(int Py, int NT, bool ct) {
    int cap = b_cap(Py, ct) * NT / (3 * Py), tk = 1;
    while (tk * 2 <= cap && tk * 2 <= 16) tk *= 2;
    return tk;
}
__host__ __device__ inline int b_rows_c(int Lh, int NT, bool ct) { return b_cap(Lh, ct) * NT / (3 * Lh); }

template <int LX, int NT, int DIR>
__device__ __forceinline__ void row_fft(float2* sm, int nl, int nin, const ClsDev& cd) {
    if constexpr (LX > 0) ct_fft<float, DIR, LX, LX + 1, NT, kMaxVB>(sm, nl, nin, cd.twx, 2);
    else fft_lines<float, DIR>(sm, nl, cd.Lh + 1, cd.ph, nin, cd.twx, 2);
}

template <int LY, int NT, int DIR>
__device__ __forceinline__ void col_fft(float2* sm, int nl, int nin, const ClsDev& cd) {
    if constexpr (LY > 0) ct_fft<float, DIR, LY, LY + 1, NT, kMaxVB>(sm, nl, nin, cd.twy, 1);
    else fft_lines<float, DIR>(sm, nl, cd.Py + 1, cd.py, nin, cd.twy, 1);
}

// One replica, one stage, in three phases.  Each phase is its own
// (non-inlined) function so the register allocation of one phase does not
// burden the others.  LX / LY: compile-time half length / column length
// (0 = runtime plan).

// phase X: rows (c, y) of Ms*m -> half spectra in S[(c ny + y) Wk + kx]
template <int LX, int NT>
__device__ __noinline__ void stage_phase_x(const float* mE, long long N, int nx, int ny, float ms, const ClsDev& cd,
                                           float2* S, float2* sm) {
    const int Lh = LX > 0 ? LX : cd.Lh;
    const int pitch = Lh + 1;
    float* smr = reinterpret_cast<float*>(sm);
    // ---- phase X: rows (c, y) -> half spectra in S[(c ny + y) Wk + kx]
    const int RB = b_rows_x(Lh, NT, LX > 0);
    for (int r0 = 0; r0 < 3 * ny; r0 += RB) {
        const int nl = min(RB, 3 * ny - r0);
        for (int l = 0; l < nl; ++l) {
            const int row = r0 + l, c = row / ny, y = row - c * ny;
            const float* src = mE + c * N + (long long)y * nx;
            for (int q = threadIdx.x; q < 2 * Lh; q += NT) smr[2 * l * pitch + q] = q < nx ? src[q] * ms : 0.f;
        }
        __syncthreads();
        row_fft<LX, NT, 1>(sm, nl, (nx + 1) / 2, cd);
        for (int l = 0; l < nl; ++l) {
            float2* out = S + (long long)(r0 + l) * cd.Wk;
            for (int k = threadIdx.x; k <= Lh; k += NT) {
                const float2 zk = sm[l * pitch + (k == Lh ? 0 : k)];
                const float2 zc = cconj<float>(sm[l * pitch + (k == 0 ? 0 : Lh - k)]);
                const float2 E = cscale<float>(cadd<float>(zk, zc), 0.5f);
                const float2 O = cscale<float>(mul_mi<float, 1>(csub<float>(zk, zc)), 0.5f);
                out[k] = cadd<float>(E, cmul<float>(__ldg(&cd.twx[k]), O));
            }
        }
        __syncthreads();
    }
}

// phase Y: columns, FFT along y, tensor multiply, inverse, keep ny
template <int LY, int NT>
__device__ __noinline__ void stage_phase_y(int ny, const ClsDev& cd, float2* S, float2* sm) {
    const int Py = LY > 0 ? LY : cd.Py;
    // ---- phase Y: columns, FFT along y, tensor multiply, inverse, keep ny
    const int TK = b_tk(Py, NT, LY > 0);
    const int tks = __ffs(TK) - 1;
    const int cp = Py + 1;
    for (int kx0 = 0; kx0 < cd.Kx; kx0 += TK) {
        for (int c = 0; c < 3; ++c)
            for (int e = threadIdx.x; e < (ny << tks); e += NT) {
                const int kxl = e & (TK - 1), pt = e >> tks;
                float2 v = mkc<float>(0.f, 0.f);
                if (kx0 + kxl < cd.Kx) v = S[(long long)(c * ny + pt) * cd.Wk + kx0 + kxl];
                sm[(c * TK + kxl) * cp + pt] = v;
            }
        __syncthreads();
        col_fft<LY, NT, 1>(sm, 3 * TK, ny, cd);
        const long long kcs = (long long)cd.Ky * cd.Wk;
        for (int e = threadIdx.x; e < (Py << tks); e += NT) {
            const int kxl = e & (TK - 1), kk = e >> tks;
            const int kx = kx0 + kxl;
            if (kx >= cd.Kx) continue;
            const int kf = kk <= Py / 2 ? kk : Py - kk;
            const float sy = kk <= Py / 2 ? 1.f : -1.f;
            const float* K = cd.khat + (long long)kf * cd.Wk + kx;
            const float kxx = __ldg(K), kyy = __ldg(K + kcs), kzz = __ldg(K + 2 * kcs), kxy = sy * __ldg(K + 3 * kcs);
            float2* px = &sm[(0 * TK + kxl) * cp + kk];
            float2* py = &sm[(1 * TK + kxl) * cp + kk];
            float2* pz = &sm[(2 * TK + kxl) * cp + kk];
            const float2 mx = *px, my = *py, mz = *pz;
            *px = mkc<float>(kxx * mx.x + kxy * my.x, kxx * mx.y + kxy * my.y);
            *py = mkc<float>(kxy * mx.x + kyy * my.x, kxy * mx.y + kyy * my.y);
            *pz = mkc<float>(kzz * mz.x, kzz * mz.y);
        }
        __syncthreads();
        col_fft<LY, NT, -1>(sm, 3 * TK, Py, cd);
        for (int c = 0; c < 3; ++c)
            for (int e = threadIdx.x; e < (ny << tks); e += NT) {
                const int kxl = e & (TK - 1), pt = e >> tks;
                if (kx0 + kxl < cd.Kx) S[(long long)(c * ny + pt) * cd.Wk + kx0 + kxl] = sm[(c * TK + kxl) * cp + pt];
            }
        __syncthreads();
    }
}

// phase C: C2R rows of a block of y (three components) + field + update
// Returns this thread's share of sum over cells of m_new . axis (stage 2
// with retire/refill on; 0 otherwise).
template <int LX, int NT>
__device__ __noinline__ float stage_phase_c(const BatchArgs& a, const RepDev& rp, const ClsDev& cd, float* mE,
                                            long long N, int nx, int ny, float2* S, float2* sm, long long step,
                                            float dt) {
    FieldArgs<float> fa = a.fa;
    fa.m = mE;
    fa.N = N;
    fa.nx = nx;
    fa.ny = ny;
    fa.nz = 1;
    fa.key0 = rp.key0;
    fa.key1 = rp.key1;
    fa.th_scale = rp.th_scale;
    fa.tq_base = rp.tq_base;
    const Region<float>& R = fa.lut[0];
    const bool proj_on = a.trials && a.stage == 2;
    const v3<float> ax = mk3<float>(a.tr.axis[0], a.tr.axis[1], a.tr.axis[2]);
    float proj = 0.f;
    const int Lh = LX > 0 ? LX : cd.Lh;
    const int pitch = Lh + 1;
    float* smr = reinterpret_cast<float*>(sm);
    // ---- phase C: C2R rows of a block of y (three components) + field + update
    const int RBc = a.demag ? max(1, b_rows_c(Lh, NT, LX > 0)) : ny;
    for (int y0 = 0; y0 < ny; y0 += RBc) {
        const int nyb = min(RBc, ny - y0);
        if (a.demag) {
            const int nl = 3 * nyb;
            for (int l = 0; l < nl; ++l) {
                const int c = l / nyb, y = y0 + (l - c * nyb);
                const float2* in = S + (long long)(c * ny + y) * cd.Wk;
                for (int k = threadIdx.x; k <= Lh; k += NT) sm[l * pitch + k] = in[k];
            }
            __syncthreads();
            const int half = Lh / 2;
            for (int l = 0; l < nl; ++l)
                for (int k = threadIdx.x; k <= half; k += NT) {
                    const int k2 = Lh - k;
                    const float2 xk = sm[l * pitch + k], xk2 = sm[l * pitch + k2];
                    const float2 w1 = __ldg(&cd.twx[k]), w2 = __ldg(&cd.twx[k2]);
                    const float2 E1 = cadd<float>(xk, cconj<float>(xk2));
                    const float2 O1 = cmulc<float>(csub<float>(xk, cconj<float>(xk2)), w1);
                    const float2 E2 = cadd<float>(xk2, cconj<float>(xk));
                    const float2 O2 = cmulc<float>(csub<float>(xk2, cconj<float>(xk)), w2);
                    sm[l * pitch + k] = cadd<float>(E1, mul_mi<float, -1>(O1));
                    if (k2 != k && k2 < Lh) sm[l * pitch + k2] = cadd<float>(E2, mul_mi<float, -1>(O2));
                }
            __syncthreads();
            row_fft<LX, NT, -1>(sm, nl, Lh, cd);
        }
        for (int e = threadIdx.x; e < nyb * nx; e += NT) {
            const int yl = e / nx, x = e - yl * nx, y = y0 + yl;
            const long long i = (long long)y * nx + x;
            const v3<float> m = ld3(mE, N, i);
            v3<float> hd = mk3<float>(0.f, 0.f, 0.f);
            if (a.demag)
                hd = mk3<float>(smr[2 * (0 * nyb + yl) * pitch + x], smr[2 * (1 * nyb + yl) * pitch + x],
                                smr[2 * (2 * nyb + yl) * pitch + x]);
            v3<float> H, k;
            cell_field<float>(fa, x, y, 0, i, 0, R, m, a.demag ? &hd : nullptr, step - rp.step0, H, k, true,
                              a.dm != 0);
            // k: the slope (Heun) or the rotation vector Omega (Depondt-Mertens)
            if (a.stage == 1) {
                st3(a.k1 + rp.off, N, i, k);
                st3(a.ms + rp.off, N, i, a.dm ? rodrigues<float>(m, k, dt) : m + dt * k);
            } else {
                const v3<float> m0 = ld3(a.m0 + rp.off, N, i);
                const v3<float> kp = ld3(a.k1 + rp.off, N, i);
                const v3<float> mn = a.dm ? rodrigues<float>(m0, 0.5f * (kp + k), dt) : m0 + (0.5f * dt) * (kp + k);
                const v3<float> mu = rsqrtf(dot(mn, mn)) * mn;
                st3(a.m0 + rp.off, N, i, mu);
                if (proj_on) proj += dot(mu, ax);
            }
        }
        __syncthreads();
    }
    return proj;
}

// Retire/refill after the corrector: the mean of m . axis over the replica
// (block reduction), the stop test by one thread, and, when a new trial
// takes the slot, its initial state written by the whole CTA.
template <int NT>
__device__ __forceinline__ void slot_retire_refill(const BatchArgs& a, RepDev rp, int idx, float part, long long N,
                                                   long long step) {
    __shared__ float s_red[NT / 32];
    __shared__ int s_new;
    float v = part;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < NT / 32; ++w) tot += s_red[w];
        s_new = trial_check(a.tr, rp, a.rep + idx, tot / (float)N, step + 1 - rp.step0, step + 1);
    }
    __syncthreads();
    if (s_new) {
        float* m = a.m0 + rp.off;
        for (long long e = threadIdx.x; e < 3 * N; e += NT) m[e] = __ldg(a.tr.m_init + e);
    }
    __syncthreads();
}

template <int LX, int LY, int NT>
__device__ __forceinline__ void replica_stage(const BatchArgs& a, const RepDev& rp, int idx, const ClsDev& cd,
                                              float2* S, float2* sm, long long step, float dt) {
    const int nx = rp.nx, ny = rp.ny;
    const long long N = (long long)nx * ny;
    float* mE = (a.stage == 1 ? a.m0 : a.ms) + rp.off;
    if (a.demag) {
        stage_phase_x<LX, NT>(mE, N, nx, ny, a.fa.lut[0].Ms, cd, S, sm);
        stage_phase_y<LY, NT>(ny, cd, S, sm);
    }
    const float part = stage_phase_c<LX, NT>(a, rp, cd, mE, N, nx, ny, S, sm, step, dt);
    if (a.trials && a.stage == 2) slot_retire_refill<NT>(a, rp, idx, part, N, step);
}

template <int NT>
__global__ void __launch_bounds__(NT) batch_stage_kernel(BatchArgs a) {
    if (!a.st->active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    const long long step = a.st->step;
    const float dt = (float)a.st->dt;
    float2* S = a.scratch + blockIdx.x * a.scratch_stride;
    // the launch parameters and the current replica's descriptor live in
    // shared memory, so the non-inlined phases take them by reference
    // without a private copy in every thread's local memory
    __shared__ BatchArgs sa;
    __shared__ RepDev srp;
    if (threadIdx.x == 0) sa = a;
    __shared__ int s_w;
    for (;;) {
        // dynamic schedule: each CTA takes the next replica of the work order
        if (threadIdx.x == 0) s_w = atomicAdd(a.next, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= a.R) break;
        const int idx = a.order[w];
        if (threadIdx.x == 0) srp = a.rep[idx];
        __syncthreads();
        const RepDev& rp = srp;
        if (!rp.active) { __syncthreads(); continue; }   // uniform across the CTA
        const ClsDev& cd = a.cls[rp.cls];
        const int key = cd.Lh * 10000 + cd.Py;
        switch (key) {
#define MM_B(lh, py) case lh * 10000 + py: replica_stage<lh, py, NT>(sa, rp, idx, cd, S, sm, step, dt); break;
            MM_B(16, 32) MM_B(32, 64) MM_B(48, 96) MM_B(64, 128) MM_B(96, 192) MM_B(128, 256) MM_B(256, 512)
#undef MM_B
            default: replica_stage<0, 0, NT>(sa, rp, idx, cd, S, sm, step, dt); break;
        }
        __syncthreads();   // srp is rewritten for the next replica
    }
}

// Fused blocks of steps for replicas without demag (macro.cu): one-cell
// replicas (the macrospin ensemble of the paper's batching table and
// switching sweep) take one thread per slot with the moment in registers;
// films of up to 1024 cells take one CTA per replica with the state in
// shared memory and one cell per thread.
struct MacroArgs {
    RepDev* rep;
    int R;
    float* m;               // state, replica-outermost
    FieldArgs<float> fa;
    int dm;
    int trials;
    TrialDev tr;
    const DevState* st;
    int nsteps;
    int nmax;               // tile kernel: largest replica (cells)
    int ext;                // bulk DMI or a further local term is on
};
constexpr int kTileMaxCells = 1024;

// One size class of the stacked launch shape (batch_stacked.cu).
struct StackArgs {
    const RepDev* rep;
    const int* members;     // replica index of each class member, in storage order
    int nx, ny;
    float* m0;              // state (all replicas)
    float* ms;              // predictor state
    float* k1;              // predictor slope / rotation vector
    const float* hd;        // the class's demag field [member][3][ny][nx], or null
    FieldArgs<float> fa;
    int stage;              // 1 predictor, 2 corrector
    int dm;
    int ext;
    const DevState* st;
};
void stacked_field_launch(const StackArgs& a, int Rc, cudaStream_t s);
void stacked_trials_launch(const BatchArgs& a, int R, cudaStream_t s);
void macro_kernel_launch(const MacroArgs& a, cudaStream_t s);
void tile_kernel_launch(const MacroArgs& a, cudaStream_t s);
cudaError_t tile_kernel_attributes();
void macro_advance_launch(DevState* st, int nsteps, cudaStream_t s);

// host wrappers, one set per instantiated thread count
cudaError_t batch_kernel_attributes_256();
cudaError_t batch_kernel_attributes_512();
void batch_kernel_launch_256(const BatchArgs& a, int blocks, size_t smem, cudaStream_t s);
void batch_kernel_launch_512(const BatchArgs& a, int blocks, size_t smem, cudaStream_t s);
int batch_kernel_occupancy_256(size_t smem);
int batch_kernel_occupancy_512(size_t smem);

}  // namespace mm
