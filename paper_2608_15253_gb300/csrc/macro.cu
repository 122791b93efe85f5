// Replica-batched blocks of fused steps for replicas without demag (Results,
// "Replica batching": the single-cell ensemble with local fields, spin
// torque and thermal noise, the thermally assisted switching sweep, and
// the small exchange-coupled films of the batching table).  A one-cell
// replica's step is local: one thread per slot holds the moment in
// registers for a block of steps and runs the predictor, the corrector and,
// with retire/refill on, the stop test and the start of the next trial,
// without leaving the thread.  A small film is one CTA with its state in
// shared memory (tile_kernel).
#include <cuda_runtime.h>

#include "batch_dev.cuh"

namespace mm {

template <bool EXT>
__global__ void __launch_bounds__(32) macro_kernel(MacroArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    RepDev rp = a.rep[r];
    if (!rp.active) return;
    FieldArgs<float> fa = a.fa;
    fa.N = 1;
    fa.nx = fa.ny = fa.nz = 1;
    fa.m = a.m + rp.off;            // never read: every neighbour is absent
    fa.key0 = rp.key0;
    fa.key1 = rp.key1;
    fa.th_scale = rp.th_scale;
    fa.tq_base = rp.tq_base;
    const Region<float>& R = fa.lut[0];
    // the step's thermal draw is the same in both evaluations: drawn once
    // per step and added through the precomputed-field slot
    const bool hot = (fa.terms & MM_TERM_THERMAL) != 0;
    fa.terms = (fa.terms & ~MM_TERM_THERMAL) | MM_TERM_DEMAG;
    const float dt = (float)a.st->dt;
    const long long step0 = a.st->step;
    const bool dm = a.dm != 0;
    const v3<float> ax = mk3<float>(a.tr.axis[0], a.tr.axis[1], a.tr.axis[2]);
    float* mp = a.m + rp.off;
    v3<float> m = mk3<float>(mp[0], mp[1], mp[2]);
    const v3<float> zero = mk3<float>(0.f, 0.f, 0.f);
    // the draws do not depend on the state: the next step's is computed one
    // step ahead, so its Philox rounds overlap this step's dependent chain
    v3<float> hnext = hot && fa.th_scale != 0.f ? thermal_h<float>(fa, 0, R, step0 - rp.step0) : zero;
    for (int s = 0; s < a.nsteps; ++s) {
        const long long step = step0 + s;
        const long long ctr = step - rp.step0;    // the trial's own step: its noise counter
        v3<float> H, w1, w2;
        const v3<float> hth = hnext;
        if (hot && fa.th_scale != 0.f) hnext = thermal_h<float>(fa, 0, R, ctr + 1);
        cell_field<float, false, EXT>(fa, 0, 0, 0, 0, 0, R, m, &hth, ctr, H, w1, true, dm);
        const v3<float> ms = dm ? rodrigues<float>(m, w1, dt) : m + dt * w1;
        cell_field<float, false, EXT>(fa, 0, 0, 0, 0, 0, R, ms, &hth, ctr, H, w2, true, dm);
        const v3<float> mn = dm ? rodrigues<float>(m, 0.5f * (w1 + w2), dt) : m + (0.5f * dt) * (w1 + w2);
        m = rsqrtf(dot(mn, mn)) * mn;
        if (a.trials) {
            if (trial_check(a.tr, rp, a.rep + r, dot(m, ax), step + 1 - rp.step0, step + 1)) {
                m = mk3<float>(__ldg(a.tr.m_init), __ldg(a.tr.m_init + 1), __ldg(a.tr.m_init + 2));
                fa.key0 = rp.key0;
                fa.key1 = rp.key1;
                fa.th_scale = rp.th_scale;
                fa.tq_base = rp.tq_base;
                hnext = hot && fa.th_scale != 0.f ? thermal_h<float>(fa, 0, R, 0) : zero;
            }
            if (!rp.active) break;
        }
    }
    mp[0] = m.x;
    mp[1] = m.y;
    mp[2] = m.z;
}

// One film replica (nz = 1, no demag, at most 1024 cells) per CTA, one cell
// per thread: the state lives in shared memory buffer A, the predictor in
// buffer B, each thread's own m and Omega_1 (or slope k1) in registers.  Per
// step: predictor from A's neighbours -> B, barrier, corrector from B's
// neighbours -> A, (retire/refill: block reduction and the stop test),
// barrier.  Neighbours come from shared memory, ghosts where the film ends.
template <bool EXT>
__global__ void __launch_bounds__(kTileMaxCells) tile_kernel(MacroArgs a) {
    extern __shared__ float tsm[];
    __shared__ float s_red[kTileMaxCells / 32];
    __shared__ int s_new;
    RepDev rp = a.rep[blockIdx.x];
    if (!rp.active) return;   // uniform across the CTA
    const int nx = rp.nx, ny = rp.ny, N = nx * ny;
    float* A = tsm;
    float* B = tsm + 3 * a.nmax;
    FieldArgs<float> fa = a.fa;
    fa.N = N;
    fa.nx = nx;
    fa.ny = ny;
    fa.nz = 1;
    fa.key0 = rp.key0;
    fa.key1 = rp.key1;
    fa.th_scale = rp.th_scale;
    fa.tq_base = rp.tq_base;
    const Region<float>& R = fa.lut[0];
    const float c_pair = __ldg(fa.cpair);
    const int i = threadIdx.x;
    const bool own = i < N;
    const int x = own ? i % nx : 0, y = own ? i / nx : 0;
    const float dt = (float)a.st->dt;
    const long long step0 = a.st->step;
    const bool dm = a.dm != 0;
    const v3<float> ax = mk3<float>(a.tr.axis[0], a.tr.axis[1], a.tr.axis[2]);
    float* mg = a.m + rp.off;
    v3<float> m = own ? mk3<float>(mg[i], mg[N + i], mg[2 * N + i]) : mk3<float>(0.f, 0.f, 0.f);
    if (own) { A[i] = m.x; A[N + i] = m.y; A[2 * N + i] = m.z; }
    __syncthreads();
    // neighbour values of cell i from buffer S (ghosts outside the film)
    auto gather = [&](const float* S, const v3<float>& mc, v3<float>* nbv, bool* nbp, float* cnb) {
        const int pos[2] = {x, y}, dim[2] = {nx, ny}, stride[2] = {1, nx};
        const float hh[2] = {fa.hx, fa.hy};
#pragma unroll
        for (int d = 0; d < 2; ++d) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int sg = s == 0 ? 1 : -1;
                const int q = pos[d] + sg;
                const int slot = 2 * d + s;
                const bool in = q >= 0 && q < dim[d];
                nbp[slot] = in;
                if (in) {
                    const int j = i + sg * stride[d];
                    nbv[slot] = mk3<float>(S[j], S[N + j], S[2 * N + j]);
                    cnb[slot] = c_pair;
                } else {
                    nbv[slot] = ghost_value<float, EXT>(mc, d, sg, hh[d], R.ratio, R.ratio_b);
                    cnb[slot] = R.cg;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            nbp[4 + s] = false;
            nbv[4 + s] = ghost_value<float, EXT>(mc, 2, s == 0 ? 1 : -1, fa.hz, R.ratio, R.ratio_b);
            cnb[4 + s] = R.cg;
        }
    };
    const v3<float> zero = mk3<float>(0.f, 0.f, 0.f);
    for (int s = 0; s < a.nsteps; ++s) {
        const long long step = step0 + s;
        const long long ctr = step - rp.step0;
        v3<float> w1 = zero, H;
        if (own) {
            v3<float> nbv[6];
            bool nbp[6];
            float cnb[6];
            gather(A, m, nbv, nbp, cnb);
            cell_field_nb<float, EXT>(fa, i, R, m, nbv, nbp, cnb, false, zero, ctr, H, w1, true, dm);
            const v3<float> ms = dm ? rodrigues<float>(m, w1, dt) : m + dt * w1;
            B[i] = ms.x; B[N + i] = ms.y; B[2 * N + i] = ms.z;
        }
        __syncthreads();
        float proj = 0.f;
        if (own) {
            const v3<float> ms = mk3<float>(B[i], B[N + i], B[2 * N + i]);
            v3<float> nbv[6];
            bool nbp[6];
            float cnb[6];
            gather(B, ms, nbv, nbp, cnb);
            v3<float> w2;
            cell_field_nb<float, EXT>(fa, i, R, ms, nbv, nbp, cnb, false, zero, ctr, H, w2, true, dm);
            const v3<float> mn = dm ? rodrigues<float>(m, 0.5f * (w1 + w2), dt) : m + (0.5f * dt) * (w1 + w2);
            m = rsqrtf(dot(mn, mn)) * mn;
            A[i] = m.x; A[N + i] = m.y; A[2 * N + i] = m.z;
            proj = dot(m, ax);
        }
        if (a.trials) {
            for (int o = 16; o > 0; o >>= 1) proj += __shfl_xor_sync(0xffffffffu, proj, o);
            if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = proj;
            __syncthreads();
            if (threadIdx.x == 0) {
                float tot = 0.f;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_red[w];
                s_new = trial_check(a.tr, rp, a.rep + blockIdx.x, tot / (float)N, step + 1 - rp.step0, step + 1);
                s_red[0] = rp.active ? 1.f : 0.f;
            }
            __syncthreads();
            const int refill = s_new;
            const bool alive = s_red[0] != 0.f;
            if (refill) {
                rp = a.rep[blockIdx.x];   // the new trial's key, scales and start step
                fa.key0 = rp.key0;
                fa.key1 = rp.key1;
                fa.th_scale = rp.th_scale;
                fa.tq_base = rp.tq_base;
                if (own) {
                    m = mk3<float>(__ldg(a.tr.m_init + i), __ldg(a.tr.m_init + N + i), __ldg(a.tr.m_init + 2 * N + i));
                    A[i] = m.x; A[N + i] = m.y; A[2 * N + i] = m.z;
                }
            }
            __syncthreads();
            if (!alive) break;
        } else {
            __syncthreads();
        }
    }
    if (own) { mg[i] = m.x; mg[N + i] = m.y; mg[2 * N + i] = m.z; }
}

cudaError_t tile_kernel_attributes() {
    cudaError_t e = cudaFuncSetAttribute(tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(6 * kTileMaxCells * sizeof(float)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(6 * kTileMaxCells * sizeof(float)));
}

void tile_kernel_launch(const MacroArgs& a, cudaStream_t s) {
    const int nt = (a.nmax + 31) / 32 * 32;
    if (a.ext) tile_kernel<true><<<a.R, nt, 6 * a.nmax * sizeof(float), s>>>(a);
    else tile_kernel<false><<<a.R, nt, 6 * a.nmax * sizeof(float), s>>>(a);
}

// fixed-step bookkeeping of a block of n steps
__global__ void macro_advance_kernel(DevState* st, int n) {
    st->t += n * st->dt;
    st->step += n;
    st->accepted += n;
    st->attempts += n;
}

void macro_kernel_launch(const MacroArgs& a, cudaStream_t s) {
    const int nt = 32;
    if (a.ext) macro_kernel<true><<<(a.R + nt - 1) / nt, nt, 0, s>>>(a);
    else macro_kernel<false><<<(a.R + nt - 1) / nt, nt, 0, s>>>(a);
}

void macro_advance_launch(DevState* st, int nsteps, cudaStream_t s) {
    macro_advance_kernel<<<1, 1, 0, s>>>(st, nsteps);
}

}  // namespace mm
