// Replica-batched macrospins (Results, "Replica batching": the single-cell
// ensemble with local fields, spin torque and thermal noise, and the
// thermally assisted switching sweep).  A one-cell replica has no
// neighbours and no demag coupling, so its whole step is local: one thread
// per slot holds the moment in registers for a block of steps and runs the
// predictor, the corrector and, with retire/refill on, the stop test and
// the start of the next trial, without leaving the thread.
#include <cuda_runtime.h>

#include "batch_dev.cuh"

namespace mm {

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
    for (int s = 0; s < a.nsteps; ++s) {
        const long long step = step0 + s;
        const long long ctr = step - rp.step0;    // the trial's own step: its noise counter
        v3<float> H, w1, w2;
        const v3<float> hth = hot && fa.th_scale != 0.f ? thermal_h<float>(fa, 0, R, ctr) : mk3<float>(0.f, 0.f, 0.f);
        cell_field<float>(fa, 0, 0, 0, 0, 0, R, m, &hth, ctr, H, w1, true, dm);
        const v3<float> ms = dm ? rodrigues<float>(m, w1, dt) : m + dt * w1;
        cell_field<float>(fa, 0, 0, 0, 0, 0, R, ms, &hth, ctr, H, w2, true, dm);
        const v3<float> mn = dm ? rodrigues<float>(m, 0.5f * (w1 + w2), dt) : m + (0.5f * dt) * (w1 + w2);
        m = rsqrtf(dot(mn, mn)) * mn;
        if (a.trials) {
            if (trial_check(a.tr, rp, a.rep + r, dot(m, ax), step + 1 - rp.step0, step + 1)) {
                m = mk3<float>(__ldg(a.tr.m_init), __ldg(a.tr.m_init + 1), __ldg(a.tr.m_init + 2));
                fa.key0 = rp.key0;
                fa.key1 = rp.key1;
                fa.th_scale = rp.th_scale;
                fa.tq_base = rp.tq_base;
            }
            if (!rp.active) break;
        }
    }
    mp[0] = m.x;
    mp[1] = m.y;
    mp[2] = m.z;
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
    macro_kernel<<<(a.R + nt - 1) / nt, nt, 0, s>>>(a);
}

void macro_advance_launch(DevState* st, int nsteps, cudaStream_t s) {
    macro_advance_kernel<<<1, 1, 0, s>>>(st, nsteps);
}

}  // namespace mm
