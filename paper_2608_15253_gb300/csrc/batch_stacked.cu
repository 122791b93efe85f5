// Replica batching by size class (the "stacked" launch shape): the replicas
// of one grid size are stored back to back, so a stage runs, per class, the
// 2-D demag passes over all of its films at once (demag_apply_stacked2d) and
// then this kernel: field, torque and the Heun or Depondt-Mertens stage
// update of every cell of the class, one thread per cell, each replica with
// its own Philox key, temperature and current.  A few well-filled launches
// per class replace one CTA per replica.  With retire/refill on, idle slots
// are skipped and a per-slot stop test follows the corrector.
#include <cuda_runtime.h>

#include "batch_dev.cuh"

namespace mm {

template <bool EXT>
__global__ void __launch_bounds__(256) stacked_field_kernel(StackArgs a) {
    if (!a.st->active) return;
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int q = blockIdx.z;
    const int nx = a.nx, ny = a.ny;
    if (x >= nx || y >= ny) return;
    const RepDev& rp = a.rep[a.members[q]];
    if (!rp.active) return;              // an idle retire/refill slot keeps its state
    const long long N = (long long)nx * ny;
    const long long i = (long long)y * nx + x;
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
    const float* mE = (a.stage == 1 ? a.m0 : a.ms) + rp.off;
    const v3<float> m = ld3(mE, N, i);
    v3<float> nbv[6];
    bool nbp[6];
    float cnb[6];
    const float c_pair = __ldg(fa.cpair);
    const int pos[2] = {x, y}, dim[2] = {nx, ny};
    const long long stride[2] = {1, nx};
    const float hh[2] = {fa.hx, fa.hy};
#pragma unroll
    for (int d = 0; d < 2; ++d) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int sg = s == 0 ? 1 : -1;
            const int qd = pos[d] + sg;
            const int slot = 2 * d + s;
            const bool in = qd >= 0 && qd < dim[d];
            nbp[slot] = in;
            if (in) {
                nbv[slot] = ld3(mE, N, i + sg * stride[d]);
                cnb[slot] = c_pair;
            } else {
                nbv[slot] = ghost_value<float, EXT>(m, d, sg, hh[d], R.ratio, R.ratio_b);
                cnb[slot] = R.cg;
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        nbp[4 + s] = false;
        nbv[4 + s] = ghost_value<float, EXT>(m, 2, s == 0 ? 1 : -1, fa.hz, R.ratio, R.ratio_b);
        cnb[4 + s] = R.cg;
    }
    const bool dem = a.hd != nullptr;
    const v3<float> hd = dem ? ld3(a.hd + (long long)q * 3 * N, N, i) : mk3<float>(0.f, 0.f, 0.f);
    const long long step = a.st->step - rp.step0;
    v3<float> H, k;
    cell_field_nb<float, EXT>(fa, i, R, m, nbv, nbp, cnb, dem, hd, step, H, k, true, a.dm != 0);
    const float dt = (float)a.st->dt;
    if (a.stage == 1) {
        st3(a.k1 + rp.off, N, i, k);
        st3(a.ms + rp.off, N, i, a.dm ? rodrigues<float>(m, k, dt) : m + dt * k);
    } else {
        const v3<float> m0 = ld3(a.m0 + rp.off, N, i);
        const v3<float> kp = ld3(a.k1 + rp.off, N, i);
        const v3<float> mn = a.dm ? rodrigues<float>(m0, 0.5f * (kp + k), dt) : m0 + (0.5f * dt) * (kp + k);
        st3(a.m0 + rp.off, N, i, rsqrtf(dot(mn, mn)) * mn);
    }
}

// Retire/refill on the stacked shape (Results, "Replica batching"): after
// the corrector of every class, one CTA per slot forms the mean of m . axis
// over its replica, runs the stop test and, when a new trial takes the
// slot, writes its initial state.
__global__ void __launch_bounds__(256) stacked_trials_kernel(BatchArgs a) {
    if (!a.st->active) return;
    const int idx = blockIdx.x;
    const RepDev rp = a.rep[idx];
    if (!rp.active) return;                           // uniform over the CTA
    const long long N = (long long)rp.nx * rp.ny;
    const float* m = a.m0 + rp.off;
    const float ax = a.tr.axis[0], ay = a.tr.axis[1], az = a.tr.axis[2];
    float part = 0.f;
    for (long long i = threadIdx.x; i < N; i += 256) part += m[i] * ax + m[N + i] * ay + m[2 * N + i] * az;
    slot_retire_refill<256>(a, rp, idx, part, N, a.st->step);
}

void stacked_trials_launch(const BatchArgs& a, int R, cudaStream_t s) {
    stacked_trials_kernel<<<R, 256, 0, s>>>(a);
}

void stacked_field_launch(const StackArgs& a, int Rc, cudaStream_t s) {
    dim3 grid((a.nx + 31) / 32, (a.ny + 7) / 8, Rc);
    if (a.ext) stacked_field_kernel<true><<<grid, 256, 0, s>>>(a);
    else stacked_field_kernel<false><<<grid, 256, 0, s>>>(a);
}

}  // namespace mm
