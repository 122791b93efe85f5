// Replica batching (Methods, "Replica batching"): R independent thin-film
// replicas (nz = 1) of possibly different sizes advance together, each with
// its own Philox key, temperature and current density.  One persistent
// launch per Heun stage: every CTA takes whole replicas from a
// largest-first work order and runs, for each, the three demag phases
// (row R2C, column convolution with the size class's tensor spectrum,
// row C2R) and the fused field + torque + stage update.  The replica's
// half spectrum lives in a CTA-private scratch slab (small enough to stay
// in L2); every transform runs in shared memory.  No grid-wide
// synchronisation is needed: a CTA owns its replica for the whole stage.
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

constexpr int kMaxVB = 24;

struct RepDev {
    int nx, ny, cls, pad;
    long long off;          // element offset of the replica's [3][ny][nx] block
    uint32_t key0, key1;    // Philox key
    float th_scale;         // sqrt(T / (V dt))
    float tq_base;          // hbar J / (e mu0 t_F)
};

struct ClsDev {
    int nx, ny, Lh, Py, Kx, Wk, Ky;
    const float* khat;      // [4][Ky][Wk]: xx, yy, zz, xy
    const float2* twx;      // exp(-2 pi i q / (2 Lh))
    const float2* twy;      // exp(-2 pi i q / Py)
    Plan ph, py;            // runtime plans (generic path)
};

struct BatchArgs {
    const RepDev* rep;
    const ClsDev* cls;
    const int* order;
    int R;
    float* m0;              // state
    float* ms;              // predictor state
    float* k1;              // predictor slope
    float2* scratch;
    long long scratch_stride;
    FieldArgs<float> fa;    // shared field parameters (per-replica fields set in-kernel)
    int demag;
    int stage;              // 1: predictor, 2: corrector
    const DevState* st;
};

__host__ __device__ constexpr int b_rows_x(int Lh, int NT) { return (kMaxVB * NT) / Lh; }
__host__ __device__ inline int b_tk(int Py, int NT) {
    int cap = (kMaxVB * NT) / (3 * Py), tk = 1;
    while (tk * 2 <= cap && tk * 2 <= 16) tk *= 2;
    return tk;
}
__host__ __device__ constexpr int b_rows_c(int Lh, int NT) { return (kMaxVB * NT) / (3 * Lh); }

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

// One replica, one stage.  LX / LY: compile-time half length / column
// length (0 = runtime plan).
template <int LX, int LY, int NT>
__device__ void replica_stage(const BatchArgs& a, const RepDev& rp, const ClsDev& cd, float2* S, float2* sm,
                              long long step, float dt) {
    const int nx = rp.nx, ny = rp.ny;
    const long long N = (long long)nx * ny;
    float* mE = (a.stage == 1 ? a.m0 : a.ms) + rp.off;
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
    const int Lh = LX > 0 ? LX : cd.Lh;
    const int Py = LY > 0 ? LY : cd.Py;
    const int pitch = Lh + 1;
    float* smr = reinterpret_cast<float*>(sm);
    const float ms = R.Ms;

    if (a.demag) {
        // ---- phase X: rows (c, y) -> half spectra in S[(c ny + y) Wk + kx]
        const int RB = b_rows_x(Lh, NT);
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
        // ---- phase Y: columns, FFT along y, tensor multiply, inverse, keep ny
        const int TK = b_tk(Py, NT);
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
    // ---- phase C: C2R rows of a block of y (three components) + field + update
    const int RBc = a.demag ? max(1, b_rows_c(Lh, NT)) : ny;
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
            cell_field<float>(fa, x, y, 0, i, 0, R, m, a.demag ? &hd : nullptr, step, H, k, true);
            if (a.stage == 1) {
                st3(a.k1 + rp.off, N, i, k);
                st3(a.ms + rp.off, N, i, m + dt * k);
            } else {
                const v3<float> m0 = ld3(a.m0 + rp.off, N, i);
                const v3<float> kp = ld3(a.k1 + rp.off, N, i);
                const v3<float> mn = m0 + (0.5f * dt) * (kp + k);
                st3(a.m0 + rp.off, N, i, rsqrtf(dot(mn, mn)) * mn);
            }
        }
        __syncthreads();
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) batch_stage_kernel(BatchArgs a) {
    if (!a.st->active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    const long long step = a.st->step;
    const float dt = (float)a.st->dt;
    float2* S = a.scratch + blockIdx.x * a.scratch_stride;
    for (int w = blockIdx.x; w < a.R; w += gridDim.x) {
        const RepDev rp = a.rep[a.order[w]];
        const ClsDev& cd = a.cls[rp.cls];
        const int key = cd.Lh * 10000 + cd.Py;
        switch (key) {
#define MM_B(lh, py) case lh * 10000 + py: replica_stage<lh, py, NT>(a, rp, cd, S, sm, step, dt); break;
            MM_B(16, 32) MM_B(32, 64) MM_B(48, 96) MM_B(64, 128) MM_B(96, 192) MM_B(128, 256) MM_B(256, 512)
#undef MM_B
            default: replica_stage<0, 0, NT>(a, rp, cd, S, sm, step, dt); break;
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct BatchHost {
    std::vector<RepDev> rep;
    std::vector<ClsDev> cls;
    std::vector<DemagPlan> plans;
    std::vector<mm_grid> cgrid;
    std::vector<int> order;
    RepDev* d_rep = nullptr;
    ClsDev* d_cls = nullptr;
    int* d_order = nullptr;
    float2* d_scratch = nullptr;
    long long scratch_stride = 0;
    int nt = 256;
    int blocks = 0;
    size_t smem = 0;
    double sigma_V = 1.0;   // cell volume used in the thermal scale
};

static size_t batch_smem(const BatchHost& b, int NT) {
    size_t mx = 0;
    for (const ClsDev& cd : b.cls) {
        const size_t x = (size_t)std::min(b_rows_x(cd.Lh, NT), 3 * cd.ny) * (cd.Lh + 1) * 8;
        const size_t y = (size_t)3 * b_tk(cd.Py, NT) * (cd.Py + 1) * 8;
        const size_t cc = (size_t)3 * std::min(std::max(1, b_rows_c(cd.Lh, NT)), cd.ny) * (cd.Lh + 1) * 8;
        mx = std::max(mx, std::max(x, std::max(y, cc)));
    }
    return std::max<size_t>(mx, 16);
}

BatchHost* batch_new() { return new BatchHost(); }

void batch_free(BatchHost* b) {
    if (!b) return;
    cudaFree(b->d_rep);
    cudaFree(b->d_cls);
    cudaFree(b->d_order);
    cudaFree(b->d_scratch);
    for (auto& p : b->plans) demag_free_plan(p);
    delete b;
}

// Builds size classes, per-class tensor spectra and the device tables.
mm_status batch_setup(mm_ctx* c, BatchHost* b, const std::vector<mm_grid>& grids, const std::vector<uint64_t>& keys,
                      bool demag) {
    const int R = (int)grids.size();
    b->rep.resize(R);
    long long off = 0;
    for (int r = 0; r < R; ++r) {
        const mm_grid& g = grids[r];
        int cls = -1;
        for (size_t q = 0; q < b->cgrid.size(); ++q) {
            const mm_grid& h = b->cgrid[q];
            if (h.nx == g.nx && h.ny == g.ny && h.dx == g.dx && h.dy == g.dy && h.dz == g.dz) cls = (int)q;
        }
        if (cls < 0) {
            b->cgrid.push_back(g);
            cls = (int)b->cgrid.size() - 1;
        }
        RepDev d{};
        d.nx = g.nx;
        d.ny = g.ny;
        d.cls = cls;
        d.off = off;
        d.key0 = (uint32_t)(keys[r] & 0xFFFFFFFFull);
        d.key1 = (uint32_t)(keys[r] >> 32);
        b->rep[r] = d;
        off += 3LL * g.nx * g.ny;
    }
    long long max_spec = 1;
    for (size_t q = 0; q < b->cgrid.size(); ++q) {
        const mm_grid& g = b->cgrid[q];
        ClsDev cd{};
        cd.nx = g.nx;
        cd.ny = g.ny;
        DemagPlan p{};
        if (demag) {
            mm_status s = demag_setup_for(c, g, &p);
            if (s != MM_OK) return s;
            cd.Lh = p.Lh;
            cd.Py = p.Py;
            cd.Kx = p.Kx;
            cd.Wk = p.Wk;
            cd.Ky = p.Py / 2 + 1;
            cd.khat = (const float*)p.khat;
            cd.twx = (const float2*)p.tw_x;
            cd.twy = (const float2*)p.tw_y;
            make_plan(cd.Lh, &cd.ph);
            make_plan(cd.Py, &cd.py);
            max_spec = std::max(max_spec, 3LL * g.ny * cd.Wk);
        }
        b->plans.push_back(p);
        b->cls.push_back(cd);
    }
    b->order.resize(R);
    for (int r = 0; r < R; ++r) b->order[r] = r;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return (long long)b->rep[x].nx * b->rep[x].ny > (long long)b->rep[y].nx * b->rep[y].ny;
    });
    cudaError_t e = cudaMalloc(&b->d_rep, sizeof(RepDev) * R);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_cls, sizeof(ClsDev) * b->cls.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int) * R);
    if (e != cudaSuccess) return cuda_check(c, e, "batch tables");
    cudaMemcpy(b->d_cls, b->cls.data(), sizeof(ClsDev) * b->cls.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * R, cudaMemcpyHostToDevice);
    // launch shape: the default; batch_autotune may replace it
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->nt = 256;
    b->smem = batch_smem(*b, b->nt);
    b->blocks = std::min(R, sms * 2);
    b->scratch_stride = (max_spec + 31) / 32 * 32;
    const int max_blocks = std::min(R, sms * 8);
    if (demag) {
        e = cudaMalloc(&b->d_scratch, sizeof(float2) * b->scratch_stride * max_blocks);
        if (e != cudaSuccess) return cuda_check(c, e, "batch scratch");
    }
    e = cudaFuncSetAttribute(batch_stage_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_stage_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    return cuda_check(c, e, "batch kernel attributes");
}

// per-replica temperature / current -> device descriptors
mm_status batch_upload(mm_ctx* c, BatchHost* b, const std::vector<double>& T, const std::vector<double>& J) {
    const mm_torque& q = c->tq;
    for (size_t r = 0; r < b->rep.size(); ++r) {
        const mm_grid& g = b->cgrid[b->rep[r].cls];
        const double V = g.dx * g.dy * g.dz;
        b->rep[r].th_scale = T[r] > 0 ? (float)std::sqrt(T[r] / (V * c->cfg.dt)) : 0.f;
        const double tF = q.t_F > 0 ? q.t_F : g.nz * g.dz;
        b->rep[r].tq_base = (float)(kHbar * J[r] / (kQe * kMu0 * tF));
    }
    return cuda_check(c, cudaMemcpy(b->d_rep, b->rep.data(), sizeof(RepDev) * b->rep.size(), cudaMemcpyHostToDevice),
                      "batch descriptors");
}

static void launch_stage(mm_ctx* c, BatchHost* b, int stage) {
    BatchArgs a{};
    a.rep = b->d_rep;
    a.cls = b->d_cls;
    a.order = b->d_order;
    a.R = (int)b->rep.size();
    a.m0 = (float*)c->d_m;
    a.ms = (float*)c->d_mtmp;
    a.k1 = (float*)c->d_k[0];
    a.scratch = b->d_scratch;
    a.scratch_stride = b->scratch_stride;
    a.demag = (c->terms & MM_TERM_DEMAG) ? 1 : 0;
    a.stage = stage;
    a.st = c->d_state;
    FieldArgs<float>& f = a.fa;
    const mm_grid& g = c->grid;
    f.lut = (const Region<float>*)c->d_lut;
    f.cpair = (const float*)c->d_cpair;
    f.nreg = c->nreg;
    f.hx = (float)g.dx; f.hy = (float)g.dy; f.hz = (float)g.dz;
    f.ix2 = (float)(1.0 / (g.dx * g.dx)); f.iy2 = (float)(1.0 / (g.dy * g.dy)); f.iz2 = (float)(1.0 / (g.dz * g.dz));
    for (int d = 0; d < 3; ++d) f.hext[d] = (float)c->Hext[d];
    f.terms = c->terms & ~MM_TERM_DEMAG;
    f.terms |= a.demag ? MM_TERM_DEMAG : 0;
    f.st = c->d_state;
    const mm_torque& q = c->tq;
    f.tq = q.kind;
    double pn = std::sqrt(q.p[0] * q.p[0] + q.p[1] * q.p[1] + q.p[2] * q.p[2]);
    if (pn == 0) pn = 1;
    for (int d = 0; d < 3; ++d) f.p[d] = (float)(q.p[d] / pn);
    f.theta_half = (float)(0.5 * q.theta_SH);
    f.fl_ratio = (float)q.fl_ratio;
    f.P = (float)q.P;
    f.L2 = (float)(q.Lambda * q.Lambda);
    f.eps_p = (float)q.eps_prime;
    double cells = 0;
    for (const RepDev& r : b->rep) cells += (double)r.nx * r.ny;
    LaunchScope ls(c, stage == 1 ? "batch_stage1" : "batch_stage2", cells * (stage == 1 ? 36.0 : 48.0));
    if (b->nt == 512) batch_stage_kernel<512><<<b->blocks, 512, b->smem, c->stream>>>(a);
    else batch_stage_kernel<256><<<b->blocks, 256, b->smem, c->stream>>>(a);
}

void batch_heun_step(mm_ctx* c, BatchHost* b) {
    heun_batch_begin(c);
    launch_stage(c, b, 1);
    launch_stage(c, b, 2);
    heun_batch_advance(c);
}

void batch_set_shape(BatchHost* b, int nt, int blocks) {
    b->nt = nt;
    b->blocks = blocks;
    b->smem = batch_smem(*b, nt);
}

int batch_max_blocks(BatchHost* b) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::min((int)b->rep.size(), sms * 8);
}

size_t batch_smem_for(BatchHost* b, int nt) { return batch_smem(*b, nt); }

const DemagPlan& batch_plan(BatchHost* b, int cls) { return b->plans[cls]; }

int batch_occupancy(BatchHost* b, int nt) {
    int nb = 0;
    const size_t smem = batch_smem(*b, nt);
    if (nt == 512) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_stage_kernel<512>, 512, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_stage_kernel<256>, 256, smem);
    return nb;
}

void batch_get_shape(BatchHost* b, int* nt, int* blocks) {
    *nt = b->nt;
    *blocks = b->blocks;
}

// signature of the batch for the autotuner cache: sizes histogram + demag flag
std::string batch_signature(BatchHost* b, unsigned terms) {
    std::vector<std::pair<long long, int>> h;
    for (const RepDev& r : b->rep) {
        const long long key = (long long)r.nx * 100000 + r.ny;
        bool f = false;
        for (auto& e : h) if (e.first == key) { e.second++; f = true; }
        if (!f) h.push_back({key, 1});
    }
    std::sort(h.begin(), h.end());
    std::string s = "t" + std::to_string(terms);
    for (auto& e : h) s += "_" + std::to_string(e.first / 100000) + "x" + std::to_string(e.first % 100000) + "n" + std::to_string(e.second);
    return s;
}

int batch_class_of(BatchHost* b, int r) { return b->rep[r].cls; }

}  // namespace mm
