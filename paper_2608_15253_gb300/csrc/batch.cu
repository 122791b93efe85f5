// Replica batching, host side: size classes, per-class tensor spectra,
// largest-first work order, CTA-private scratch, launch shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "batch_dev.cuh"

namespace mm {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// one size class of the stacked launch shape: members stored back to back
struct ClassHost {
    int nx = 0, ny = 0, Rc = 0;
    long long off0 = 0;            // element offset of the first member's block
    std::vector<int> members;      // replica indices in storage order
    int* d_members = nullptr;
    void* S = nullptr;             // spectra [member][3][PyA][Wk] complex
    float* Hd = nullptr;           // demag field [member][3][ny][nx]
};

struct BatchHost {
    std::vector<ClassHost> ch;
    bool stacked = false;          // launch shape: per-class passes instead of the persistent kernel
    std::vector<RepDev> rep;
    std::vector<ClsDev> cls;
    std::vector<DemagPlan> plans;
    std::vector<mm_grid> cgrid;
    std::vector<int> order;
    RepDev* d_rep = nullptr;
    ClsDev* d_cls = nullptr;
    int* d_order = nullptr;
    int* d_next = nullptr;     // per-stage work counters
    float2* d_scratch = nullptr;
    long long scratch_stride = 0;
    int nt = 256;
    int blocks = 0;
    size_t smem = 0;
    double sigma_V = 1.0;   // cell volume used in the thermal scale
    bool macro = false;     // every replica one cell, no demag: macro_kernel
    bool tile = false;      // no demag, every replica at most kTileMaxCells cells: tile_kernel
    int nmax = 0;           // largest replica (cells)
    // retire/refill
    bool trials_on = false;
    TrialDev tr{};
    float* d_trJ = nullptr;
    float* d_trT = nullptr;
    float* d_minit = nullptr;
    unsigned long long* d_trc = nullptr;   // next, done
    long long* d_trsteps = nullptr;
    int* d_trstop = nullptr;
};

static size_t batch_smem(const BatchHost& b, int NT) {
    size_t mx = 0;
    for (const ClsDev& cd : b.cls) {
        const bool ct = b_compiled(cd.Lh, cd.Py);
        const size_t x = (size_t)std::min(b_rows_x(cd.Lh, NT, ct), 3 * cd.ny) * (cd.Lh + 1) * 8;
        const size_t y = (size_t)3 * b_tk(cd.Py, NT, ct) * (cd.Py + 1) * 8;
        const size_t cc = (size_t)3 * std::min(std::max(1, b_rows_c(cd.Lh, NT, ct)), cd.ny) * (cd.Lh + 1) * 8;
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
    cudaFree(b->d_next);
    cudaFree(b->d_scratch);
    cudaFree(b->d_trJ);
    cudaFree(b->d_trT);
    cudaFree(b->d_minit);
    cudaFree(b->d_trc);
    cudaFree(b->d_trsteps);
    cudaFree(b->d_trstop);
    for (auto& k : b->ch) {
        cudaFree(k.d_members);
        cudaFree(k.S);
        cudaFree(k.Hd);
    }
    for (auto& p : b->plans) demag_free_plan(p);
    delete b;
}

// Builds size classes, per-class tensor spectra and the device tables.
mm_status batch_setup(mm_ctx* c, BatchHost* b, const std::vector<mm_grid>& grids, const std::vector<uint64_t>& keys,
                      bool demag) {
    const int R = (int)grids.size();
    b->rep.resize(R);
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
        d.off = c->roff[r];
        d.active = 1;
        d.trial = -1;
        d.step0 = 0;
        d.key0 = (uint32_t)(keys[r] & 0xFFFFFFFFull);
        d.key1 = (uint32_t)(keys[r] >> 32);
        b->rep[r] = d;
    }
    // size classes for the stacked launch shape: members in storage order
    b->ch.assign(b->cgrid.size(), ClassHost{});
    {
        std::vector<int> idx(R);
        for (int r = 0; r < R; ++r) idx[r] = r;
        std::sort(idx.begin(), idx.end(), [&](int x, int y) { return b->rep[x].off < b->rep[y].off; });
        for (int r : idx) {
            ClassHost& k = b->ch[b->rep[r].cls];
            if (k.members.empty()) {
                k.nx = b->rep[r].nx;
                k.ny = b->rep[r].ny;
                k.off0 = b->rep[r].off;
            }
            k.members.push_back(r);
        }
        for (ClassHost& k : b->ch) {
            k.Rc = (int)k.members.size();
            cudaError_t e = cudaMalloc(&k.d_members, sizeof(int) * k.Rc);
            if (e != cudaSuccess) return cuda_check(c, e, "class members");
            cudaMemcpy(k.d_members, k.members.data(), sizeof(int) * k.Rc, cudaMemcpyHostToDevice);
        }
    }
    b->macro = !demag;
    b->nmax = 0;
    for (const RepDev& d : b->rep) {
        b->macro = b->macro && d.nx == 1 && d.ny == 1;
        b->nmax = std::max(b->nmax, d.nx * d.ny);
    }
    b->tile = !demag && !b->macro && b->nmax <= kTileMaxCells;
    if (b->tile) {
        cudaError_t ea = tile_kernel_attributes();
        if (ea != cudaSuccess) return cuda_check(c, ea, "tile kernel attributes");
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
    // work order: replicas sorted by size, the largest paired with the
    // smallest of the head so the CTA-private spectra in flight at any time
    // stay within L2; the smallest quarter closes the order so the dynamic
    // schedule ends on short jobs
    std::vector<int> desc(R);
    for (int r = 0; r < R; ++r) desc[r] = r;
    std::stable_sort(desc.begin(), desc.end(), [&](int x, int y) {
        return (long long)b->rep[x].nx * b->rep[x].ny > (long long)b->rep[y].nx * b->rep[y].ny;
    });
    const int tail = R / 4, head = R - tail;
    b->order.clear();
    for (int lo = 0, hi = head - 1; lo <= hi; ++lo, --hi) {
        b->order.push_back(desc[lo]);
        if (hi != lo) b->order.push_back(desc[hi]);
    }
    for (int q = head; q < R; ++q) b->order.push_back(desc[q]);
    cudaError_t e = cudaMalloc(&b->d_rep, sizeof(RepDev) * R);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_cls, sizeof(ClsDev) * b->cls.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int) * R);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(int) * 2);
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
    e = batch_kernel_attributes_256();
    if (e == cudaSuccess) e = batch_kernel_attributes_512();
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

// field parameters shared by every replica (per-replica ones are set in
// the kernels)
static void batch_field_args(mm_ctx* c, FieldArgs<float>& f) {
    const mm_grid& g = c->grid;
    f.lut = (const Region<float>*)c->d_lut;
    f.cpair = (const float*)c->d_cpair;
    f.nreg = c->nreg;
    f.hx = (float)g.dx; f.hy = (float)g.dy; f.hz = (float)g.dz;
    f.ix2 = (float)(1.0 / (g.dx * g.dx)); f.iy2 = (float)(1.0 / (g.dy * g.dy)); f.iz2 = (float)(1.0 / (g.dz * g.dz));
    for (int d = 0; d < 3; ++d) f.hext[d] = (float)c->Hext[d];
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
    f.cubic_w1 = f.cubic_w2 = 1.f;
    for (int k = 0; k < 6; ++k) f.strain[k] = (float)c->strain[k];
    f.strain_cell = nullptr;
}

static void launch_stage(mm_ctx* c, BatchHost* b, int stage) {
    BatchArgs a{};
    a.rep = b->d_rep;
    a.cls = b->d_cls;
    a.order = b->d_order;
    a.next = b->d_next + (stage - 1);
    a.R = (int)b->rep.size();
    a.m0 = (float*)c->d_m;
    a.ms = (float*)c->d_mtmp;
    a.k1 = (float*)c->d_k[0];
    a.scratch = b->d_scratch;
    a.scratch_stride = b->scratch_stride;
    a.demag = (c->terms & MM_TERM_DEMAG) ? 1 : 0;
    a.stage = stage;
    a.dm = c->integrator == MM_DM ? 1 : 0;
    a.trials = b->trials_on ? 1 : 0;
    a.tr = b->tr;
    a.st = c->d_state;
    FieldArgs<float>& f = a.fa;
    batch_field_args(c, f);
    f.terms = c->terms & ~MM_TERM_DEMAG;
    f.terms |= a.demag ? MM_TERM_DEMAG : 0;
    double cells = 0;
    for (const RepDev& r : b->rep) cells += (double)r.nx * r.ny;
    cudaMemsetAsync(a.next, 0, sizeof(int), c->stream);
    LaunchScope ls(c, stage == 1 ? "batch_stage1" : "batch_stage2", cells * (stage == 1 ? 36.0 : 48.0));
    if (b->nt == 512) batch_kernel_launch_512(a, b->blocks, b->smem, c->stream);
    else batch_kernel_launch_256(a, b->blocks, b->smem, c->stream);
}

bool batch_is_fused(BatchHost* b) { return b->macro || b->tile; }

// one launch of `nsteps` fused steps of every replica (one-cell or small
// films without demag), then the step bookkeeping
void batch_macro_steps(mm_ctx* c, BatchHost* b, int nsteps) {
    MacroArgs a{};
    a.rep = b->d_rep;
    a.R = (int)b->rep.size();
    a.m = (float*)c->d_m;
    a.dm = c->integrator == MM_DM ? 1 : 0;
    a.trials = b->trials_on ? 1 : 0;
    a.tr = b->tr;
    a.st = c->d_state;
    a.nsteps = nsteps;
    a.nmax = b->nmax;
    a.ext = c->ext_terms ? 1 : 0;
    batch_field_args(c, a.fa);
    a.fa.terms = c->terms & ~MM_TERM_DEMAG;
    if (b->macro) {
        LaunchScope ls(c, "macro_steps", (double)a.R * 24.0);
        macro_kernel_launch(a, c->stream);
    } else {
        double cells = 0;
        for (const RepDev& r : b->rep) cells += (double)r.nx * r.ny;
        LaunchScope ls(c, "tile_steps", cells * 24.0);
        tile_kernel_launch(a, c->stream);
    }
    LaunchScope ls(c, "macro_advance", 0.0);
    macro_advance_launch(c->d_state, nsteps, c->stream);
}

// Retire/refill (Results, "Replica batching"): trial tables, results, and
// the first min(R, n_trials) trials loaded into the slots at the current
// global step.
mm_status batch_trials_start(mm_ctx* c, BatchHost* b, const mm_trials* sp, long long step_now) {
    const long long n = sp->n_trials;
    const int R = (int)b->rep.size();
    const long long N = (long long)b->rep[0].nx * b->rep[0].ny;
    cudaFree(b->d_trJ); cudaFree(b->d_trT); cudaFree(b->d_minit); cudaFree(b->d_trc);
    cudaFree(b->d_trsteps); cudaFree(b->d_trstop);
    b->d_trJ = b->d_trT = b->d_minit = nullptr;
    b->d_trc = nullptr; b->d_trsteps = nullptr; b->d_trstop = nullptr;
    cudaError_t e = cudaMalloc(&b->d_trJ, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_trT, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_minit, sizeof(float) * 3 * N);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_trc, sizeof(unsigned long long) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_trsteps, sizeof(long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_trstop, sizeof(int) * n);
    if (e != cudaSuccess) return cuda_check(c, e, "trial tables");
    std::vector<float> J(n), T(n);
    for (long long q = 0; q < n; ++q) { J[q] = (float)sp->J[q]; T[q] = (float)sp->T[q]; }
    std::vector<float> m0(3 * N, 0.f);
    for (long long i = 0; i < N; ++i) {
        const double x = sp->m_init[i], y = sp->m_init[N + i], z = sp->m_init[2 * N + i];
        const double nn = std::sqrt(x * x + y * y + z * z);
        if (nn > 0) { m0[i] = (float)(x / nn); m0[N + i] = (float)(y / nn); m0[2 * N + i] = (float)(z / nn); }
    }
    const unsigned long long cnt[2] = {(unsigned long long)std::min<long long>(R, n), 0ull};
    std::vector<long long> steps(n, -1);
    cudaMemcpy(b->d_trJ, J.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_trT, T.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_minit, m0.data(), sizeof(float) * 3 * N, cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_trc, cnt, sizeof(cnt), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_trsteps, steps.data(), sizeof(long long) * n, cudaMemcpyHostToDevice);
    cudaMemset(b->d_trstop, 0, sizeof(int) * n);
    const mm_grid& g = b->cgrid[0];
    const mm_torque& q = c->tq;
    const double tF = q.t_F > 0 ? q.t_F : g.nz * g.dz;
    TrialDev& t = b->tr;
    t = TrialDev{};
    t.n_trials = n;
    t.max_steps = sp->max_steps;
    t.J = b->d_trJ;
    t.T = b->d_trT;
    t.m_init = b->d_minit;
    const double an = std::sqrt(sp->axis[0] * sp->axis[0] + sp->axis[1] * sp->axis[1] + sp->axis[2] * sp->axis[2]);
    for (int d = 0; d < 3; ++d) t.axis[d] = (float)(sp->axis[d] / an);
    t.threshold = (float)sp->threshold;
    t.base_seed = sp->base_seed;
    t.tq_per_J = (float)(kHbar / (kQe * kMu0 * tF));
    t.th_per_sqrtT = (float)(1.0 / std::sqrt(g.dx * g.dy * g.dz * c->cfg.dt));
    t.refill = sp->refill ? 1 : 0;
    t.next = b->d_trc;
    t.done = b->d_trc + 1;
    t.steps = b->d_trsteps;
    t.stopped = b->d_trstop;
    std::vector<float> all(3 * c->Ntot);
    e = cudaMemcpy(all.data(), c->d_m, sizeof(float) * 3 * c->Ntot, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(c, e, "trial state");
    for (int r = 0; r < R; ++r) {
        RepDev& d = b->rep[r];
        if (r < n) {
            const unsigned long long key = splitmix64_dev(sp->base_seed + (unsigned long long)r);
            d.active = 1;
            d.trial = r;
            d.step0 = step_now;
            d.key0 = (uint32_t)(key & 0xFFFFFFFFull);
            d.key1 = (uint32_t)(key >> 32);
            d.th_scale = T[r] > 0 ? (float)std::sqrt((double)T[r]) * t.th_per_sqrtT : 0.f;
            d.tq_base = J[r] * t.tq_per_J;
            std::copy(m0.begin(), m0.end(), all.begin() + d.off);
        } else {
            d.active = 0;
            d.trial = -1;
        }
    }
    cudaMemcpy(c->d_m, all.data(), sizeof(float) * 3 * c->Ntot, cudaMemcpyHostToDevice);
    b->trials_on = true;
    return cuda_check(c, cudaMemcpy(b->d_rep, b->rep.data(), sizeof(RepDev) * R, cudaMemcpyHostToDevice),
                      "trial slots");
}

mm_status batch_trials_result(mm_ctx* c, BatchHost* b, long long* steps, int* stopped, long long* done) {
    if (!b->trials_on) return set_error(c, MM_ERR_STATE, "no trials started");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    const long long n = b->tr.n_trials;
    if (e == cudaSuccess && steps) e = cudaMemcpy(steps, b->d_trsteps, sizeof(long long) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && stopped) e = cudaMemcpy(stopped, b->d_trstop, sizeof(int) * n, cudaMemcpyDeviceToHost);
    unsigned long long cnt[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(cnt, b->d_trc, sizeof(cnt), cudaMemcpyDeviceToHost);
    if (done) *done = (long long)cnt[1];
    return cuda_check(c, e, "trial results");
}

bool batch_trials_on(BatchHost* b) { return b->trials_on; }

// stacked launch shape: per size class, the 2-D demag passes over all of
// its films, then the field + stage kernel over all of its cells
static void stacked_stage(mm_ctx* c, BatchHost* b, int stage) {
    const bool demag = (c->terms & MM_TERM_DEMAG) != 0;
    for (size_t q = 0; q < b->ch.size(); ++q) {
        ClassHost& k = b->ch[q];
        const float* in = (const float*)(stage == 1 ? c->d_m : c->d_mtmp) + k.off0;
        if (demag) demag_apply_stacked2d(c, b->plans[q], in, k.Hd, k.S, k.nx, k.ny, k.Rc);
        StackArgs a{};
        a.rep = b->d_rep;
        a.members = k.d_members;
        a.nx = k.nx;
        a.ny = k.ny;
        a.m0 = (float*)c->d_m;
        a.ms = (float*)c->d_mtmp;
        a.k1 = (float*)c->d_k[0];
        a.hd = demag ? k.Hd : nullptr;
        batch_field_args(c, a.fa);
        a.fa.terms = c->terms;
        a.stage = stage;
        a.dm = c->integrator == MM_DM ? 1 : 0;
        a.ext = c->ext_terms ? 1 : 0;
        a.st = c->d_state;
        const double cells = (double)k.Rc * k.nx * k.ny;
        LaunchScope ls(c, stage == 1 ? "stacked_field1" : "stacked_field2",
                       cells * (stage == 1 ? 36.0 : 48.0) + (demag ? cells * 12.0 : 0.0));
        stacked_field_launch(a, k.Rc, c->stream);
    }
}

void batch_step(mm_ctx* c, BatchHost* b) {
    if (b->stacked) {
        heun_batch_begin(c);
        stacked_stage(c, b, 1);
        stacked_stage(c, b, 2);
        if (b->trials_on) {
            BatchArgs a{};
            a.rep = b->d_rep;
            a.m0 = (float*)c->d_m;
            a.trials = 1;
            a.tr = b->tr;
            a.st = c->d_state;
            LaunchScope ls(c, "stacked_trials", 12.0 * (double)c->Ntot);
            stacked_trials_launch(a, (int)b->rep.size(), c->stream);
        }
        heun_batch_advance(c);
        return;
    }
    heun_batch_begin(c);
    launch_stage(c, b, 1);
    launch_stage(c, b, 2);
    heun_batch_advance(c);
}

// nt = 0 selects the stacked launch shape (its per-class buffers are
// allocated here, outside any graph capture; on failure the persistent
// kernel stays)
void batch_set_shape(BatchHost* b, int nt, int blocks) {
    if (nt == 0) {
        bool ok = true;
        for (size_t q = 0; q < b->ch.size() && ok; ++q) {
            ClassHost& k = b->ch[q];
            const DemagPlan& p = b->plans[q];
            if (!p.on || (k.S && k.Hd)) continue;
            cudaFree(k.S);
            cudaFree(k.Hd);
            k.S = nullptr;
            k.Hd = nullptr;
            const size_t sb = sizeof(float2) * (size_t)k.Rc * 3 * p.PyA * p.Wk;
            const size_t hb = sizeof(float) * (size_t)k.Rc * 3 * k.nx * k.ny;
            ok = cudaMalloc(&k.S, sb) == cudaSuccess && cudaMalloc(&k.Hd, hb) == cudaSuccess;
            if (!ok) {   // neither half of a pair is kept
                cudaFree(k.S);
                cudaFree(k.Hd);
                k.S = nullptr;
                k.Hd = nullptr;
            }
        }
        if (ok) {
            b->stacked = true;
            return;
        }
        cudaGetLastError();
        nt = 256;
        blocks = std::max(1, std::min((int)b->rep.size(), 304));
    }
    b->stacked = false;
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
    const size_t smem = batch_smem(*b, nt);
    return nt == 512 ? batch_kernel_occupancy_512(smem) : batch_kernel_occupancy_256(smem);
}

void batch_get_shape(BatchHost* b, int* nt, int* blocks) {
    *nt = b->stacked ? 0 : b->nt;
    *blocks = b->stacked ? 0 : b->blocks;
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
