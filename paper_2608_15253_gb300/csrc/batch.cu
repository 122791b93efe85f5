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
struct BatchHost {
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
    cudaMemsetAsync(a.next, 0, sizeof(int), c->stream);
    LaunchScope ls(c, stage == 1 ? "batch_stage1" : "batch_stage2", cells * (stage == 1 ? 36.0 : 48.0));
    if (b->nt == 512) batch_kernel_launch_512(a, b->blocks, b->smem, c->stream);
    else batch_kernel_launch_256(a, b->blocks, b->smem, c->stream);
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
    const size_t smem = batch_smem(*b, nt);
    return nt == 512 ? batch_kernel_occupancy_512(smem) : batch_kernel_occupancy_256(smem);
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
