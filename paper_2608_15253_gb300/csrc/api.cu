// C ABI of libmm (include/mm.h): context lifetime, material regions, state
// transfer, stepping (chunks of integrator attempts replayed from CUDA
// graphs), observables, checkpoints, profiling and host-side fault
// injection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace mm {

mm_status demag_kernel_copy(mm_ctx* c, double* out, size_t n_out, int* dims);

static thread_local std::string g_create_error;

mm_status set_error(mm_ctx* c, mm_status s, const std::string& msg) {
    if (c) c->last_error = msg;
    else g_create_error = msg;
    return s;
}

mm_status cuda_check(mm_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MM_OK;
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return set_error(c, e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA, msg);
}

LaunchScope::LaunchScope(mm_ctx* cc, const char* name, double bytes) : c(cc), slot(-1) {
    c->launches += 1;
    if (!c->profiling) return;
    for (size_t q = 0; q < c->prof.size(); ++q)
        if (c->prof[q].name == name) slot = (int)q;
    if (slot < 0) {
        ProfileSlot p;
        p.name = name;
        c->prof.push_back(p);
        slot = (int)c->prof.size() - 1;
    }
    c->prof[slot].bytes = bytes;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
}

LaunchScope::~LaunchScope() {
    if (!c->profiling || slot < 0) return;
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c->prof[slot].launches += 1;
    c->prof[slot].total_ms += ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

template <typename T>
static Region<T> region_coeffs(const RegionHost& r, double /*V*/) {
    Region<T> o{};
    const bool present = r.Ms > 0;
    const double imu = present ? 1.0 / (kMu0 * r.Ms) : 0.0;
    o.present = present ? (T)1 : (T)0;
    o.inv_mu0Ms = (T)imu;
    o.Ms = (T)r.Ms;
    o.cg = (T)(2.0 * r.A * imu);
    o.ratio = r.A > 0 ? (T)(r.D / (2.0 * r.A)) : (T)0;
    o.dmi = (T)(2.0 * r.D * imu);
    o.ku = (T)(2.0 * r.Ku1 * imu);
    double un = std::sqrt(r.u[0] * r.u[0] + r.u[1] * r.u[1] + r.u[2] * r.u[2]);
    if (un == 0) un = 1;
    o.ux = (T)(r.u[0] / un);
    o.uy = (T)(r.u[1] / un);
    o.uz = (T)(r.u[2] / un);
    o.alpha = (T)r.alpha;
    o.gm = (T)(kGamma0 * kMu0 / (1.0 + r.alpha * r.alpha));
    o.sigma0 = present ? (T)std::sqrt(2.0 * r.alpha * kKB / (kMu0 * kMu0 * r.Ms * kGamma0)) : (T)0;
    o.inv_Ms = present ? (T)(1.0 / r.Ms) : (T)0;
    o.ratio_b = r.A > 0 ? (T)(r.Db / (2.0 * r.A)) : (T)0;
    o.dmib = (T)(2.0 * r.Db * imu);
    o.kc1 = (T)(2.0 * r.Kc1 * imu);
    o.kc2 = (T)(2.0 * r.Kc2 * imu);
    // cubic axes: c1 normalised, c2 with its c1 part removed, c3 = c1 x c2
    double a1[3] = {r.c1[0], r.c1[1], r.c1[2]}, a2[3] = {r.c2[0], r.c2[1], r.c2[2]};
    double n1 = std::sqrt(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
    if (n1 == 0) { a1[0] = 1; a1[1] = a1[2] = 0; n1 = 1; }
    for (double& v : a1) v /= n1;
    const double p12 = a2[0] * a1[0] + a2[1] * a1[1] + a2[2] * a1[2];
    for (int k = 0; k < 3; ++k) a2[k] -= p12 * a1[k];
    double n2 = std::sqrt(a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2]);
    if (n2 == 0) {   // any direction normal to c1
        const double t[3] = {std::fabs(a1[0]) < 0.9 ? 1.0 : 0.0, std::fabs(a1[0]) < 0.9 ? 0.0 : 1.0, 0.0};
        const double q = t[0] * a1[0] + t[1] * a1[1];
        for (int k = 0; k < 3; ++k) a2[k] = t[k] - q * a1[k];
        n2 = std::sqrt(a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2]);
    }
    for (double& v : a2) v /= n2;
    const double a3[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
    o.c1x = (T)a1[0]; o.c1y = (T)a1[1]; o.c1z = (T)a1[2];
    o.c2x = (T)a2[0]; o.c2y = (T)a2[1]; o.c2z = (T)a2[2];
    o.c3x = (T)a3[0]; o.c3y = (T)a3[1]; o.c3z = (T)a3[2];
    o.ks = (T)(2.0 * r.Ks * imu);
    o.b1 = (T)(2.0 * r.B1 * imu);
    o.b2 = (T)(2.0 * r.B2 * imu);
    return o;
}

template <typename T>
static mm_status upload_regions_t(mm_ctx* c) {
    const int nr = c->nreg;
    std::vector<Region<T>> lut(nr);
    const double V = c->grid.dx * c->grid.dy * c->grid.dz;
    for (int q = 0; q < nr; ++q) lut[q] = region_coeffs<T>(c->regions[q], V);
    std::vector<T> cp((size_t)nr * nr);
    for (int a = 0; a < nr; ++a)
        for (int b = 0; b < nr; ++b) {
            const double Aa = c->regions[a].A, Ab = c->regions[b].A;
            const double Aij = (Aa + Ab > 0) ? 2.0 * Aa * Ab / (Aa + Ab) : 0.0;
            const double imu = c->regions[a].Ms > 0 ? 1.0 / (kMu0 * c->regions[a].Ms) : 0.0;
            cp[(size_t)a * nr + b] = (T)(2.0 * Aij * imu);
        }
    cudaError_t e = cudaMalloc(&c->d_lut, sizeof(Region<T>) * nr);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cpair, sizeof(T) * nr * nr);
    if (e != cudaSuccess) return cuda_check(c, e, "material tables");
    cudaMemcpy(c->d_lut, lut.data(), sizeof(Region<T>) * nr, cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_cpair, cp.data(), sizeof(T) * nr * nr, cudaMemcpyHostToDevice);
    if constexpr (sizeof(T) == 4) { c->r0f = lut[0]; c->c00f = cp[0]; }
    else { c->r0d = lut[0]; c->c00d = cp[0]; }
    if (!c->uniform) {
        e = cudaMalloc(&c->d_region, c->N);
        if (e != cudaSuccess) return cuda_check(c, e, "region map");
        cudaMemcpy(c->d_region, c->region_of_cell.data(), c->N, cudaMemcpyHostToDevice);
    }
    return MM_OK;
}

static mm_status build_regions(mm_ctx* c, const mm_material* mat) {
    const long long N = c->N;
    const bool percell = mat->Ms_cell || mat->A_cell || mat->alpha_cell || mat->Ku1_cell || mat->u_cell ||
                         mat->D_cell || mat->D_bulk_cell;
    RegionHost base{mat->Ms, mat->A, mat->alpha, mat->Ku1, {mat->u[0], mat->u[1], mat->u[2]}, mat->D, mat->D_bulk,
                    mat->Kc1, mat->Kc2, {mat->c1[0], mat->c1[1], mat->c1[2]}, {mat->c2[0], mat->c2[1], mat->c2[2]},
                    mat->Ks, mat->B1, mat->B2};
    c->regions.clear();
    if (!percell) {
        c->regions.push_back(base);
        c->nreg = 1;
        c->uniform = base.Ms > 0 ? 1 : 0;
        if (!c->uniform) c->region_of_cell.assign(N, 0);
        return MM_OK;
    }
    c->region_of_cell.resize(N);
    for (long long i = 0; i < N; ++i) {
        RegionHost r = base;
        if (mat->Ms_cell) r.Ms = mat->Ms_cell[i];
        if (mat->A_cell) r.A = mat->A_cell[i];
        if (mat->alpha_cell) r.alpha = mat->alpha_cell[i];
        if (mat->Ku1_cell) r.Ku1 = mat->Ku1_cell[i];
        if (mat->D_cell) r.D = mat->D_cell[i];
        if (mat->D_bulk_cell) r.Db = mat->D_bulk_cell[i];
        if (mat->u_cell) { r.u[0] = mat->u_cell[i]; r.u[1] = mat->u_cell[N + i]; r.u[2] = mat->u_cell[2 * N + i]; }
        if (!(r.Ms >= 0) || !(r.A >= 0) || !(r.alpha >= 0))
            return set_error(c, MM_ERR_ARG, "per-cell Ms, A and alpha must be non-negative");
        int found = -1;
        for (size_t q = 0; q < c->regions.size(); ++q)
            if (c->regions[q] == r) { found = (int)q; break; }
        if (found < 0) {
            if ((int)c->regions.size() >= kMaxRegions)
                return set_error(c, MM_ERR_ARG, "more than 256 distinct per-cell material tuples");
            c->regions.push_back(r);
            found = (int)c->regions.size() - 1;
        }
        c->region_of_cell[i] = (uint8_t)found;
    }
    c->nreg = (int)c->regions.size();
    c->uniform = (c->nreg == 1 && c->regions[0].Ms > 0) ? 1 : 0;
    return MM_OK;
}

static void invalidate_graph(mm_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph1) cudaGraphExecDestroy(c->graph1);
    c->graph = nullptr;
    c->graph1 = nullptr;
    c->graph_chunk = 0;
    surrogate_invalidate_graph(c);
}

static mm_status sync_state(mm_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(&c->h_state, c->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "state readback");
}

static mm_status push_state(mm_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->d_state, &c->h_state, sizeof(DevState), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "state upload");
}

static mm_status status_from_device(mm_ctx* c) {
    if (c->h_state.status == MM_ERR_DT_UNDERFLOW) return set_error(c, MM_ERR_DT_UNDERFLOW, "RK45 step fell below dt_min");
    if (c->h_state.status == MM_ERR_NONFINITE) return set_error(c, MM_ERR_NONFINITE, "non-finite value in the state");
    return MM_OK;
}

// Effective terms: the requested ones without those whose parameters are
// all zero (cubic, surface, magnetoelastic, RKKY), so they cost nothing
// unless used.
static void update_terms(mm_ctx* c) {
    unsigned t = c->terms_req;
    bool cubic = false, surf = false, mel = false;
    for (const RegionHost& r : c->regions) {
        cubic = cubic || r.Kc1 != 0 || r.Kc2 != 0;
        surf = surf || r.Ks != 0;
        mel = mel || r.B1 != 0 || r.B2 != 0;
    }
    bool strain = c->d_strain != nullptr;
    for (double e : c->strain) strain = strain || e != 0;
    if (!cubic) t &= ~MM_TERM_CUBIC;
    if (!surf) t &= ~MM_TERM_SURFACE;
    if (!mel || !strain) t &= ~MM_TERM_MEL;
    if (c->rkky_J == 0) t &= ~MM_TERM_RKKY;
    c->terms = t;
    bool bulk = false;
    for (const RegionHost& r : c->regions) bulk = bulk || r.Db != 0;
    c->ext_terms = (bulk && (t & MM_TERM_DMI)) ||
                   (t & (MM_TERM_CUBIC | MM_TERM_SURFACE | MM_TERM_RKKY | MM_TERM_MEL)) != 0;
}

static void free_all(mm_ctx* c) {
    invalidate_graph(c);
    demag_free(c);
    batch_free(c->batch);
    c->batch = nullptr;
    surrogate_free(c);
    void* bufs[] = {c->d_region, c->d_lut, c->d_cpair, c->d_m, c->d_mtmp, c->d_kslot, c->d_hd, c->d_hbuf,
                    c->d_bcell, c->d_state, c->d_replay, c->d_red, c->d_stage, c->d_strain, c->d_flag};
    for (void* b : bufs) cudaFree(b);
    for (auto& k : c->d_k) cudaFree(k);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
}

static mm_status alloc(mm_ctx* c, void** p, size_t bytes, const char* what) {
    if (c->inject == 1) {
        c->inject = 0;
        return set_error(c, MM_ERR_OOM, std::string("injected allocation failure: ") + what);
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_check(c, e, what);
    return MM_OK;
}

static mm_status check_device(mm_ctx* c) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(c, MM_ERR_DEVICE, std::string("no CUDA device: ") + cudaGetErrorString(e));
    cudaDeviceProp p;
    e = cudaGetDeviceProperties(&p, dev);
    if (e != cudaSuccess) return set_error(c, MM_ERR_DEVICE, cudaGetErrorString(e));
    if (!(p.major == 10 && p.minor == 3))
        return set_error(c, MM_ERR_DEVICE, "libmm is built for sm_103a (GB300); found compute capability " +
                                               std::to_string(p.major) + "." + std::to_string(p.minor));
    return MM_OK;
}

static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename T>
static void host_to_state(const double* m, long long N, const std::vector<uint8_t>& reg,
                          const std::vector<RegionHost>& regions, int uniform, std::vector<T>& out) {
    out.resize(3 * N);
    for (long long i = 0; i < N; ++i) {
        const bool present = uniform ? true : regions[reg[i]].Ms > 0;
        double x = m[i], y = m[N + i], z = m[2 * N + i];
        const double n = std::sqrt(x * x + y * y + z * z);
        if (!present || n == 0) x = y = z = 0;
        else { x /= n; y /= n; z /= n; }
        out[i] = (T)x; out[N + i] = (T)y; out[2 * N + i] = (T)z;
    }
}

// Host doubles (already copied to the device) -> normalised state in the
// working precision; absent cells (Ms = 0) and zero vectors become 0.
template <typename T>
__global__ void state_in_kernel(const double* __restrict__ src, long long N, const uint8_t* __restrict__ region,
                                const Region<T>* __restrict__ lut, T* __restrict__ dst, int* __restrict__ changed) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const bool present = region ? lut[region[i]].present != (T)0 : true;
    double x = src[i], y = src[N + i], z = src[2 * N + i];
    const double n2 = x * x + y * y + z * z;
    // unit to within a few units in the last place of T: taken as it is
    // (a state read back and written again stays bit for bit the same)
    const double tol = sizeof(T) == 4 ? 4.8e-7 : 8.9e-16;
    if (!present || n2 == 0.0) {
        x = y = z = 0.0;
    } else if (fabs(n2 - 1.0) > tol) {
        const double n = sqrt(n2);
        x /= n; y /= n; z /= n;
    }
    const T v[3] = {(T)x, (T)y, (T)z};
    bool diff = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T old = dst[c * N + i];
        if (sizeof(T) == 4) diff = diff || __float_as_uint((float)old) != __float_as_uint((float)v[c]);
        else diff = diff || __double_as_longlong((double)old) != __double_as_longlong((double)v[c]);
        dst[c * N + i] = v[c];
    }
    if (diff) *changed = 1;
}

template <typename T>
__global__ void state_out_kernel(const T* __restrict__ src, long long n, double* __restrict__ dst) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

// Device staging buffer for host <-> state transfers (3 N doubles of the
// largest replica), allocated on first use.
static mm_status ensure_stage(mm_ctx* c, long long n3) {
    if (c->d_stage && c->stage_n >= n3) return MM_OK;
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_n = 0;
    mm_status s = alloc(c, &c->d_stage, sizeof(double) * n3, "host transfer staging");
    if (s == MM_OK) c->stage_n = n3;
    return s;
}

}  // namespace mm

using namespace mm;

extern "C" {

const char* mm_status_string(mm_status s) {
    switch (s) {
        case MM_OK: return "ok";
        case MM_ERR_ARG: return "invalid argument";
        case MM_ERR_DEVICE: return "unsupported device";
        case MM_ERR_OOM: return "out of device memory";
        case MM_ERR_CUDA: return "CUDA error";
        case MM_ERR_NONFINITE: return "non-finite state";
        case MM_ERR_DT_UNDERFLOW: return "time step underflow";
        case MM_ERR_TIMEOUT: return "device wait timed out";
        case MM_ERR_STATE: return "invalid state";
    }
    return "unknown";
}

const char* mm_last_error(const mm_ctx* c) { return c ? c->last_error.c_str() : g_create_error.c_str(); }

mm_status mm_create(const mm_grid* grid, const mm_material* mat, const mm_config* cfg, mm_ctx** out) {
    if (!grid || !mat || !cfg || !out) return set_error(nullptr, MM_ERR_ARG, "null argument");
    *out = nullptr;
    if (grid->nx <= 0 || grid->ny <= 0 || grid->nz <= 0 || !(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0))
        return set_error(nullptr, MM_ERR_ARG, "grid sizes and cell edges must be positive");
    if (cfg->precision != 32 && cfg->precision != 64) return set_error(nullptr, MM_ERR_ARG, "precision must be 32 or 64");
    if (cfg->integrator != MM_HEUN && cfg->integrator != MM_RK45 && cfg->integrator != MM_RK4 &&
        cfg->integrator != MM_DM && cfg->integrator != MM_DM_ADAPTIVE)
        return set_error(nullptr, MM_ERR_ARG, "bad integrator");
    if (cfg->integrator == MM_DM_ADAPTIVE && cfg->T > 0)
        return set_error(nullptr, MM_ERR_ARG, "adaptive Depondt-Mertens with T > 0: use the fixed-step scheme");
    if (cfg->integrator == MM_RK45 && cfg->T > 0)
        return set_error(nullptr, MM_ERR_ARG, "RK45 with T > 0: adaptive stepping of white noise is not defined; use Heun");
    if (cfg->integrator == MM_RK4 && cfg->T > 0)
        return set_error(nullptr, MM_ERR_ARG, "RK4 with T > 0: the thermal field needs Heun or Depondt-Mertens");
    if (cfg->demag == MM_DEMAG_SURROGATE) return set_error(nullptr, MM_ERR_ARG, "surrogate demag needs mm_surrogate_*");
    if (grid->pbc[0] < 0 || grid->pbc[1] < 0 || grid->pbc[2] < 0 || grid->pbc[0] > 4096 || grid->pbc[1] > 4096 ||
        grid->pbc[2] > 4096)
        return set_error(nullptr, MM_ERR_ARG, "pbc[d] is an image count in [0, 4096]");
    if (!(cfg->dt > 0)) return set_error(nullptr, MM_ERR_ARG, "dt must be positive");
    mm_ctx* c = new mm_ctx();
    mm_status s = check_device(c);
    if (s != MM_OK) {
        g_create_error = c->last_error;
        delete c;
        return s;
    }
    c->prec = cfg->precision;
    c->esz = c->prec == 32 ? 4 : 8;
    c->integrator = cfg->integrator;
    c->terms = cfg->terms ? cfg->terms : MM_TERM_ALL;
    if (cfg->demag != MM_DEMAG_EXACT) c->terms &= ~MM_TERM_DEMAG;
    c->terms_req = c->terms;
    c->grid = *grid;
    c->N = (long long)grid->nx * grid->ny * grid->nz;
    c->cfg = *cfg;
    c->Tr = cfg->T;
    c->seed = splitmix64(cfg->seed);
    const long long N = c->N;
    cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    c->stream = c->own_stream;
#define TRY(x) do { mm_status _s = (x); if (_s != MM_OK) { g_create_error = c->last_error; free_all(c); delete c; return _s; } } while (0)
    TRY(build_regions(c, mat));
    update_terms(c);
    TRY(c->prec == 32 ? upload_regions_t<float>(c) : upload_regions_t<double>(c));
    const size_t vb = 3 * N * c->esz;
    TRY(alloc(c, &c->d_m, vb, "state"));
    TRY(alloc(c, &c->d_mtmp, vb, "stage state"));
    TRY(alloc(c, &c->d_hbuf, vb, "field scratch"));
    const int nk = c->integrator == MM_RK45 ? 7 : c->integrator == MM_RK4 ? 4 : c->integrator == MM_DM_ADAPTIVE ? 2 : 1;
    for (int q = 0; q < nk; ++q) TRY(alloc(c, &c->d_k[q], vb, "slopes"));
    TRY(alloc(c, &c->d_kslot, sizeof(void*) * 7, "slot table"));
    cudaMemcpy(c->d_kslot, c->d_k, sizeof(void*) * 7, cudaMemcpyHostToDevice);
    TRY(alloc(c, (void**)&c->d_state, sizeof(DevState), "device state"));
    c->red_cap = 2 * 304 + 32;
    TRY(alloc(c, (void**)&c->d_red, sizeof(double) * c->red_cap, "reduction partials"));
    TRY(alloc(c, (void**)&c->d_flag, sizeof(int), "state flag"));
    if (c->terms & MM_TERM_DEMAG) {
        TRY(alloc(c, &c->d_hd, vb, "demag field"));
        TRY(demag_setup(c));
    }
    // state: m along +z
    {
        std::vector<double> m0(3 * N, 0.0);
        for (long long i = 0; i < N; ++i) m0[2 * N + i] = 1.0;
        if (c->prec == 32) {
            std::vector<float> h;
            host_to_state<float>(m0.data(), N, c->region_of_cell, c->regions, c->uniform, h);
            cudaMemcpy(c->d_m, h.data(), vb, cudaMemcpyHostToDevice);
        } else {
            std::vector<double> h;
            host_to_state<double>(m0.data(), N, c->region_of_cell, c->regions, c->uniform, h);
            cudaMemcpy(c->d_m, h.data(), vb, cudaMemcpyHostToDevice);
        }
    }
    DevState& st = c->h_state;
    st = DevState{};
    st.dt = cfg->dt;
    st.rtol = cfg->rtol > 0 ? cfg->rtol : 1e-6;
    st.dt_min = cfg->dt_min > 0 ? cfg->dt_min : 1e-20;
    st.dt_max = cfg->dt_max > 0 ? cfg->dt_max : 1e-11;
    st.t_end = std::numeric_limits<double>::infinity();
    st.k_first = 0;
    st.fsal = c->integrator == MM_RK45 ? 1 : 0;
    st.ctrl_exp = c->integrator == MM_DM_ADAPTIVE ? 0.5 : 0.2;
    TRY(push_state(c));
    TRY(cuda_check(c, cudaDeviceSynchronize(), "create"));
#undef TRY
    *out = c;
    return MM_OK;
}

mm_status mm_create_batch(int R, const mm_grid* grids, const mm_material* mat, const mm_config* cfg,
                          const uint64_t* seeds, mm_ctx** out) {
    if (!grids || !mat || !cfg || !out || R <= 0) return set_error(nullptr, MM_ERR_ARG, "null argument or R <= 0");
    *out = nullptr;
    if (R == 1) {
        mm_status s = mm_create(grids, mat, cfg, out);
        if (s == MM_OK && seeds) (*out)->seed = seeds[0];
        return s;
    }
    // replica-batched thin films (Methods, "Replica batching")
    if (cfg->precision != 32) return set_error(nullptr, MM_ERR_ARG, "replica batching runs in FP32");
    if (cfg->integrator != MM_HEUN && cfg->integrator != MM_DM)
        return set_error(nullptr, MM_ERR_ARG, "replica batching integrates with Heun or Depondt-Mertens");
    if (cfg->demag == MM_DEMAG_SURROGATE) return set_error(nullptr, MM_ERR_ARG, "surrogate demag is single-instance");
    if (!(cfg->dt > 0)) return set_error(nullptr, MM_ERR_ARG, "dt must be positive");
    if (mat->Ms_cell || mat->A_cell || mat->alpha_cell || mat->Ku1_cell || mat->u_cell || mat->D_cell ||
        mat->D_bulk_cell || !(mat->Ms > 0))
        return set_error(nullptr, MM_ERR_ARG, "replica batching takes one uniform material with Ms > 0");
    for (int r = 0; r < R; ++r) {
        const mm_grid& g = grids[r];
        if (g.nx <= 0 || g.ny <= 0 || g.nz != 1) return set_error(nullptr, MM_ERR_ARG, "batched replicas are nz = 1 films");
        if (g.dx != grids[0].dx || g.dy != grids[0].dy || g.dz != grids[0].dz || !(g.dx > 0) || !(g.dy > 0) || !(g.dz > 0))
            return set_error(nullptr, MM_ERR_ARG, "batched replicas share one cell size");
        if (g.pbc[0] || g.pbc[1] || g.pbc[2]) return set_error(nullptr, MM_ERR_ARG, "batched replicas are open films");
        if (g.nx > 1024 || g.ny > 1024) return set_error(nullptr, MM_ERR_ARG, "batched replicas are at most 1024 x 1024");
        if (cfg->demag == MM_DEMAG_EXACT && (g.nx < 2 || g.ny < 2))
            return set_error(nullptr, MM_ERR_ARG, "batched demag needs replicas of at least 2 x 2 cells; turn demag off");
    }
    mm_ctx* c = new mm_ctx();
    mm_status s = check_device(c);
    if (s != MM_OK) {
        g_create_error = c->last_error;
        delete c;
        return s;
    }
    c->prec = 32;
    c->esz = 4;
    c->integrator = cfg->integrator;
    c->terms = cfg->terms ? cfg->terms : MM_TERM_ALL;
    if (cfg->demag != MM_DEMAG_EXACT) c->terms &= ~MM_TERM_DEMAG;
    c->terms_req = c->terms;
    c->cfg = *cfg;
    c->R = R;
    c->grid = grids[0];
    c->Tr = cfg->T;
    // storage: replicas of one grid size together (sizes in order of first
    // appearance, replicas by index within a size), so that each size class
    // is one contiguous block [replica][component][y][x]
    // each size class starts on a 16-byte boundary (the FFT passes load
    // rows as float2 / float4 vectors); the device-layout calls skip the gaps
    long long off = 0, packed = 0, maxN = 0;
    c->roff.assign(R, 0);
    c->sblocks.clear();
    std::vector<char> placed(R, 0);
    for (int r = 0; r < R; ++r) {
        if (placed[r]) continue;
        off = (off + 3) / 4 * 4;
        const long long start = off;
        for (int q = r; q < R; ++q) {
            if (placed[q] || grids[q].nx != grids[r].nx || grids[q].ny != grids[r].ny) continue;
            placed[q] = 1;
            c->roff[q] = off;
            off += 3LL * grids[q].nx * grids[q].ny;
        }
        c->sblocks.push_back({start, packed, off - start});
        packed += off - start;
    }
    for (int r = 0; r < R; ++r) {
        c->rgrid.push_back(grids[r]);
        maxN = std::max(maxN, (long long)grids[r].nx * grids[r].ny);
        c->rkey.push_back(seeds ? seeds[r] : splitmix64(cfg->seed + (uint64_t)r));
        c->rT.push_back(cfg->T);
        c->rJ.push_back(0.0);
    }
    c->Ntot = (off + 2) / 3;
    c->N = maxN;
    c->seed = c->rkey[0];
    cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    c->stream = c->own_stream;
#define TRY(x) do { mm_status _s = (x); if (_s != MM_OK) { g_create_error = c->last_error; free_all(c); delete c; return _s; } } while (0)
    TRY(build_regions(c, mat));
    update_terms(c);
    TRY(upload_regions_t<float>(c));
    const size_t vb = 3 * c->Ntot * 4;
    TRY(alloc(c, &c->d_m, vb, "state"));
    TRY(alloc(c, &c->d_mtmp, vb, "predictor state"));
    TRY(alloc(c, &c->d_k[0], vb, "predictor slope"));
    TRY(alloc(c, &c->d_hbuf, 3 * maxN * 4, "field scratch"));
    TRY(alloc(c, &c->d_hd, 3 * maxN * 4, "demag field"));
    TRY(alloc(c, &c->d_kslot, sizeof(void*) * 7, "slot table"));
    cudaMemcpy(c->d_kslot, c->d_k, sizeof(void*) * 7, cudaMemcpyHostToDevice);
    TRY(alloc(c, (void**)&c->d_state, sizeof(DevState), "device state"));
    c->red_cap = 2 * 304 + 32;
    TRY(alloc(c, (void**)&c->d_red, sizeof(double) * c->red_cap, "reduction partials"));
    TRY(alloc(c, (void**)&c->d_flag, sizeof(int), "state flag"));
    c->batch = batch_new();
    TRY(batch_setup(c, c->batch, c->rgrid, c->rkey, (c->terms & MM_TERM_DEMAG) != 0));
    TRY(batch_upload(c, c->batch, c->rT, c->rJ));
    {
        std::vector<float> h(3 * c->Ntot, 0.f);
        for (int r = 0; r < R; ++r) {
            const long long n = (long long)grids[r].nx * grids[r].ny;
            for (long long i = 0; i < n; ++i) h[c->roff[r] + 2 * n + i] = 1.f;
        }
        cudaMemcpy(c->d_m, h.data(), vb, cudaMemcpyHostToDevice);
    }
    DevState& st = c->h_state;
    st = DevState{};
    st.dt = cfg->dt;
    st.rtol = 1e-6;
    st.dt_min = 1e-20;
    st.dt_max = 1e-11;
    st.t_end = std::numeric_limits<double>::infinity();
    st.fsal = 0;
    st.ctrl_exp = 0.2;
    TRY(push_state(c));
    TRY(cuda_check(c, cudaDeviceSynchronize(), "create batch"));
#undef TRY
    *out = c;
    return MM_OK;
}

mm_status mm_destroy(mm_ctx* c) {
    if (!c) return MM_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return MM_OK;
}

mm_status mm_set_stream(mm_ctx* c, void* stream) {
    if (!c) return MM_ERR_ARG;
    cudaStreamSynchronize(c->stream);
    c->stream = stream ? (cudaStream_t)stream : c->own_stream;
    invalidate_graph(c);
    return MM_OK;
}

}  // extern "C"

namespace mm {
// sums of m_x, m_y, m_z and the present-cell count (reduce.cu)
void mean_launch(mm_ctx* c, const void* m, int layer, double* d_out);
}  // namespace mm

static mm_status check_replica(mm_ctx* c, int r) {
    if (!c) return MM_ERR_ARG;
    if (r < 0 || r >= c->R) return set_error(c, MM_ERR_ARG, "replica index out of range");
    return MM_OK;
}

// Points the single-instance view of the context (grid, N, state pointer,
// seed, temperature, current, demag plan) at replica r of a batch, so the
// per-instance observables run unchanged; restored on scope exit.
struct ReplicaView {
    mm_ctx* c;
    bool on;
    mm_grid g;
    long long N;
    void* m;
    uint64_t seed;
    double T, J;
    DemagPlan dm;
    ReplicaView(mm_ctx* cc, int r) : c(cc), on(cc->batch != nullptr) {
        if (!on) return;
        g = c->grid; N = c->N; m = c->d_m; seed = c->seed; T = c->Tr; J = c->J; dm = c->dm;
        c->grid = c->rgrid[r];
        c->N = (long long)c->grid.nx * c->grid.ny;
        c->d_m = (char*)c->d_m + c->roff[r] * 4;
        c->seed = c->rkey[r];
        c->Tr = c->rT[r];
        c->J = c->rJ[r];
        if (c->terms & MM_TERM_DEMAG) c->dm = batch_plan(c->batch, batch_class_of(c->batch, r));
    }
    ~ReplicaView() {
        if (!on) return;
        c->grid = g; c->N = N; c->d_m = m; c->seed = seed; c->Tr = T; c->J = J; c->dm = dm;
    }
};

extern "C" {

// Device address of page-locked host memory (null for pageable memory):
// the transfer kernels then read or write the host buffer directly, one
// pass over the interconnect instead of a copy plus a device pass.
static const void* mapped_host(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

mm_status mm_set_m(mm_ctx* c, int r, const double* m) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    if (!m) return set_error(c, MM_ERR_ARG, "null m");
    ReplicaView view(c, r);
    const long long n3 = 3 * c->N;
    const double* src = (const double*)mapped_host(m);
    cudaError_t e = cudaSuccess;
    if (!src) {
        s = ensure_stage(c, n3);
        if (s != MM_OK) return s;
        e = cudaMemcpyAsync(c->d_stage, m, sizeof(double) * n3, cudaMemcpyHostToDevice, c->stream);
        src = (const double*)c->d_stage;
    }
    const unsigned nb = (unsigned)((c->N + 255) / 256);
    const uint8_t* reg = c->uniform ? nullptr : (const uint8_t*)c->d_region;
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
        if (c->prec == 32)
            state_in_kernel<float><<<nb, 256, 0, c->stream>>>(src, c->N, reg, (const Region<float>*)c->d_lut,
                                                             (float*)c->d_m, c->d_flag);
        else
            state_in_kernel<double><<<nb, 256, 0, c->stream>>>(src, c->N, reg, (const Region<double>*)c->d_lut,
                                                              (double*)c->d_m, c->d_flag);
        e = cudaGetLastError();
    }
    int changed = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&changed, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    // the first-same-as-last slope stays valid only for the very same state
    if (e != cudaSuccess || changed) c->k1_valid = false;
    return cuda_check(c, e, "mm_set_m");
}

mm_status mm_get_m(mm_ctx* c, int r, double* m) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    if (!m) return set_error(c, MM_ERR_ARG, "null m");
    ReplicaView view(c, r);
    const long long n3 = 3 * c->N;
    cudaError_t e;
    double* dst = (double*)mapped_host(m);
    if (c->prec == 32 && dst) {
        state_out_kernel<float><<<(unsigned)((n3 + 255) / 256), 256, 0, c->stream>>>((const float*)c->d_m, n3, dst);
        e = cudaGetLastError();
    } else if (c->prec == 32) {
        s = ensure_stage(c, n3);
        if (s != MM_OK) return s;
        state_out_kernel<float><<<(unsigned)((n3 + 255) / 256), 256, 0, c->stream>>>((const float*)c->d_m, n3,
                                                                                    (double*)c->d_stage);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(m, c->d_stage, sizeof(double) * n3, cudaMemcpyDeviceToHost, c->stream);
    } else {
        e = cudaMemcpyAsync(m, c->d_m, sizeof(double) * n3, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "mm_get_m");
}

mm_status mm_set_m_device(mm_ctx* c, const void* m) {
    if (!c || !m) return MM_ERR_ARG;
    cudaError_t e = cudaSuccess;
    if (c->batch) {
        for (const auto& b : c->sblocks)
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((char*)c->d_m + b[0] * c->esz, (const char*)m + b[1] * c->esz, b[2] * c->esz,
                                    cudaMemcpyDeviceToDevice, c->stream);
    } else {
        e = cudaMemcpyAsync(c->d_m, m, 3 * c->N * c->esz, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (c->batch) {
        for (int r = 0; r < c->R; ++r) {
            ReplicaView view(c, r);
            normalize_launch(c, c->d_m);
        }
    } else {
        normalize_launch(c, c->d_m);
    }
    c->k1_valid = false;
    return cuda_check(c, e, "mm_set_m_device");
}

mm_status mm_get_m_device(mm_ctx* c, void* m) {
    if (!c || !m) return MM_ERR_ARG;
    cudaError_t e = cudaSuccess;
    if (c->batch) {
        for (const auto& b : c->sblocks)
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((char*)m + b[1] * c->esz, (const char*)c->d_m + b[0] * c->esz, b[2] * c->esz,
                                    cudaMemcpyDeviceToDevice, c->stream);
    } else {
        e = cudaMemcpyAsync(m, c->d_m, 3 * c->N * c->esz, cudaMemcpyDeviceToDevice, c->stream);
    }
    return cuda_check(c, e, "mm_get_m_device");
}

mm_status mm_set_field(mm_ctx* c, int r, const double B[3], const double* B_cell) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    if (c->batch && B_cell) return set_error(c, MM_ERR_ARG, "batched replicas take one uniform applied field");
    if (B) for (int d = 0; d < 3; ++d) c->Hext[d] = B[d] / kMu0;
    else for (int d = 0; d < 3; ++d) c->Hext[d] = 0.0;
    if (B_cell) {
        const long long n3 = 3 * c->N;
        if (!c->d_bcell) {
            mm_status a = alloc(c, &c->d_bcell, n3 * c->esz, "per-cell field");
            if (a != MM_OK) return a;
        }
        cudaError_t e;
        if (c->prec == 32) {
            std::vector<float> h(n3);
            for (long long i = 0; i < n3; ++i) h[i] = (float)(B_cell[i] / kMu0);
            e = cudaMemcpy(c->d_bcell, h.data(), n3 * 4, cudaMemcpyHostToDevice);
        } else {
            std::vector<double> h(n3);
            for (long long i = 0; i < n3; ++i) h[i] = B_cell[i] / kMu0;
            e = cudaMemcpy(c->d_bcell, h.data(), n3 * 8, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return cuda_check(c, e, "mm_set_field");
    } else if (c->d_bcell) {
        cudaFree(c->d_bcell);
        c->d_bcell = nullptr;
    }
    c->k1_valid = false;
    invalidate_graph(c);
    return MM_OK;
}

mm_status mm_set_strain(mm_ctx* c, const double eps[6], const double* eps_cell) {
    if (!c || (!eps && !eps_cell)) return set_error(c, MM_ERR_ARG, "strain: eps or eps_cell is required");
    if (eps_cell && c->batch) return set_error(c, MM_ERR_ARG, "replica-batched contexts take a uniform strain");
    cudaStreamSynchronize(c->stream);
    if (eps_cell) {
        const long long n6 = 6 * c->N;
        if (!c->d_strain) {
            mm_status a = alloc(c, &c->d_strain, n6 * c->esz, "per-cell strain");
            if (a != MM_OK) return a;
        }
        cudaError_t e;
        if (c->prec == 32) {
            std::vector<float> h(eps_cell, eps_cell + n6);
            e = cudaMemcpy(c->d_strain, h.data(), n6 * 4, cudaMemcpyHostToDevice);
        } else {
            e = cudaMemcpy(c->d_strain, eps_cell, n6 * 8, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return cuda_check(c, e, "strain upload");
        for (double& v : c->strain) v = 0.0;
    } else {
        cudaFree(c->d_strain);
        c->d_strain = nullptr;
        for (int k = 0; k < 6; ++k) c->strain[k] = eps[k];
    }
    update_terms(c);
    c->k1_valid = false;
    invalidate_graph(c);
    return MM_OK;
}

mm_status mm_set_rkky(mm_ctx* c, int k1, int k2, double J) {
    if (!c) return MM_ERR_ARG;
    if (c->batch) return set_error(c, MM_ERR_STATE, "RKKY couples layers of a single-instance context");
    if (k1 < 0 || k2 < 0 || k1 >= c->grid.nz || k2 >= c->grid.nz || k1 == k2 || !std::isfinite(J))
        return set_error(c, MM_ERR_ARG, "RKKY layers must be two different z indices of the grid");
    cudaStreamSynchronize(c->stream);
    c->rkky_k1 = k1;
    c->rkky_k2 = k2;
    c->rkky_J = J;
    update_terms(c);
    c->k1_valid = false;
    invalidate_graph(c);
    return MM_OK;
}

mm_status mm_set_temperature(mm_ctx* c, const double* T) {
    if (!c || !T) return MM_ERR_ARG;
    if (c->batch && batch_trials_on(c->batch))
        return set_error(c, MM_ERR_STATE, "retire/refill sets each trial's temperature");
    for (int r = 0; r < c->R; ++r)
        if (!(T[r] >= 0)) return set_error(c, MM_ERR_ARG, "negative temperature");
    bool hot = false;
    for (int r = 0; r < c->R; ++r) hot = hot || T[r] > 0;
    if (hot && c->integrator != MM_HEUN && c->integrator != MM_DM)
        return set_error(c, MM_ERR_ARG, "T > 0 needs the Heun or Depondt-Mertens integrator");
    c->Tr = T[0];
    if (c->batch) {
        for (int r = 0; r < c->R; ++r) c->rT[r] = T[r];
        mm_status s = batch_upload(c, c->batch, c->rT, c->rJ);
        if (s != MM_OK) return s;
    }
    invalidate_graph(c);
    return MM_OK;
}

mm_status mm_set_torque(mm_ctx* c, const mm_torque* tq, const double* J) {
    if (!c || !tq) return MM_ERR_ARG;
    if (tq->kind < MM_TORQUE_NONE || tq->kind > MM_TORQUE_ZL) return set_error(c, MM_ERR_ARG, "bad torque kind");
    if (c->batch && tq->kind == MM_TORQUE_ZL) return set_error(c, MM_ERR_ARG, "batched replicas take SOT or STT");
    if (c->batch && batch_trials_on(c->batch))
        return set_error(c, MM_ERR_STATE, "retire/refill sets each trial's current; set the torque before");
    c->tq = *tq;
    c->J = J ? J[0] : 0.0;
    if (c->batch) {
        for (int r = 0; r < c->R; ++r) c->rJ[r] = J ? J[r] : 0.0;
        mm_status s = batch_upload(c, c->batch, c->rT, c->rJ);
        if (s != MM_OK) return s;
    }
    c->k1_valid = false;
    invalidate_graph(c);
    return MM_OK;
}

}  // extern "C"

// one chunk of `n` integrator attempts (or Heun steps) on the stream
static void launch_attempts(mm_ctx* c, int n) {
    for (int q = 0; q < n; ++q) {
        if (c->batch) batch_step(c, c->batch);
        else if (c->integrator == MM_RK45) rk45_attempt(c);
        else if (c->integrator == MM_RK4) rk4_step(c);
        else if (c->integrator == MM_DM) dm_step(c);
        else if (c->integrator == MM_DM_ADAPTIVE) dm_adaptive_attempt(c);
        else heun_step(c);
    }
}

static const int kChunk = 8;
static const int kMacroBlock = 1024;   // steps per launch of the one-cell replica kernel

// Capture `n` attempts on the context stream into an executable graph;
// *launches receives the kernel launches one replay makes.
static mm_status capture_attempts(mm_ctx* c, int n, cudaGraphExec_t* out, long long* launches) {
    cudaGraph_t g;
    const long long before = c->launches;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_check(c, e, "graph capture");
    launch_attempts(c, n);
    e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return cuda_check(c, e, "graph capture end");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_check(c, e, "graph instantiate");
    *launches = c->launches - before;   // counted on replay instead
    c->launches = before;
    return MM_OK;
}

// One attempt from the graph *g (captured on first use with the context's
// current settings); eager launches while profiling.
mm_status mm::attempt_graph_launch(mm_ctx* c, cudaGraphExec_t* g, long long* launches) {
    if (c->profiling) {
        launch_attempts(c, 1);
        return cuda_check(c, cudaGetLastError(), "launch");
    }
    if (!*g) {
        mm_status s = capture_attempts(c, 1, g, launches);
        if (s != MM_OK) return s;
    }
    cudaError_t e = cudaGraphLaunch(*g, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "graph launch");
    c->launches += *launches;
    return MM_OK;
}

static mm_status run_attempts(mm_ctx* c, long long n_attempts) {
    if (c->profiling) {
        launch_attempts(c, (int)n_attempts);
        return cuda_check(c, cudaGetLastError(), "launch");
    }
    long long left = n_attempts;
    if (left >= kChunk && !c->graph) {
        mm_status s = capture_attempts(c, kChunk, &c->graph, &c->launches_per_chunk);
        if (s != MM_OK) return s;
        c->graph_chunk = kChunk;
    }
    while (left >= kChunk) {
        cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "graph launch");
        c->launches += c->launches_per_chunk;
        left -= kChunk;
    }
    if (left > 0 && !c->graph1) {
        mm_status s = capture_attempts(c, 1, &c->graph1, &c->launches_per_attempt);
        if (s != MM_OK) return s;
    }
    for (; left > 0; --left) {
        cudaError_t e = cudaGraphLaunch(c->graph1, c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "graph launch");
        c->launches += c->launches_per_attempt;
    }
    return cuda_check(c, cudaGetLastError(), "launch");
}

static mm_status ensure_k1(mm_ctx* c) {
    if (c->integrator != MM_RK45 || c->k1_valid) return MM_OK;
    rk45_first_slope(c);
    c->k1_valid = true;
    return cuda_check(c, cudaGetLastError(), "first slope");
}

// Advance until `target` accepted steps (or t_end / a device error).
static mm_status advance(mm_ctx* c, long long add_steps, double t_end, int replay) {
    mm_status s = sync_state(c);
    if (s != MM_OK) return s;
    if (c->h_state.status) {
        // a sticky device error from an earlier call: clear it for a fresh attempt
        c->h_state.status = 0;
    }
    if (c->inject == 2) {
        c->inject = 0;
        std::vector<unsigned char> nanbuf(c->esz, 0xFF);
        cudaMemcpyAsync(c->d_m, nanbuf.data(), c->esz, cudaMemcpyHostToDevice, c->stream);
        c->k1_valid = false;
    }
    if (c->inject == 3) {
        c->inject = 0;
        c->h_state.dt_min = 1e300;
        c->h_state.rtol = 0.0;
    }
    const long long start = c->h_state.accepted;
    c->h_state.target = add_steps >= 0 ? start + add_steps : std::numeric_limits<long long>::max();
    c->h_state.t_end = t_end;
    c->h_state.replay = replay;
    if (replay) {
        c->h_state.replay_dts = c->d_replay - start;   // indexed by the accepted-step counter
        c->h_state.replay_n = start + add_steps;
    }
    s = push_state(c);
    if (s != MM_OK) return s;
    s = ensure_k1(c);
    if (s != MM_OK) return s;
    // fixed-step schemes: every attempt is accepted
    const bool heun = c->integrator != MM_RK45 && c->integrator != MM_DM_ADAPTIVE;
    if (c->batch && batch_is_fused(c->batch)) {
        // one-cell replicas: blocks of fused steps, no graph needed
        long long want = add_steps >= 0 ? add_steps
                                        : (long long)std::ceil((t_end - c->h_state.t) / c->h_state.dt);
        while (want > 0) {
            const int k = (int)std::min<long long>(want, kMacroBlock);
            batch_macro_steps(c, c->batch, k);
            want -= k;
        }
        s = cuda_check(c, cudaGetLastError(), "launch");
        if (s != MM_OK) return s;
        s = sync_state(c);
        if (s != MM_OK) return s;
        return status_from_device(c);
    }
    if (surrogate_stepping(c) && !surrogate_fallen_back(c)) {
        // host-driven blocks: exact refresh (with the error monitor) + k-1
        // network attempts; after a fallback the exact loop below takes over
        bool done = false;
        for (int round = 0; round < 100000000; ++round) {
            s = surrogate_block(c);
            if (s != MM_OK) return s;
            s = sync_state(c);
            if (s != MM_OK) return s;
            if (c->h_state.status) { done = true; break; }
            if (add_steps >= 0 && c->h_state.accepted >= c->h_state.target) { done = true; break; }
            if (add_steps < 0 && !(c->h_state.t < t_end)) { done = true; break; }
            if (surrogate_fallen_back(c)) break;
        }
        if (done) {
            if (replay) {
                c->h_state.replay = 0;
                push_state(c);
            }
            return status_from_device(c);
        }
    }
    const long long attempts0 = c->h_state.attempts;
    for (int round = 0; round < 1000000; ++round) {
        long long want;
        if (add_steps >= 0) {
            want = c->h_state.target - c->h_state.accepted;
        } else {
            // attempts still needed at the current step size, at most 64 per
            // round: an adaptive dt grows by up to 5x a step, so estimates
            // from an early small dt overshoot, and every attempt past
            // t_end is a launched no-op
            const double left = t_end - c->h_state.t;
            const double dt = c->h_state.dt > 0 ? c->h_state.dt : 1e-13;
            want = (long long)std::min(64.0, std::ceil(left / dt) + 1.0);
        }
        if (want <= 0) break;
        if (heun) want = std::min<long long>(want, 1 << 20);
        else want = std::min<long long>(std::max<long long>(want, 1), 1 << 16);
        s = run_attempts(c, want);
        if (s != MM_OK) return s;
        s = sync_state(c);
        if (s != MM_OK) return s;
        if (c->h_state.status) break;
        if (add_steps >= 0 && c->h_state.accepted >= c->h_state.target) break;
        if (add_steps < 0 && !(c->h_state.t < t_end)) break;
    }
    if (surrogate_stepping(c)) surrogate_count_exact(c, c->h_state.attempts - attempts0);
    if (replay) {
        c->h_state.replay = 0;
        push_state(c);
    }
    return status_from_device(c);
}

extern "C" {

mm_status mm_step(mm_ctx* c, long n) {
    if (!c || n < 0) return MM_ERR_ARG;
    if (n == 0) return MM_OK;
    return advance(c, n, std::numeric_limits<double>::infinity(), 0);
}

mm_status mm_step_dt(mm_ctx* c, const double* dts, long n) {
    if (!c || (!dts && n > 0) || n < 0) return MM_ERR_ARG;
    if (c->integrator != MM_RK45 && c->integrator != MM_DM_ADAPTIVE)
        return set_error(c, MM_ERR_STATE, "mm_step_dt replays RK45 or adaptive Depondt-Mertens steps");
    if (n == 0) return MM_OK;
    if ((size_t)n > c->replay_cap) {
        cudaFree(c->d_replay);
        c->d_replay = nullptr;
        mm_status a = alloc(c, (void**)&c->d_replay, sizeof(double) * n, "replay steps");
        if (a != MM_OK) return a;
        c->replay_cap = n;
        invalidate_graph(c);
    }
    cudaError_t e = cudaMemcpy(c->d_replay, dts, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_check(c, e, "replay upload");
    return advance(c, n, std::numeric_limits<double>::infinity(), 1);
}

mm_status mm_trials_start(mm_ctx* c, const mm_trials* sp) {
    if (!c || !sp) return MM_ERR_ARG;
    if (!c->batch) return set_error(c, MM_ERR_STATE, "retire/refill needs a replica-batched context (R >= 2)");
    if (sp->n_trials < 1 || sp->max_steps < 1 || !sp->J || !sp->T || !sp->m_init)
        return set_error(c, MM_ERR_ARG, "n_trials, max_steps >= 1 and the J, T, m_init tables are required");
    for (int r = 1; r < c->R; ++r)
        if (c->rgrid[r].nx != c->rgrid[0].nx || c->rgrid[r].ny != c->rgrid[0].ny)
            return set_error(c, MM_ERR_ARG, "retire/refill needs replicas of one grid");
    if (!(sp->axis[0] * sp->axis[0] + sp->axis[1] * sp->axis[1] + sp->axis[2] * sp->axis[2] > 0))
        return set_error(c, MM_ERR_ARG, "zero stop axis");
    for (long long q = 0; q < sp->n_trials; ++q)
        if (!(sp->T[q] >= 0) || !std::isfinite(sp->J[q])) return set_error(c, MM_ERR_ARG, "bad trial T or J");
    mm_status s = sync_state(c);
    if (s != MM_OK) return s;
    s = batch_trials_start(c, c->batch, sp, c->h_state.step);
    if (s != MM_OK) return s;
    invalidate_graph(c);
    return MM_OK;
}

mm_status mm_trials_result(mm_ctx* c, long long* steps, int* stopped, long long* done) {
    if (!c) return MM_ERR_ARG;
    if (!c->batch) return set_error(c, MM_ERR_STATE, "no trials on a single-instance context");
    return batch_trials_result(c, c->batch, steps, stopped, done);
}

mm_status mm_run(mm_ctx* c, double t_end) {
    if (!c) return MM_ERR_ARG;
    mm_status s = sync_state(c);
    if (s != MM_OK) return s;
    if (!(t_end > c->h_state.t)) return MM_OK;
    return advance(c, -1, t_end, 0);
}

mm_status mm_get_heff(mm_ctx* c, int r, double* H, unsigned mask) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    ReplicaView view(c, r);
    if (!H) return set_error(c, MM_ERR_ARG, "null output");
    const unsigned terms = mask & (c->terms | MM_TERM_THERMAL);
    const bool demag = (terms & MM_TERM_DEMAG) && c->dm.on;
    if (demag) demag_apply(c, c->d_m, c->d_hd);
    field_launch(c, MODE_H, terms, c->d_m, demag ? c->d_hd : nullptr, c->d_hbuf, nullptr, nullptr, nullptr, -1, 0, 0);
    const long long n3 = 3 * c->N;
    cudaError_t e;
    if (c->prec == 32) {
        std::vector<float> h(n3);
        e = cudaMemcpyAsync(h.data(), c->d_hbuf, n3 * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        for (long long i = 0; i < n3; ++i) H[i] = h[i];
    } else {
        e = cudaMemcpyAsync(H, c->d_hbuf, n3 * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    return cuda_check(c, e, "mm_get_heff");
}

mm_status mm_energy(mm_ctx* c, int r, double* E) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    ReplicaView view(c, r);
    if (!E) return set_error(c, MM_ERR_ARG, "null output");
    // e = -1/2 mu0 Ms m.H_term for the terms quadratic in m (-mu0 Ms m.H for
    // Zeeman); the cubic term is quartic (Kc1) and sextic (Kc2) in m, so its
    // two parts enter with weights 1/2 and 1/3 (Euler: m.dE/dm = 4E, 6E)
    static const unsigned term_of[9] = {MM_TERM_EXCHANGE, MM_TERM_DMI, MM_TERM_ANISOTROPY, MM_TERM_ZEEMAN,
                                        MM_TERM_DEMAG, MM_TERM_CUBIC, MM_TERM_SURFACE, MM_TERM_RKKY, MM_TERM_MEL};
    static const int slot_of[9] = {MM_E_EXCHANGE, MM_E_DMI, MM_E_ANISOTROPY, MM_E_ZEEMAN, MM_E_DEMAG,
                                   MM_E_CUBIC, MM_E_SURFACE, MM_E_RKKY, MM_E_MEL};
    double* d_out = c->d_red + 2 * 304;
    double h[MM_NENERGY] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    cudaMemsetAsync(d_out, 0, sizeof(double) * MM_NENERGY, c->stream);
    for (int q = 0; q < 9; ++q) {
        if (!(c->terms & term_of[q]) || (q == 4 && !c->dm.on)) continue;
        if (q == 4) demag_apply(c, c->d_m, c->d_hd);
        c->cubic_energy = q == 5;
        field_launch(c, MODE_H, term_of[q], c->d_m, q == 4 ? c->d_hd : nullptr, c->d_hbuf, nullptr, nullptr, nullptr,
                     -1, 0, 0);
        c->cubic_energy = false;
        energy_term_launch(c, c->d_m, c->d_hbuf, slot_of[q], d_out + slot_of[q]);
    }
    cudaError_t e = cudaMemcpyAsync(h, d_out, sizeof(double) * MM_NENERGY, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "mm_energy");
    double tot = 0.0, comp = 0.0;
    for (int q = 0; q < MM_NENERGY; ++q) {
        if (q == MM_E_TOTAL) continue;
        E[q] = h[q];
        const double t = tot + h[q];
        comp += std::fabs(tot) >= std::fabs(h[q]) ? (tot - t) + h[q] : (h[q] - t) + tot;
        tot = t;
    }
    E[MM_E_TOTAL] = tot + comp;
    return MM_OK;
}

mm_status mm_topo_charge(mm_ctx* c, int r, int layer, double* Q) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    ReplicaView view(c, r);
    if (!Q || layer >= c->grid.nz || layer < -1)
        return set_error(c, MM_ERR_ARG, "bad layer (-1 for the mean over layers) or null output");
    double* d_out = c->d_red + 2 * 304 + 16;
    topo_launch(c, c->d_m, layer, d_out);
    double h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, d_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "mm_topo_charge");
    *Q = layer >= 0 ? h : h / c->grid.nz;
    return MM_OK;
}

mm_status mm_mean_m(mm_ctx* c, int r, int layer, double* m_mean) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    ReplicaView view(c, r);
    if (!m_mean || layer >= c->grid.nz) return set_error(c, MM_ERR_ARG, "bad layer or null output");
    double* d_out = c->d_red + 2 * 304 + 20;
    mean_launch(c, c->d_m, layer, d_out);
    double h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, d_out, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "mm_mean_m");
    for (int q = 0; q < 3; ++q) m_mean[q] = h[3] > 0 ? h[q] / h[3] : 0.0;
    return MM_OK;
}

mm_status mm_get_time(mm_ctx* c, int r, double* t, double* dt, long long* steps) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    s = sync_state(c);
    if (s != MM_OK) return s;
    if (t) *t = c->h_state.t;
    if (dt) *dt = c->h_state.dt;
    if (steps) *steps = c->h_state.accepted;
    return MM_OK;
}

mm_status mm_get_stats(mm_ctx* c, mm_stats* st) {
    if (!c || !st) return MM_ERR_ARG;
    mm_status s = sync_state(c);
    if (s != MM_OK) return s;
    st->accepted = c->h_state.accepted;
    st->rejected = c->h_state.rejected;
    st->attempts = c->h_state.attempts;
    st->kernel_launches = c->launches;
    st->t = c->h_state.t;
    st->dt = c->h_state.dt;
    return MM_OK;
}

// checkpoint layout: header | DevState | m | k1 (RK45)
struct CkptHeader {
    char magic[8];
    int prec, integrator;
    long long N;
    uint64_t seed;
    int k1_valid, pad;
};

mm_status mm_get_state(mm_ctx* c, void* buf, size_t* nbytes) {
    if (!c || !nbytes) return MM_ERR_ARG;
    const size_t vb = 3 * (c->batch ? c->Ntot : c->N) * c->esz;
    const bool k1 = c->integrator == MM_RK45;
    const size_t need = sizeof(CkptHeader) + sizeof(DevState) + vb * (k1 ? 2 : 1);
    if (!buf) { *nbytes = need; return MM_OK; }
    if (*nbytes < need) return set_error(c, MM_ERR_ARG, "checkpoint buffer too small");
    mm_status s = sync_state(c);
    if (s != MM_OK) return s;
    CkptHeader h{};
    memcpy(h.magic, "MMCKPT1", 8);
    h.prec = c->prec; h.integrator = c->integrator; h.N = c->batch ? c->Ntot : c->N; h.seed = c->seed;
    h.k1_valid = c->k1_valid;
    char* p = (char*)buf;
    memcpy(p, &h, sizeof h);
    memcpy(p + sizeof h, &c->h_state, sizeof(DevState));
    char* mp = p + sizeof h + sizeof(DevState);
    cudaError_t e = cudaMemcpyAsync(mp, c->d_m, vb, cudaMemcpyDeviceToHost, c->stream);
    if (k1 && e == cudaSuccess) {
        void* slots[7];
        memcpy(slots, c->d_k, sizeof slots);
        e = cudaMemcpyAsync(mp + vb, slots[c->h_state.k_first], vb, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    *nbytes = need;
    return cuda_check(c, e, "mm_get_state");
}

mm_status mm_set_state(mm_ctx* c, const void* buf, size_t nbytes) {
    if (!c || !buf) return MM_ERR_ARG;
    const size_t vb = 3 * (c->batch ? c->Ntot : c->N) * c->esz;
    const bool k1 = c->integrator == MM_RK45;
    const size_t need = sizeof(CkptHeader) + sizeof(DevState) + vb * (k1 ? 2 : 1);
    if (nbytes < need) return set_error(c, MM_ERR_ARG, "checkpoint too small");
    CkptHeader h;
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, "MMCKPT1", 8) != 0 || h.prec != c->prec || h.integrator != c->integrator ||
        h.N != (c->batch ? c->Ntot : c->N))
        return set_error(c, MM_ERR_ARG, "checkpoint does not match this context");
    const char* p = (const char*)buf;
    DevState st;
    memcpy(&st, p + sizeof h, sizeof st);
    // the slope-slot index selects device pointers: a damaged blob must not
    // reach the kernels
    if ((st.k_first != 0 && st.k_first != 6) || (st.fsal != 0 && st.fsal != 1) || !std::isfinite(st.t) ||
        !(st.dt >= 0) || !std::isfinite(st.dt))
        return set_error(c, MM_ERR_ARG, "checkpoint integrator state is damaged");
    st.replay = 0;
    st.replay_dts = nullptr;
    c->h_state = st;
    c->seed = h.seed;
    const char* mp = p + sizeof h + sizeof(DevState);
    cudaError_t e = cudaMemcpyAsync(c->d_m, mp, vb, cudaMemcpyHostToDevice, c->stream);
    if (k1 && e == cudaSuccess) {
        e = cudaMemcpyAsync(c->d_k[st.k_first], mp + vb, vb, cudaMemcpyHostToDevice, c->stream);
        c->k1_valid = h.k1_valid != 0;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "mm_set_state");
    invalidate_graph(c);
    return push_state(c);
}

mm_status mm_get_thermal(mm_ctx* c, int r, long long step, uint32_t* raw, double* H_th) {
    mm_status s = check_replica(c, r);
    if (s != MM_OK) return s;
    ReplicaView view(c, r);
    uint32_t* d_raw = nullptr;
    if (raw) {
        s = alloc(c, (void**)&d_raw, sizeof(uint32_t) * 4 * c->N, "thermal words");
        if (s != MM_OK) return s;
    }
    thermal_raw_launch(c, step, d_raw, H_th ? c->d_hbuf : nullptr);
    cudaError_t e = cudaSuccess;
    if (raw) e = cudaMemcpyAsync(raw, d_raw, sizeof(uint32_t) * 4 * c->N, cudaMemcpyDeviceToHost, c->stream);
    const long long n3 = 3 * c->N;
    std::vector<float> hf;
    if (H_th && e == cudaSuccess) {
        if (c->prec == 32) {
            hf.resize(n3);
            e = cudaMemcpyAsync(hf.data(), c->d_hbuf, n3 * 4, cudaMemcpyDeviceToHost, c->stream);
        } else {
            e = cudaMemcpyAsync(H_th, c->d_hbuf, n3 * 8, cudaMemcpyDeviceToHost, c->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (H_th && c->prec == 32 && e == cudaSuccess)
        for (long long i = 0; i < n3; ++i) H_th[i] = hf[i];
    cudaFree(d_raw);
    return cuda_check(c, e, "mm_get_thermal");
}

mm_status mm_get_demag_kernel(mm_ctx* c, double* out, size_t n_out, int* dims) {
    if (!c) return MM_ERR_ARG;
    return demag_kernel_copy(c, out, n_out, dims);
}

mm_status mm_newell(long count, const int* ijk, double dx, double dy, double dz, double* out) {
    if (count < 0 || (count > 0 && (!ijk || !out)) || !(dx > 0) || !(dy > 0) || !(dz > 0))
        return set_error(nullptr, MM_ERR_ARG, "mm_newell: bad arguments");
    mm_ctx tmp;
    mm_status s = check_device(&tmp);
    if (s != MM_OK) { g_create_error = tmp.last_error; return s; }
    return newell_gpu(count, ijk, dx, dy, dz, out);
}

static bool cache_lookup(const char* path, const std::string& key, int* nt, int* blocks) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        const std::string l(line);
        const std::string tag = "\"" + key + "\"";
        const size_t p = l.find(tag);
        if (p == std::string::npos) continue;
        int a = 0, b = 0;
        if (sscanf(l.c_str() + p + tag.size(), ": {\"nt\": %d, \"blocks\": %d", &a, &b) == 2 && a > 0 && b > 0) {
            *nt = a;
            *blocks = b;
            found = true;
        }
    }
    fclose(f);
    return found;
}

mm_status mm_batch_set_shape(mm_ctx* c, int nt, int blocks) {
    if (!c) return MM_ERR_ARG;
    if (!c->batch) return set_error(c, MM_ERR_STATE, "launch shapes apply to replica-batched contexts");
    if (!(nt == 0 || ((nt == 256 || nt == 512) && blocks >= 1)))
        return set_error(c, MM_ERR_ARG, "nt must be 0 (stacked), 256 or 512, with blocks >= 1");
    cudaStreamSynchronize(c->stream);
    batch_set_shape(c->batch, nt, nt == 0 ? 0 : std::min(blocks, batch_max_blocks(c->batch)));
    int got_nt = -1, got_b = -1;
    batch_get_shape(c->batch, &got_nt, &got_b);
    invalidate_graph(c);
    if (nt == 0 && got_nt != 0) return set_error(c, MM_ERR_OOM, "stacked shape buffers");
    return MM_OK;
}

mm_status mm_batch_autotune(mm_ctx* c, const char* cache_path, int* nt_out, int* blocks_out) {
    if (!c) return MM_ERR_ARG;
    if (!c->batch) return set_error(c, MM_ERR_STATE, "autotuning applies to replica-batched contexts");
    const std::string key = batch_signature(c->batch, c->terms);
    int nt = 0, blocks = 0;
    if (cache_lookup(cache_path, key, &nt, &blocks)) {
        batch_set_shape(c->batch, nt, blocks);
        invalidate_graph(c);
    } else {
        mm_status s = sync_state(c);
        if (s != MM_OK) return s;
        const DevState saved = c->h_state;
        const size_t vb = 3 * c->Ntot * 4;
        void* backup = nullptr;
        s = alloc(c, &backup, vb, "autotune backup");
        if (s != MM_OK) return s;
        cudaMemcpyAsync(backup, c->d_m, vb, cudaMemcpyDeviceToDevice, c->stream);
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        float best = 1e30f;
        int bnt = 256, bblocks = std::min(c->R, 2 * sms);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const bool prof = c->profiling;
        c->profiling = false;
        for (int cand_nt : {256, 512}) {
            const int occ = batch_occupancy(c->batch, cand_nt);
            for (int k = 1; k <= std::max(1, occ); ++k) {
                const int nb = std::min(c->R, k * sms);
                batch_set_shape(c->batch, cand_nt, nb);
                c->h_state.target = std::numeric_limits<long long>::max();
                c->h_state.t_end = std::numeric_limits<double>::infinity();
                push_state(c);
                launch_attempts(c, 1);     // warm-up
                cudaEventRecord(e0, c->stream);
                launch_attempts(c, 3);
                cudaEventRecord(e1, c->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; bnt = cand_nt; bblocks = nb; }
                if (nb == c->R) break;
            }
        }
        {
            // the stacked shape: per size class, passes over all of its replicas
            batch_set_shape(c->batch, 0, 0);
            int got_nt = -1, got_b = -1;
            batch_get_shape(c->batch, &got_nt, &got_b);
            if (got_nt == 0) {
                c->h_state.target = std::numeric_limits<long long>::max();
                c->h_state.t_end = std::numeric_limits<double>::infinity();
                push_state(c);
                launch_attempts(c, 1);
                cudaEventRecord(e0, c->stream);
                launch_attempts(c, 3);
                cudaEventRecord(e1, c->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; bnt = 0; bblocks = 0; }
            }
        }
        c->profiling = prof;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaMemcpyAsync(c->d_m, backup, vb, cudaMemcpyDeviceToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        cudaFree(backup);
        c->h_state = saved;
        s = push_state(c);
        if (s != MM_OK) return s;
        batch_set_shape(c->batch, bnt, bblocks);
        invalidate_graph(c);
        if (cache_path) {
            FILE* f = fopen(cache_path, "a");
            if (f) {
                fprintf(f, "{\"%s\": {\"nt\": %d, \"blocks\": %d, \"ms_per_step\": %.6f}}\n", key.c_str(), bnt,
                        bblocks, best / 3.0f);
                fclose(f);
            }
        }
        nt = bnt;
        blocks = bblocks;
    }
    if (nt_out) *nt_out = nt;
    if (blocks_out) *blocks_out = blocks;
    return cuda_check(c, cudaGetLastError(), "autotune");
}

mm_status mm_set_profiling(mm_ctx* c, int on) {
    if (!c) return MM_ERR_ARG;
    c->profiling = on != 0;
    if (on) c->prof.clear();
    return MM_OK;
}

mm_status mm_get_profile(mm_ctx* c, mm_profile_entry* out, int* n) {
    if (!c || !n) return MM_ERR_ARG;
    const int cnt = (int)c->prof.size();
    if (!out) { *n = cnt; return MM_OK; }
    const int w = std::min(*n, cnt);
    for (int q = 0; q < w; ++q) {
        memset(&out[q], 0, sizeof(mm_profile_entry));
        strncpy(out[q].name, c->prof[q].name.c_str(), sizeof(out[q].name) - 1);
        out[q].launches = c->prof[q].launches;
        out[q].total_ms = c->prof[q].total_ms;
        out[q].bytes_per_launch = c->prof[q].bytes;
    }
    *n = w;
    return MM_OK;
}

mm_status mm_debug_inject(mm_ctx* c, int fault) {
    if (!c || fault < 0 || fault > 4) return MM_ERR_ARG;
    c->inject = fault;
    return MM_OK;
}

}  // extern "C"
