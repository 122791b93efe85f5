// Fused effective field + LLG torque + stage update (Methods, "Physics and
// discretization", Eq. 1; the spin torques enter every integrator stage).
//
// One thread per cell.  The six-point exchange Laplacian, interfacial DMI
// (central differences; at an absent neighbour in the plane the ghost value
// m_i - h (D/2A)(z x n) x m_i, the sign that makes the discrete field the
// gradient of the discrete energy), uniaxial anisotropy, Zeeman, the demag
// field read from the FFT path, and the Philox4x32-10 thermal field are
// summed in registers; the torque and the requested stage update follow
// without writing H.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "ctx.h"
#include "field_dev.cuh"
#include "fft_direct.cuh"

namespace mm {

// Output of one present cell for the launch's mode: H, the slope k (to
// `out` or to the FSAL slot of stage kstage), the Heun / Depondt-Mertens
// predictor (m*, with k or Omega to out2) or corrector (renormalised); the
// step is the attempt's dt_eff (the fixed dt for the fixed-step schemes).
template <typename T>
__device__ __forceinline__ void cell_store(const FieldArgs<T>& a, long long i, const v3<T>& m, const v3<T>& H,
                                           const v3<T>& k) {
    const long long N = a.N;
    if (a.mode == MODE_H) {
        st3(a.out, N, i, H);
    } else if (a.mode == MODE_K) {
        T* o = a.out;
        if (!o) {
            const int kf = a.st->k_first;
            o = a.kptr[a.kstage == 0 ? kf : 6 - kf];
        }
        st3(o, N, i, k);
    } else if (a.mode == MODE_HEUN1) {
        const T dt = (T)a.st->dt_eff;
        st3(a.out2, N, i, k);
        st3(a.out, N, i, m + dt * k);
    } else if (a.mode == MODE_HEUN2) {  // m_new = normalise(m0 + dt/2 (k1 + k2))
        const T dt = (T)a.st->dt_eff;
        const v3<T> m0 = ld3(a.m0, N, i);
        const v3<T> k1 = ld3(a.k1, N, i);
        v3<T> mn = m0 + ((T)0.5 * dt) * (k1 + k);
        const T inv = (T)1 / sqrt(dot(mn, mn));
        st3(a.out, N, i, inv * mn);
    } else if (a.mode == MODE_DM1) {   // Omega_1 and m* = R(Omega_1 dt) m
        const T dt = (T)a.st->dt_eff;
        st3(a.out2, N, i, k);
        st3(a.out, N, i, rodrigues<T>(m, k, dt));
    } else {  // MODE_DM2: m_new = R((Omega_1 + Omega_2) dt / 2) m0
        const T dt = (T)a.st->dt_eff;
        const v3<T> m0 = ld3(a.m0, N, i);
        const v3<T> w1 = ld3(a.k1, N, i);
        const v3<T> mn = rodrigues<T>(m0, (T)0.5 * (w1 + k), dt);
        const T inv = (T)1 / sqrt(dot(mn, mn));
        st3(a.out, N, i, inv * mn);
    }
}

// UNIF: one material (coefficients passed by value in the launch
// parameters, no region map or coefficient-table loads).
template <typename T, bool UNIF, bool EXT>
__global__ void __launch_bounds__(256) field_kernel(FieldArgs<T> a) {
    if (a.gate && !a.st->active) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const long long N = a.N;
    const long long i = ((long long)z * a.ny + y) * a.nx + x;
    const int ri = UNIF ? 0 : (a.region ? a.region[i] : 0);
    const Region<T>& R = UNIF ? a.R0 : a.lut[ri];
    const v3<T> m = ld3(a.m, N, i);
    if (R.present == (T)0) {
        const v3<T> zero = mk3<T>(0, 0, 0);
        T* o = a.out;
        if (!o) {
            const int kf = a.st->k_first;
            o = a.kptr[a.kstage == 0 ? kf : 6 - kf];
        }
        if (a.mode == MODE_HEUN1 || a.mode == MODE_DM1) { st3(o, N, i, zero); st3(a.out2, N, i, zero); }
        else st3(o, N, i, zero);
        return;
    }
    const long long step = a.step_override >= 0 ? a.step_override : (a.st ? a.st->step : 0);
    v3<T> H, k;
    cell_field<T, UNIF, EXT>(a, x, y, z, i, ri, R, m, nullptr, step, H, k, a.mode != MODE_H, a.mode >= MODE_DM1);
    cell_store<T>(a, i, m, H, k);
}

// One material, FP32, nx a multiple of V (2 or 4): each thread owns V
// consecutive cells of a row.  The state, its y/z neighbours, the demag
// field and the outputs move as 8- or 16-byte vectors; the x neighbours of
// the inner cells come from the thread's own registers, only the two
// row-end neighbours are scalar loads.
template <int V> struct fvec;
template <> struct fvec<2> { using t = float2; };
template <> struct fvec<4> { using t = float4; };

template <int V>
__device__ __forceinline__ typename fvec<V>::t ldv(const float* p) {
    return __ldg(reinterpret_cast<const typename fvec<V>::t*>(p));
}
template <int V>
__device__ __forceinline__ void stv(float* p, const typename fvec<V>::t& v) {
    *reinterpret_cast<typename fvec<V>::t*>(p) = v;
}
__device__ __forceinline__ float fget(const float2& v, int q) { return q == 0 ? v.x : v.y; }
__device__ __forceinline__ float fget(const float4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }
__device__ __forceinline__ void fset(float2& v, int q, float x) { if (q == 0) v.x = x; else v.y = x; }
__device__ __forceinline__ void fset(float4& v, int q, float x) {
    if (q == 0) v.x = x; else if (q == 1) v.y = x; else if (q == 2) v.z = x; else v.w = x;
}

// The V cells x0 .. x0 + V - 1 of row (z, y).  HD_SMEM: the demag field of
// the cells comes from shared memory (hds[c * hd_stride + q], the fused
// inverse-X-pass kernel below), else from a.Hd in global memory.  QUIET:
// slopes only (MODE_K), no thermal field, no spin torque -- the variant for
// deterministic runs without current, with far fewer registers.
template <int V, bool EXT, bool HD_SMEM, bool QUIET = false>
__device__ __forceinline__ void field_vec_cells(const FieldArgs<float>& a, int x0, int y, int z, const float* hds,
                                                int hd_stride) {
    using VT = typename fvec<V>::t;
    const long long N = a.N;
    const long long i0 = ((long long)z * a.ny + y) * a.nx + x0;
    const Region<float>& R = a.R0;
    const long long step = a.step_override >= 0 ? a.step_override : (a.st ? a.st->step : 0);
    VT mc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) mc[c] = ldv<V>(a.m + c * N + i0);
    const unsigned nbt = MM_TERM_EXCHANGE | MM_TERM_DMI | (EXT ? MM_TERM_SURFACE : 0u);
    const bool need_nb = (a.terms & nbt) || (!QUIET && a.tq == MM_TORQUE_ZL);
    // neighbour rows (y+, y-, z+, z-) as vectors, row-end x neighbours as scalars
    VT nr[4][3];
    bool rin[4] = {false, false, false, false};
    float xl[3] = {0, 0, 0}, xr[3] = {0, 0, 0};
    bool lin = false, rinx = false;
    if (need_nb) {
        const long long sy = a.nx, sz = (long long)a.nx * a.ny;
        const int ny = a.ny, nz = a.nz;
        const int qs[4] = {y + 1, y - 1, z + 1, z - 1};
        const int dm[4] = {ny, ny, nz, nz};
        const int pr[4] = {a.py, a.py, a.pz, a.pz};
        const int ps[4] = {y, y, z, z};
        const long long st[4] = {sy, sy, sz, sz};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int q = qs[s];
            bool inside = q >= 0 && q < dm[s];
            if (!inside && pr[s]) { q = (q + dm[s]) % dm[s]; inside = true; }
            rin[s] = inside;
            if (inside) {
                const long long j = i0 + (long long)(q - ps[s]) * st[s];
#pragma unroll
                for (int c = 0; c < 3; ++c) nr[s][c] = ldv<V>(a.m + c * N + j);
            }
        }
        int ql = x0 - 1, qr = x0 + V;
        lin = ql >= 0;
        rinx = qr < a.nx;
        if (!lin && a.px) { ql += a.nx; lin = true; }
        if (!rinx && a.px) { qr -= a.nx; rinx = true; }
        const long long row = i0 - x0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (lin) xl[c] = __ldg(a.m + c * N + row + ql);
            if (rinx) xr[c] = __ldg(a.m + c * N + row + qr);
        }
    }
    VT hd[3];
    const bool dem = (a.terms & MM_TERM_DEMAG) && (HD_SMEM || a.Hd);
    if (dem) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            hd[c] = HD_SMEM ? *reinterpret_cast<const VT*>(hds + c * hd_stride) : ldv<V>(a.Hd + c * N + i0);
    }
    VT o1[3], o2[3];
#pragma unroll
    for (int q = 0; q < V; ++q) {
        const v3<float> m = mk3<float>(fget(mc[0], q), fget(mc[1], q), fget(mc[2], q));
        v3<float> nbv[6];
        bool nbp[6];
        float cnb[6];
        if (need_nb) {
            // x+ / x-
            const bool pp = q < V - 1 || rinx, pm = q > 0 || lin;
            nbp[0] = pp;
            nbp[1] = pm;
            nbv[0] = q < V - 1 ? mk3<float>(fget(mc[0], q + 1), fget(mc[1], q + 1), fget(mc[2], q + 1))
                               : (rinx ? mk3<float>(xr[0], xr[1], xr[2]) : ghost_value<float, EXT>(m, 0, 1, a.hx, R.ratio, R.ratio_b));
            nbv[1] = q > 0 ? mk3<float>(fget(mc[0], q - 1), fget(mc[1], q - 1), fget(mc[2], q - 1))
                           : (lin ? mk3<float>(xl[0], xl[1], xl[2]) : ghost_value<float, EXT>(m, 0, -1, a.hx, R.ratio, R.ratio_b));
            cnb[0] = pp ? a.c_uniform : R.cg;
            cnb[1] = pm ? a.c_uniform : R.cg;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int slot = 2 + s, d = 1 + s / 2, sg = (s & 1) ? -1 : 1;
                nbp[slot] = rin[s];
                nbv[slot] = rin[s] ? mk3<float>(fget(nr[s][0], q), fget(nr[s][1], q), fget(nr[s][2], q))
                                   : ghost_value<float, EXT>(m, d, sg, d == 1 ? a.hy : a.hz, R.ratio, R.ratio_b);
                cnb[slot] = rin[s] ? a.c_uniform : R.cg;
            }
        }
        const v3<float> hq = dem ? mk3<float>(fget(hd[0], q), fget(hd[1], q), fget(hd[2], q)) : mk3<float>(0, 0, 0);
        v3<float> H, k;
        cell_field_nb<float, EXT, QUIET>(a, i0 + q, R, m, nbv, nbp, cnb, dem, hq, step, H, k,
                                         QUIET || a.mode != MODE_H, !QUIET && a.mode >= MODE_DM1);
        v3<float> r1 = H, r2 = k;
        if (QUIET || a.mode == MODE_K) r1 = k;
        else if (QUIET) {
        } else if (a.mode == MODE_HEUN1) {
            const float dt = (float)a.st->dt_eff;
            r1 = m + dt * k;
            r2 = k;
        } else if (a.mode == MODE_HEUN2) {
            const float dt = (float)a.st->dt_eff;
            const long long i = i0 + q;
            const v3<float> m0 = ld3(a.m0, N, i);
            const v3<float> k1 = ld3(a.k1, N, i);
            v3<float> mn = m0 + (0.5f * dt) * (k1 + k);
            r1 = (1.0f / sqrtf(dot(mn, mn))) * mn;
        } else if (a.mode == MODE_DM1) {
            r1 = rodrigues<float>(m, k, (float)a.st->dt_eff);
            r2 = k;
        } else if (a.mode == MODE_DM2) {
            const long long i = i0 + q;
            const v3<float> m0 = ld3(a.m0, N, i);
            const v3<float> w1 = ld3(a.k1, N, i);
            const v3<float> mn = rodrigues<float>(m0, 0.5f * (w1 + k), (float)a.st->dt_eff);
            r1 = (1.0f / sqrtf(dot(mn, mn))) * mn;
        }
        fset(o1[0], q, r1.x); fset(o1[1], q, r1.y); fset(o1[2], q, r1.z);
        fset(o2[0], q, r2.x); fset(o2[1], q, r2.y); fset(o2[2], q, r2.z);
    }
    float* o = a.out;
    if (!o) {
        const int kf = a.st->k_first;
        o = a.kptr[a.kstage == 0 ? kf : 6 - kf];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) stv<V>(o + c * N + i0, o1[c]);
    if (!QUIET && (a.mode == MODE_HEUN1 || a.mode == MODE_DM1)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) stv<V>(a.out2 + c * N + i0, o2[c]);
    }
}

template <int V, bool EXT, bool QUIET = false>
__global__ void __launch_bounds__(256) field_vec_kernel(FieldArgs<float> a) {
    if (a.gate && !a.st->active) return;
    const int x0 = V * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x0 >= a.nx || y >= a.ny) return;
    field_vec_cells<V, EXT, false, QUIET>(a, x0, y, z, nullptr, 0);
}

// The last demag pass (inverse X, half spectrum -> real rows) fused with
// the field kernel: a CTA of kC2RWarps = 4 warps takes kC2RRows = 4 rows
// (z, y); its warps transform the three components of those rows (one row
// of one component per warp at a time, three each) into shared memory, then
// every thread forms the field, torque and stage output of 4 cells at a time
// with the demag field read from there -- H_demag never goes through global
// memory.
struct C2RSpec {
    const float2* spec;     // [3][nz][PyA][Wk]
    const float2* tw;       // exp(-2 pi i q / Px)
    int PyA, Wk;
};

constexpr int kC2RRows = 4;
constexpr int kC2RWarps = 4;
constexpr int kC2RThreads = 32 * kC2RWarps;
template <int LT>
constexpr size_t c2r_field_smem() {
    return (size_t)kC2RWarps * wline(LT) * sizeof(float2) + (size_t)3 * kC2RRows * LT * sizeof(float);
}

// Four 4-warp CTAs per SM for the QUIET form (128 registers, no spills):
// as many warps as two CTAs of 8, but more CTAs at different phases -- 4 %
// faster on rows of 512.  The full form is left uncapped (156-218
// registers, two or three CTAs per SM) rather than spill.
template <int LT, bool EXT, bool QUIET = false>
__global__ void __launch_bounds__(kC2RThreads, QUIET ? 4 : 1) c2r_field_kernel(FieldArgs<float> a, C2RSpec s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.gate && !a.st->active) return;
    const int warp = threadIdx.x >> 5;
    float2* line = reinterpret_cast<float2*>(smem_raw) + warp * wline(LT);
    float* sH = reinterpret_cast<float*>(smem_raw + (size_t)kC2RWarps * wline(LT) * sizeof(float2));   // [rpc][3][nx]
    const int nx = a.nx, rpc = kC2RRows, nrows = a.ny * a.nz;
    const int row0 = blockIdx.x * rpc;
    for (int task = warp; task < 3 * rpc; task += kC2RWarps) {
        const int rl = task / 3, comp = task - 3 * rl, row = row0 + rl;
        if (row >= nrows) break;                      // warp-uniform; later tasks have larger rows
        const int z = row / a.ny, y = row - z * a.ny;
        const float2* X = s.spec + ((long long)(comp * a.nz + z) * s.PyA + y) * s.Wk;
        float* dst = sH + (rl * 3 + comp) * nx;
        warp_c2r<LT>(X, s.tw, line, [&](int n, float2 v) {
            if (2 * n + 1 < nx) *reinterpret_cast<float2*>(dst + 2 * n) = v;
        });
        __syncwarp();
    }
    __syncthreads();
    const int tpr = nx / 4;
    for (int c = threadIdx.x; c < rpc * tpr; c += kC2RThreads) {
        const int rl = c / tpr, x0 = 4 * (c - rl * tpr);
        const int row = row0 + rl;
        if (row < nrows) {
            const int z = row / a.ny, y = row - z * a.ny;
            field_vec_cells<4, EXT, true, QUIET>(a, x0, y, z, sH + rl * 3 * nx + x0, nx);
        }
    }
}

constexpr int kFieldV = 4;   // cells per thread of the one-material FP32 kernel (4 measured faster than 2)

template <typename T>
static FieldArgs<T> field_args(mm_ctx* c, int mode, unsigned terms, const T* m, const T* Hd, T* out, T* out2,
                               const T* m0, const T* k1, long long step_override, int gate, int kstage) {
    FieldArgs<T> a{};
    a.gate = gate;
    a.kstage = kstage;
    a.kptr = (T* const*)c->d_kslot;
    const mm_grid& g = c->grid;
    a.m = m; a.m0 = m0; a.k1 = k1; a.out = out; a.out2 = out2;
    a.Hd = Hd;
    a.Bc = (const T*)c->d_bcell;
    for (int d = 0; d < 3; ++d) a.hext[d] = (T)c->Hext[d];
    a.region = c->uniform ? nullptr : (const uint8_t*)c->d_region;
    a.lut = (const Region<T>*)c->d_lut;
    a.cpair = (const T*)c->d_cpair;
    a.nreg = c->nreg;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    a.N = c->N;
    a.hx = (T)g.dx; a.hy = (T)g.dy; a.hz = (T)g.dz;
    a.ix2 = (T)(1.0 / (g.dx * g.dx)); a.iy2 = (T)(1.0 / (g.dy * g.dy)); a.iz2 = (T)(1.0 / (g.dz * g.dz));
    a.px = g.pbc[0] != 0; a.py = g.pbc[1] != 0; a.pz = g.pbc[2] != 0;
    a.terms = terms;
    a.mode = mode;
    a.key0 = (uint32_t)(c->seed & 0xFFFFFFFFull);
    a.key1 = (uint32_t)(c->seed >> 32);
    const double V = g.dx * g.dy * g.dz;
    a.th_scale = c->Tr > 0 ? (T)std::sqrt(c->Tr / (V * c->cfg.dt)) : (T)0;
    a.st = c->d_state;
    a.step_override = step_override;
    a.cubic_w1 = c->cubic_energy ? (T)0.5 : (T)1;
    a.cubic_w2 = c->cubic_energy ? (T)(1.0 / 3.0) : (T)1;
    for (int k = 0; k < 6; ++k) a.strain[k] = (T)c->strain[k];
    a.strain_cell = (const T*)c->d_strain;
    a.rk1 = c->rkky_k1;
    a.rk2 = c->rkky_k2;
    a.rkky_c = (T)(c->rkky_J / g.dz);
    const mm_torque& q = c->tq;
    a.tq = q.kind;
    if (q.kind == MM_TORQUE_SOT || q.kind == MM_TORQUE_STT) {
        const double tF = q.t_F > 0 ? q.t_F : g.nz * g.dz;
        a.tq_base = (T)(kHbar * c->J / (kQe * kMu0 * tF));
        double pn = std::sqrt(q.p[0] * q.p[0] + q.p[1] * q.p[1] + q.p[2] * q.p[2]);
        if (pn == 0) pn = 1;
        for (int d = 0; d < 3; ++d) a.p[d] = (T)(q.p[d] / pn);
        a.theta_half = (T)(0.5 * q.theta_SH);
        a.fl_ratio = (T)q.fl_ratio;
        a.P = (T)q.P;
        a.L2 = (T)(q.Lambda * q.Lambda);
        a.eps_p = (T)q.eps_prime;
    } else if (q.kind == MM_TORQUE_ZL) {
        double u = c->J * q.P * kMuB / kQe;
        if (q.match_mumax) u /= (1.0 + q.xi * q.xi);
        a.zl_u = (T)u;
        a.xi = (T)q.xi;
        double dn = std::sqrt(q.dir[0] * q.dir[0] + q.dir[1] * q.dir[1] + q.dir[2] * q.dir[2]);
        if (dn == 0) dn = 1;
        for (int d = 0; d < 3; ++d) a.dir[d] = (T)(q.dir[d] / dn);
    }
    if constexpr (sizeof(T) == 4) { a.R0 = c->r0f; a.c_uniform = c->c00f; }
    else { a.R0 = c->r0d; a.c_uniform = c->c00d; }
    return a;
}

// The QUIET kernels apply: slopes only, no thermal field, no spin torque,
// none of the further local terms.
template <typename T>
static bool field_quiet(const mm_ctx* c, int mode, unsigned terms, const FieldArgs<T>& a) {
    return mode == MODE_K && !c->ext_terms && a.tq == MM_TORQUE_NONE &&
           (!(terms & MM_TERM_THERMAL) || a.th_scale == (T)0);
}

static double field_bytes(const mm_ctx* c, int mode, unsigned terms, bool hd) {
    const double es = (double)c->esz;
    double bytes = 3 * es * 2 * c->N;          // read m, write out
    if (hd && (terms & MM_TERM_DEMAG)) bytes += 3 * es * c->N;
    if (mode == MODE_HEUN1 || mode == MODE_DM1) bytes += 3 * es * c->N;
    if (mode == MODE_HEUN2 || mode == MODE_DM2) bytes += 6 * es * c->N;
    return bytes;
}

static const char* const kFieldNames[6] = {"field_H", "field_k", "field_heun1", "field_heun2", "field_dm1",
                                           "field_dm2"};

template <typename T>
static void field_launch_t(mm_ctx* c, int mode, unsigned terms, const T* m, const T* Hd, T* out, T* out2,
                           const T* m0, const T* k1, long long step_override, int gate, int kstage) {
    FieldArgs<T> a = field_args<T>(c, mode, terms, m, Hd, out, out2, m0, k1, step_override, gate, kstage);
    const mm_grid& g = c->grid;
    dim3 blk(32, 8);
    dim3 grd((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    LaunchScope ls(c, kFieldNames[mode], field_bytes(c, mode, terms, Hd != nullptr));
    if (c->uniform && !a.region) {
        if constexpr (sizeof(T) == 4) {
            if (g.nx % kFieldV == 0 && a.R0.present != 0.f) {
                dim3 grdv((g.nx / kFieldV + 31) / 32, (g.ny + 7) / 8, g.nz);
                if (c->ext_terms) field_vec_kernel<kFieldV, true><<<grdv, blk, 0, c->stream>>>(a);
                else if (field_quiet(c, mode, terms, a))
                    field_vec_kernel<kFieldV, false, true><<<grdv, blk, 0, c->stream>>>(a);
                else field_vec_kernel<kFieldV, false><<<grdv, blk, 0, c->stream>>>(a);
                return;
            }
        }
        if (c->ext_terms) field_kernel<T, true, true><<<grd, blk, 0, c->stream>>>(a);
        else field_kernel<T, true, false><<<grd, blk, 0, c->stream>>>(a);
    } else {
        if (c->ext_terms) field_kernel<T, false, true><<<grd, blk, 0, c->stream>>>(a);
        else field_kernel<T, false, false><<<grd, blk, 0, c->stream>>>(a);
    }
}

void field_launch(mm_ctx* c, int mode, unsigned terms, const void* m, const void* Hd, void* out, void* out2,
                  const void* m0, const void* k1, long long step_override, int gate, int kstage) {
    if (c->prec == 32)
        field_launch_t<float>(c, mode, terms, (const float*)m, (const float*)Hd, (float*)out, (float*)out2,
                              (const float*)m0, (const float*)k1, step_override, gate, kstage);
    else
        field_launch_t<double>(c, mode, terms, (const double*)m, (const double*)Hd, (double*)out, (double*)out2,
                               (const double*)m0, (const double*)k1, step_override, gate, kstage);
}

// Inverse X pass + field kernel in one launch (FP32, one material, nx a
// multiple of 4 dividing 1024, the one-row-per-warp inverse X transform of
// the grid's half length available).  Measured against the two separate
// kernels: 37.6 against 18.2 + 22.4 us per 256x256x16 evaluation; at
// nx = 512 with the QUIET field variant 385 against 198 + 201 us (the
// general field variant had made it slower there: 430 against 204 + 215).
#define MM_C2R_FIELD_LENGTHS(X) X(128) X(256) X(512)

bool field_c2r_fusable(const mm_ctx* c) {
    const mm_grid& g = c->grid;
    if (c->prec != 32 || !c->dm.on || !c->uniform || c->d_region || c->r0f.present == 0.f) return false;
    if (g.nx % 4 != 0 || 1024 % g.nx != 0 || c->dm.Lh != g.nx) return false;
    switch (c->dm.Lh) {
#define MM_CASE(n) case n: return true;
        MM_C2R_FIELD_LENGTHS(MM_CASE)
#undef MM_CASE
        default: return false;
    }
}

cudaError_t field_c2r_setup() {
    cudaError_t e = cudaSuccess;
#define MM_CASE(n)                                                                                            \
    if (e == cudaSuccess)                                                                                     \
        e = cudaFuncSetAttribute(c2r_field_kernel<n, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                 (int)c2r_field_smem<n>());                                                   \
    if (e == cudaSuccess)                                                                                     \
        e = cudaFuncSetAttribute(c2r_field_kernel<n, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                 (int)c2r_field_smem<n>());                                                   \
    if (e == cudaSuccess)                                                                                     \
        e = cudaFuncSetAttribute(c2r_field_kernel<n, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)c2r_field_smem<n>());
    MM_C2R_FIELD_LENGTHS(MM_CASE)
#undef MM_CASE
    return e;
}

void field_c2r_launch(mm_ctx* c, int mode, unsigned terms, const void* m, void* out, void* out2, const void* m0,
                      const void* k1, long long step_override, int gate, int kstage) {
    FieldArgs<float> a = field_args<float>(c, mode, terms, (const float*)m, nullptr, (float*)out, (float*)out2,
                                           (const float*)m0, (const float*)k1, step_override, gate, kstage);
    const DemagPlan& d = c->dm;
    C2RSpec sp{(const float2*)d.spec, (const float2*)d.tw_x, d.PyA, d.Wk};
    const int rpc = kC2RRows;
    const long long rows = (long long)c->grid.ny * c->grid.nz;
    const unsigned grid = (unsigned)((rows + rpc - 1) / rpc);
    const double bytes = field_bytes(c, mode, terms, false) + 3.0 * rows * (d.Kx * sizeof(float2));
    LaunchScope ls(c, "c2r_field", bytes);
    const bool quiet = field_quiet(c, mode, terms, a);
    switch (d.Lh) {
#define MM_CASE(n)                                                                                            \
    case n:                                                                                                   \
        if (c->ext_terms) c2r_field_kernel<n, true><<<grid, kC2RThreads, c2r_field_smem<n>(), c->stream>>>(a, sp);      \
        else if (quiet) c2r_field_kernel<n, false, true><<<grid, kC2RThreads, c2r_field_smem<n>(), c->stream>>>(a, sp); \
        else c2r_field_kernel<n, false><<<grid, kC2RThreads, c2r_field_smem<n>(), c->stream>>>(a, sp);                 \
        break;
        MM_C2R_FIELD_LENGTHS(MM_CASE)
#undef MM_CASE
        default: break;
    }
}

// Raw Philox words and the thermal field of every cell at a given step.
template <typename T>
__global__ void thermal_raw_kernel(long long N, uint32_t k0, uint32_t k1, long long step, const uint8_t* region,
                                   const Region<T>* lut, T th_scale, uint32_t* raw, T* h) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const U4 r = philox(U4{(uint32_t)i, (uint32_t)step, (uint32_t)((unsigned long long)step >> 32), 0u}, k0, k1);
    if (raw) {
        raw[4 * i] = r.x; raw[4 * i + 1] = r.y; raw[4 * i + 2] = r.z; raw[4 * i + 3] = r.w;
    }
    if (h) {
        T n[3];
        box_muller<T>(r, n);
        const Region<T>& R = lut[region ? region[i] : 0];
        const T sg = R.present != (T)0 ? R.sigma0 * th_scale : (T)0;
        h[i] = sg * n[0]; h[N + i] = sg * n[1]; h[2 * N + i] = sg * n[2];
    }
}

void thermal_raw_launch(mm_ctx* c, long long step, uint32_t* d_raw, void* d_h) {
    const double V = c->grid.dx * c->grid.dy * c->grid.dz;
    const double sc = c->Tr > 0 ? std::sqrt(c->Tr / (V * c->cfg.dt)) : 0.0;
    const unsigned blocks = (unsigned)((c->N + 255) / 256);
    const uint8_t* reg = c->uniform ? nullptr : (const uint8_t*)c->d_region;
    LaunchScope ls(c, "thermal_raw", 0.0);
    if (c->prec == 32)
        thermal_raw_kernel<float><<<blocks, 256, 0, c->stream>>>(c->N, (uint32_t)c->seed, (uint32_t)(c->seed >> 32),
                                                                 step, reg, (const Region<float>*)c->d_lut, (float)sc,
                                                                 d_raw, (float*)d_h);
    else
        thermal_raw_kernel<double><<<blocks, 256, 0, c->stream>>>(c->N, (uint32_t)c->seed, (uint32_t)(c->seed >> 32),
                                                                  step, reg, (const Region<double>*)c->d_lut, sc,
                                                                  d_raw, (double*)d_h);
}

}  // namespace mm
