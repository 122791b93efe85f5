// Per-cell effective field and LLG torque shared by the single-instance
// field kernel and the replica-batched stage kernel (Methods, "Physics and
// discretization", Eq. 1; the spin torques enter every integrator stage).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "ctx.h"

namespace mm {

// Philox4x32-10 (Salmon et al., SC'11): ten rounds, Weyl key schedule.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// u = ((x >> 8) + 1) 2^-24 in (0, 1]: exact in float and double
template <typename T> __device__ __forceinline__ T unit_uniform(uint32_t x) {
    return (T)((x >> 8) + 1u) * (T)5.9604644775390625e-08;
}

template <typename T> __device__ __forceinline__ void box_muller(U4 r, T* n) {
    const T u0 = unit_uniform<T>(r.x), u1 = unit_uniform<T>(r.y);
    const T u2 = unit_uniform<T>(r.z), u3 = unit_uniform<T>(r.w);
    T s1, c1, s3, c3;
    if (sizeof(T) == 4) {
        const float a = sqrtf(-2.0f * logf((float)u0)), b = sqrtf(-2.0f * logf((float)u2));
        float fs1, fc1, fs3, fc3;
        sincospif(2.0f * (float)u1, &fs1, &fc1);
        sincospif(2.0f * (float)u3, &fs3, &fc3);
        n[0] = (T)(a * fc1); n[1] = (T)(a * fs1); n[2] = (T)(b * fc3);
    } else {
        const double a = sqrt(-2.0 * log((double)u0)), b = sqrt(-2.0 * log((double)u2));
        double ds1, dc1, ds3, dc3;
        sincospi(2.0 * (double)u1, &ds1, &dc1);
        sincospi(2.0 * (double)u3, &ds3, &dc3);
        n[0] = (T)(a * dc1); n[1] = (T)(a * ds1); n[2] = (T)(b * dc3);
        (void)s1; (void)c1; (void)s3; (void)c3;
    }
}

template <typename T>
struct FieldArgs {
    const T* m;           // state the field is evaluated at, [3][N]
    const T* m0;          // HEUN2: base state
    const T* k1;          // HEUN2: predictor slope
    T* out;               // H | k | m* | m_new
    T* out2;              // HEUN1: k1
    const T* Hd;          // demag field or null
    const T* Bc;          // per-cell applied field (A/m) or null
    T hext[3];
    const uint8_t* region;
    const Region<T>* lut;
    const T* cpair;
    int nreg;
    T c_uniform;          // cpair[0] when there is one material
    Region<T> R0;         // that material's coefficients
    int nx, ny, nz;
    long long N;
    T hx, hy, hz;         // cell size
    T ix2, iy2, iz2;      // 1/h^2
    int px, py, pz;       // periodic flags
    unsigned terms;
    int mode;
    // thermal
    uint32_t key0, key1;
    T th_scale;           // sqrt(T / (V dt)); sigma = lut.sigma0 * th_scale
    const DevState* st;   // step counter, dt, active flag
    int gate;             // 1: skip the launch when st->active == 0
    long long step_override;  // >= 0: use this step for the noise
    T* const* kptr;       // MODE_K with out == null: write to the FSAL slot of stage kstage
    int kstage;           // 0 (k1) or 6 (k7)
    // torques
    int tq;               // mm_torque_kind
    T tq_base;            // SOT/STT: hbar J / (e mu0 t_F) (times 1/Ms -> A/m)
    T p[3];
    T theta_half, fl_ratio, P, L2, eps_p;
    T zl_u;               // J P mu_B / e [/(1+xi^2)] (times 1/Ms -> m/s)
    T xi;
    T dir[3];
    // further local terms
    T cubic_w1, cubic_w2; // weights of the Kc1 / Kc2 parts (1; 1/2 and 1/3 for energies)
    T strain[6];          // uniform strain xx yy zz xy xz yz
    const T* strain_cell; // per-cell strain [6][N] or null
    int rk1, rk2;         // RKKY layers
    T rkky_c;             // J / dz (times 1/(mu0 Ms) -> A/m per unit m)
};

// Thermal field of cell i at noise counter `step`: Philox4x32-10 keyed by
// (key0, key1) on the counter (i, step), Box-Muller, times
// sigma = sigma0 sqrt(T / (V dt)).
template <typename T>
__device__ __forceinline__ v3<T> thermal_h(const FieldArgs<T>& a, long long i, const Region<T>& R, long long step) {
    const U4 r = philox(U4{(uint32_t)i, (uint32_t)step, (uint32_t)((unsigned long long)step >> 32), 0u},
                        a.key0, a.key1);
    T n[3];
    box_muller<T>(r, n);
    const T sg = R.sigma0 * a.th_scale;
    return mk3<T>(sg * n[0], sg * n[1], sg * n[2]);
}

template <typename T>
__device__ __forceinline__ v3<T> ld3(const T* __restrict__ a, long long N, long long i) {
    return mk3<T>(__ldg(a + i), __ldg(a + N + i), __ldg(a + 2 * N + i));
}

template <typename T>
__device__ __forceinline__ void st3(T* a, long long N, long long i, v3<T> v) {
    a[i] = v.x;
    a[N + i] = v.y;
    a[2 * N + i] = v.z;
}

// Effective field of one present cell (x, y, z; linear index i) and, when
// want_k, its LLG slope with the configured spin torque.  hd is added as the
// demag field when the caller supplies it (batched path); a.Hd otherwise.
// Field and slope of one present cell from its six neighbour values
// (nbv, ghosts already substituted where absent), their raw presence nbp
// (Zhang-Li uses the cell itself for an absent neighbour) and exchange
// coefficients cnb.  use_hd: hdv is the demag field; otherwise a.Hd[i] is
// read (when set).  Neighbour arrays are only read when the
// exchange or DMI term or the Zhang-Li torque is on.
// as_omega: k receives instead the rotation vector Omega of the
// Depondt-Mertens scheme, dm/dt = Omega x m (Methods, "Integrators"): with
// -m x H = H x m and -m x (m x H) = (m x H) x m,
//   Omega = gamma' mu0 [H + alpha m x H]
//         + gamma' mu0 [(h_DL + alpha h_FL) m x p + (h_FL - alpha h_DL) p]
//         + [(1 + alpha xi) m x u' + (xi - alpha) u'] / (1 + alpha^2),
// u' = (u.grad) m, so that Omega x m is the slope.
// EXT = false compiles out bulk DMI and the further local terms (cubic,
// surface, RKKY, magnetoelastic): the lean kernel for contexts without them.
// QUIET = true also compiles out the thermal field and every spin torque
// (contexts at T = 0 without current).
template <typename T, bool EXT = true, bool QUIET = false>
__device__ __forceinline__ void cell_field_nb(const FieldArgs<T>& a, long long i, const Region<T>& R,
                                              const v3<T>& m, const v3<T>* nbv, const bool* nbp, const T* cnb,
                                              bool use_hd, const v3<T>& hdv, long long step, v3<T>& H, v3<T>& k,
                                              bool want_k, bool as_omega = false) {
    const long long N = a.N;
    H = mk3<T>(0, 0, 0);
    k = mk3<T>(0, 0, 0);
    if (a.terms & MM_TERM_EXCHANGE) {
        v3<T> e = mk3<T>(0, 0, 0);
        e = e + (a.ix2 * cnb[0]) * (nbv[0] - m) + (a.ix2 * cnb[1]) * (nbv[1] - m);
        e = e + (a.iy2 * cnb[2]) * (nbv[2] - m) + (a.iy2 * cnb[3]) * (nbv[3] - m);
        e = e + (a.iz2 * cnb[4]) * (nbv[4] - m) + (a.iz2 * cnb[5]) * (nbv[5] - m);
        H = H + e;
    }
    if (a.terms & MM_TERM_DMI) {
        const T gx = (T)0.5 / a.hx, gy = (T)0.5 / a.hy;
        const v3<T> dx = gx * (nbv[0] - nbv[1]);
        const v3<T> dy = gy * (nbv[2] - nbv[3]);
        H = H + R.dmi * mk3<T>(dx.z, dy.z, -dx.x - dy.y);
        if (EXT && R.dmib != (T)0) {
            // bulk: H = -(2 Db / mu0 Ms) curl m
            const v3<T> dz = ((T)0.5 / a.hz) * (nbv[4] - nbv[5]);
            H = H + (-R.dmib) * mk3<T>(dy.z - dz.y, dz.x - dx.z, dx.y - dy.x);
        }
    }
    if (a.terms & MM_TERM_ANISOTROPY) {
        const v3<T> u = mk3<T>(R.ux, R.uy, R.uz);
        H = H + (R.ku * dot(m, u)) * u;
    }
    if (a.terms & MM_TERM_ZEEMAN) {
        if (a.Bc) H = H + ld3(a.Bc, N, i);
        else H = H + mk3<T>(a.hext[0], a.hext[1], a.hext[2]);
    }
    if (EXT && (a.terms & MM_TERM_CUBIC)) {
        // -(1/mu0 Ms) dE/dm of Kc1 (a^2 b^2 + b^2 c^2 + c^2 a^2) + Kc2 a^2 b^2 c^2
        const v3<T> c1 = mk3<T>(R.c1x, R.c1y, R.c1z), c2 = mk3<T>(R.c2x, R.c2y, R.c2z);
        const v3<T> c3 = mk3<T>(R.c3x, R.c3y, R.c3z);
        const T p = dot(m, c1), q = dot(m, c2), r = dot(m, c3);
        const T p2 = p * p, q2 = q * q, r2 = r * r;
        const T k1 = R.kc1 * a.cubic_w1, k2 = R.kc2 * a.cubic_w2;
        const T g1 = k1 * p * (q2 + r2) + k2 * p * q2 * r2;
        const T g2 = k1 * q * (p2 + r2) + k2 * p2 * q * r2;
        const T g3 = k1 * r * (p2 + q2) + k2 * p2 * q2 * r;
        H = H - (g1 * c1 + g2 * c2 + g3 * c3);
    }
    if (EXT && (a.terms & MM_TERM_SURFACE)) {
        // (2 Ks / mu0 Ms dz) m_z z per free z face
        const T faces = (nbp[4] ? (T)0 : (T)1) + (nbp[5] ? (T)0 : (T)1);
        H.z += R.ks / a.hz * faces * m.z;
    }
    if (EXT && (a.terms & MM_TERM_RKKY)) {
        const long long plane = (long long)a.nx * a.ny;
        const int z = (int)(i / plane);
        if (z == a.rk1 || z == a.rk2) {
            const long long j = i + (long long)((z == a.rk1 ? a.rk2 : a.rk1) - z) * plane;
            const bool there = a.region ? a.lut[a.region[j]].present != (T)0 : true;
            if (there) H = H + (a.rkky_c * R.inv_mu0Ms) * ld3(a.m, N, j);
        }
    }
    if (EXT && (a.terms & MM_TERM_MEL)) {
        T e[6];
        if (a.strain_cell) {
#pragma unroll
            for (int k = 0; k < 6; ++k) e[k] = __ldg(a.strain_cell + k * N + i);
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) e[k] = a.strain[k];
        }
        H = H - mk3<T>(R.b1 * e[0] * m.x + R.b2 * (e[3] * m.y + e[4] * m.z),
                       R.b1 * e[1] * m.y + R.b2 * (e[3] * m.x + e[5] * m.z),
                       R.b1 * e[2] * m.z + R.b2 * (e[4] * m.x + e[5] * m.y));
    }
    if (a.terms & MM_TERM_DEMAG) {
        if (use_hd) H = H + hdv;
        else if (a.Hd) H = H + ld3(a.Hd, N, i);
    }
    if (!QUIET && (a.terms & MM_TERM_THERMAL) && a.th_scale != (T)0) H = H + thermal_h<T>(a, i, R, step);
    if (!want_k) return;
    // LLG torque, Eq. 1: -gamma' mu0 [m x H + alpha m x (m x H)]
    const v3<T> mxH = cross(m, H);
    if (as_omega) k = R.gm * (H + R.alpha * mxH);
    else k = (-R.gm) * (mxH + R.alpha * cross(m, mxH));
    if (QUIET) return;
    if (a.tq == MM_TORQUE_SOT || a.tq == MM_TORQUE_STT) {
        const v3<T> p = mk3<T>(a.p[0], a.p[1], a.p[2]);
        const T base = a.tq_base * R.inv_Ms;
        T hdl, hfl;
        if (a.tq == MM_TORQUE_SOT) {
            hdl = a.theta_half * base;
            hfl = a.fl_ratio * hdl;
        } else {
            const T eps = a.P * a.L2 / ((a.L2 + (T)1) + (a.L2 - (T)1) * dot(m, p));
            hdl = eps * base;
            hfl = a.eps_p * base;
        }
        const v3<T> mxp = cross(m, p);
        const T cdl = hdl + R.alpha * hfl, cfl = hfl - R.alpha * hdl;
        if (as_omega) k = k + R.gm * (cdl * mxp + cfl * p);
        else k = k + (-R.gm) * (cdl * cross(m, mxp) + cfl * mxp);
    } else if (a.tq == MM_TORQUE_ZL) {
        // (u.grad) m, central differences, absent neighbour = the cell itself
        const T u = a.zl_u * R.inv_Ms;
        v3<T> g = mk3<T>(0, 0, 0);
        const T hh[3] = {a.hx, a.hy, a.hz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (a.dir[d] == (T)0) continue;
            const v3<T> mp = nbp[2 * d] ? nbv[2 * d] : m;
            const v3<T> mm = nbp[2 * d + 1] ? nbv[2 * d + 1] : m;
            g = g + (a.dir[d] / ((T)2 * hh[d])) * (mp - mm);
        }
        const v3<T> ug = u * g;
        const v3<T> mxug = cross(m, ug);
        const T inv = (T)1 / ((T)1 + R.alpha * R.alpha);
        if (as_omega) k = k + inv * (((T)1 + R.alpha * a.xi) * mxug + (a.xi - R.alpha) * ug);
        else k = k + inv * ((-((T)1 + R.alpha * a.xi)) * cross(m, mxug) + (-(a.xi - R.alpha)) * mxug);
    }
}

__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }

// Rotation of m about w by the angle a = |w| dt, right-handed (Rodrigues):
//   m + s (w x m) + q (w (w.m) - |w|^2 m),  s = sin(a) / |w|,
//   q = (1 - cos a) / |w|^2,
// with sin a = 2 sin(a/2) cos(a/2) and 1 - cos a = 2 sin^2(a/2) from one
// half-angle sincos; for a^2 < 1e-6 (w = 0 included) the Taylor series
// sin(a)/a = 1 - a^2/6 + a^4/120 and (1 - cos a)/a^2 = 1/2 - a^2/24 + a^4/720
// (next terms below 1e-21).  For constant w this is the exact solution of
// dm/dt = w x m over dt.
template <typename T>
__device__ __forceinline__ v3<T> rodrigues(const v3<T>& m, const v3<T>& w, T dt) {
    const T w2 = dot(w, w);
    const T a2 = w2 * dt * dt;
    T s, q;
    if (a2 < (T)1e-6) {
        s = dt * ((T)1 - a2 * ((T)(1.0 / 6.0) - a2 * (T)(1.0 / 120.0)));
        q = dt * dt * ((T)0.5 - a2 * ((T)(1.0 / 24.0) - a2 * (T)(1.0 / 720.0)));
    } else {
        const T a = sqrt(a2);
        T sh, ch;
        sincos_t((T)0.5 * a, &sh, &ch);
        s = dt * ((T)2 * sh * ch) / a;
        q = dt * dt * ((T)2 * sh * sh) / a2;
    }
    return m + s * cross(w, m) + q * (dot(w, m) * w - w2 * m);
}

// Ghost value of an absent neighbour in direction d (0 x, 1 y, 2 z) and
// side sg (+1 / -1): m - h (D/2A) (z x n) x m with n = sg e_d, plus (EXT)
// the bulk-DMI part + h (Db/2A) n x m.
template <typename T, bool EXT = true>
__device__ __forceinline__ v3<T> ghost_value(const v3<T>& m, int d, int sg, T h, T ratio, T ratio_b) {
    v3<T> zn = mk3<T>(0, 0, 0);
    if (d == 0) zn = mk3<T>(sg * m.z, (T)0, -sg * m.x);
    else if (d == 1) zn = mk3<T>((T)0, sg * m.z, -sg * m.y);
    v3<T> g = m - (h * ratio) * zn;
    if (EXT && ratio_b != (T)0) {
        // bulk DMI: + h (Db/2A) n x m, n = sg e_d
        v3<T> nm;
        if (d == 0) nm = mk3<T>((T)0, -sg * m.z, sg * m.y);
        else if (d == 1) nm = mk3<T>(sg * m.z, (T)0, -sg * m.x);
        else nm = mk3<T>(-sg * m.y, sg * m.x, (T)0);
        g = g + (h * ratio_b) * nm;
    }
    return g;
}

// Effective field of one present cell (x, y, z; linear index i) and, when
// want_k, its LLG slope with the configured spin torque (as_omega: the
// rotation vector, see cell_field_nb).  UNIF: one material
// everywhere (no region map): every in-grid neighbour is present and every
// exchange pair uses the one coefficient a.c_uniform.
template <typename T, bool UNIF = false, bool EXT = true>
__device__ __forceinline__ void cell_field(const FieldArgs<T>& a, int x, int y, int z, long long i, int ri,
                                           const Region<T>& R, const v3<T>& m, const v3<T>* hd, long long step,
                                           v3<T>& H, v3<T>& k, bool want_k, bool as_omega = false) {
    const long long N = a.N;
    const unsigned nbt = MM_TERM_EXCHANGE | MM_TERM_DMI | (EXT ? MM_TERM_SURFACE : 0u);
    const bool need_nb = (a.terms & nbt) || a.tq == MM_TORQUE_ZL;
    // neighbour values (ghosts where absent) and raw presence (Zhang-Li,
    // the free faces of the surface term)
    v3<T> nbv[6];
    bool nbp[6];
    T cnb[6];
    if (need_nb) {
        const int dims[3] = {a.nx, a.ny, a.nz};
        const int per[3] = {a.px, a.py, a.pz};
        const int pos[3] = {x, y, z};
        const long long strides[3] = {1, a.nx, (long long)a.nx * a.ny};
        const T hh[3] = {a.hx, a.hy, a.hz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int sg = s == 0 ? 1 : -1;
                int q = pos[d] + sg;
                bool inside = q >= 0 && q < dims[d];
                if (!inside && per[d]) { q = (q + dims[d]) % dims[d]; inside = true; }
                bool present = false;
                long long j = 0;
                int rj = 0;
                if (inside) {
                    j = i + (long long)(q - pos[d]) * strides[d];
                    if constexpr (UNIF) {
                        present = true;
                    } else {
                        rj = a.region ? a.region[j] : 0;
                        present = a.lut[rj].present != (T)0;
                    }
                }
                const int slot = 2 * d + s;
                nbp[slot] = present;
                if (present) {
                    nbv[slot] = ld3(a.m, N, j);
                    cnb[slot] = UNIF ? a.c_uniform : __ldg(&a.cpair[ri * a.nreg + rj]);
                } else {
                    nbv[slot] = ghost_value<T, EXT>(m, d, sg, hh[d], R.ratio, R.ratio_b);
                    cnb[slot] = R.cg;
                }
            }
        }
    }
    cell_field_nb<T, EXT>(a, i, R, m, nbv, nbp, cnb, hd != nullptr, hd ? *hd : mk3<T>(0, 0, 0), step, H, k, want_k,
                     as_omega);
}

}  // namespace mm
