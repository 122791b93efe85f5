/*
 * mm.h — C ABI of the GB300 (sm_103a) micromagnetic LLG hot path.
 *
 * What the library computes (arxiv 2608.15253, Methods):
 *  - "Physics and discretization", Eq. 1: the Landau-Lifshitz-Gilbert
 *    equation dm/dt = -gamma' mu0 m x H - gamma' alpha mu0 m x (m x H),
 *    gamma' = gamma0/(1+alpha^2), on a structured x-fastest finite-difference
 *    grid; H sums six-point exchange (Neumann or periodic), interfacial DMI
 *    with the free edge condition at grid and mask edges, uniaxial
 *    anisotropy, Zeeman, the stochastic thermal field and open-boundary
 *    demagnetisation (FFT convolution with the Newell tensor zero-padded to
 *    2N); spin-orbit, Slonczewski and Zhang-Li torques are added per stage.
 *  - "Integrators": Heun (stochastic LLG, Stratonovich) and RK45
 *    Dormand-Prince (adaptive, first-same-as-last), |m| renormalised.
 *  - "Replica batching": R independent replicas, replica-outermost /
 *    component-major / x-fastest state, per-replica J, T and Philox seeds.
 *
 * Conventions for every call:
 *  - SI units: metres, A/m for Ms, J/m for A, J/m^3 for Ku1, J/m^2 for D,
 *    tesla for applied fields, kelvin, A/m^2 for current density, seconds.
 *  - Vector fields on the host are float64, component-major and x-fastest:
 *    v[c*N + (z*ny + y)*nx + x], N = nx*ny*nz of that replica.
 *  - Host arrays passed in are copied before the call returns; the caller
 *    keeps ownership and the library never keeps a caller pointer.  Output
 *    arrays are caller-allocated.
 *  - Every call returns mm_status; MM_OK is 0.  On error the context stays
 *    valid and destroyable; mm_last_error() describes the last failure.
 *  - A context is not thread-safe.  Its precision is fixed at creation.
 *  - Device work runs on the context's stream (mm_set_stream); calls that
 *    return host data synchronise that stream.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MM_API __attribute__((visibility("default")))

typedef struct mm_ctx mm_ctx;

typedef enum mm_status {
    MM_OK = 0,
    MM_ERR_ARG = 1,           /* invalid argument (message in mm_last_error) */
    MM_ERR_DEVICE = 2,        /* no sm_103 device, or kernel image does not match */
    MM_ERR_OOM = 3,           /* device allocation failed */
    MM_ERR_CUDA = 4,          /* any other CUDA runtime error */
    MM_ERR_NONFINITE = 5,     /* NaN/Inf detected in the state or the error norm */
    MM_ERR_DT_UNDERFLOW = 6,  /* RK45 step fell below dt_min */
    MM_ERR_TIMEOUT = 7,       /* a bounded device wait ran out */
    MM_ERR_STATE = 8          /* call not valid in the current state */
} mm_status;

/* Integrators (Methods, "Integrators"): Heun (fixed dt, thermal field
 * allowed), Dormand-Prince RK45 (adaptive, FSAL), classical RK4 (fixed dt,
 * four evaluations, |m| restored after each step), and the Depondt-Mertens
 * rotation scheme MM_DM (fixed dt, thermal field allowed; the integrator of
 * the replica-batched engine): with dm/dt = Omega x m,
 *   Omega = gamma' mu0 (H + alpha m x H) + spin-torque terms,
 * the predictor rotates m about Omega(m) by |Omega| dt (Rodrigues), the
 * corrector rotates the step's initial m about the mean of Omega(m) and
 * Omega(predictor); one thermal draw serves both.  Rotations keep |m| = 1;
 * the corrector also rescales by 1/|m| (a round-off-level change). */
enum mm_integrator { MM_HEUN = 0, MM_RK45 = 1, MM_RK4 = 2, MM_DM = 3, MM_DM_ADAPTIVE = 4 };
/* MM_DM_ADAPTIVE (Methods: the Depondt-Mertens scheme run with an adaptive
 * step; T = 0 only): the predictor m* (first order) and the corrector
 * (second order) form an embedded pair, err = max over cells |m_new - m*|;
 * accept when err <= rtol; dt *= clamp(0.9 (rtol/err)^(1/2), 0.2, 5), capped
 * at 1 after a rejection, within [dt_min, dt_max]; the controller runs on
 * the device like RK45's, and mm_step_dt replays a given step sequence. */
enum mm_demag_mode { MM_DEMAG_OFF = 0, MM_DEMAG_EXACT = 1, MM_DEMAG_SURROGATE = 2 };

/* Effective-field terms (bit mask). */
enum mm_term {
    MM_TERM_EXCHANGE = 1,
    MM_TERM_DMI = 2,
    MM_TERM_ANISOTROPY = 4,
    MM_TERM_ZEEMAN = 8,
    MM_TERM_DEMAG = 16,
    MM_TERM_THERMAL = 32,
    MM_TERM_CUBIC = 64,       /* cubic anisotropy (mm_material Kc1, Kc2, c1, c2) */
    MM_TERM_SURFACE = 128,    /* surface anisotropy at free z faces (Ks) */
    MM_TERM_RKKY = 256,       /* RKKY interlayer exchange (mm_set_rkky) */
    MM_TERM_MEL = 512,        /* magnetoelastic anisotropy (B1, B2, mm_set_strain) */
    MM_TERM_ALL = 1023        /* terms whose parameters are all zero are skipped */
};

/* Energy array layout returned by mm_energy. */
enum mm_energy_index { MM_E_EXCHANGE = 0, MM_E_DMI = 1, MM_E_ANISOTROPY = 2, MM_E_ZEEMAN = 3,
                       MM_E_DEMAG = 4, MM_E_TOTAL = 5, MM_E_CUBIC = 6, MM_E_SURFACE = 7,
                       MM_E_RKKY = 8, MM_E_MEL = 9, MM_NENERGY = 10 };

enum mm_torque_kind { MM_TORQUE_NONE = 0, MM_TORQUE_SOT = 1, MM_TORQUE_STT = 2, MM_TORQUE_ZL = 3 };

/* Grid of one replica: nx*ny*nz cells of dx*dy*dz metres.  pbc[d] > 0 makes
 * axis d periodic: the local stencils (exchange, DMI, Zhang-Li) wrap, and
 * the demag field (Methods: periodic-boundary demagnetisation by an
 * image-sum kernel) is that of the sample and its copies shifted by
 * a * n_d cells for |a| <= pbc[d], seen from the central copy (the Newell
 * tensor summed over those images, then the usual zero-padded FFT
 * convolution).  pbc[d] in [0, 4096]. */
typedef struct mm_grid {
    int nx, ny, nz;
    double dx, dy, dz;
    int pbc[3];
} mm_grid;

/* Material.  Scalars apply to every cell unless the matching per-cell host
 * array (length N; u_cell 3N component-major) is non-NULL.  Cells with
 * Ms = 0 are absent (the geometry mask).  At most 256 distinct parameter
 * tuples per context (they become material regions).  D: interfacial DMI
 * (J/m^2).  D_bulk: bulk DMI (Methods, "Physics and discretization"),
 * energy density D_bulk m.(curl m), field -(2 D_bulk / mu0 Ms) curl m by
 * central differences in x, y and z; at a free face with outward normal n
 * its boundary condition dm/dn = (D_bulk/2A) n x m enters the ghost value
 * (film tops and bottoms included).  Both belong to MM_TERM_DMI. */
typedef struct mm_material {
    double Ms, A, alpha, Ku1, u[3], D;
    const double *Ms_cell, *A_cell, *alpha_cell, *Ku1_cell, *u_cell, *D_cell;
    double D_bulk;
    const double* D_bulk_cell;
    /* Further anisotropies (Methods, "Physics and discretization"), uniform
     * over the material's present cells:
     *  cubic: energy density Kc1 (a^2 b^2 + b^2 c^2 + c^2 a^2) + Kc2 a^2 b^2 c^2,
     *    a, b, c the components of m on the axes c1, c2 (its c1 component
     *    removed) and c3 = c1 x c2 (J/m^3);
     *  surface: -Ks (m.z)^2 per area of every free z face of a cell, an
     *    absent neighbour above or below (J/m^2);
     *  magnetoelastic: B1 (e_xx m_x^2 + e_yy m_y^2 + e_zz m_z^2) +
     *    2 B2 (e_xy m_x m_y + e_xz m_x m_z + e_yz m_y m_z) with the strain of
     *    mm_set_strain (J/m^3). */
    double Kc1, Kc2, c1[3], c2[3];
    double Ks;
    double B1, B2;
} mm_material;

typedef struct mm_config {
    int precision;            /* 32 or 64: arithmetic of the state, fields, FFTs */
    int integrator;           /* MM_HEUN, MM_RK45, MM_RK4, MM_DM or MM_DM_ADAPTIVE */
    int demag;                /* mm_demag_mode */
    unsigned terms;           /* mm_term mask of the effective field; 0 means all */
    double dt;                /* Heun / RK4 step; RK45 initial step (s) */
    double rtol;              /* RK45: accept when max_cell |m5 - m4| <= rtol */
    double dt_min, dt_max;    /* RK45 step bounds (s); 0 selects 1e-20 / 1e-11 */
    double T;                 /* temperature (K) of every replica (Heun only; > 0 is rejected otherwise) */
    uint64_t seed;            /* base Philox seed; replica r uses splitmix64(seed + r) */
} mm_config;

/* Spin-torque parameters (Methods: the torques enter every integrator stage).
 * Landau-Lifshitz form with damping-like h_DL and field-like h_FL along p:
 *   tau = -gamma' mu0 [(h_DL + alpha h_FL) m x (m x p) + (h_FL - alpha h_DL) m x p]
 *  SOT: h_DL = theta_SH hbar J / (2 e mu0 Ms t_F), h_FL = fl_ratio * h_DL
 *  STT: h_DL = eps(m) hbar J / (e mu0 Ms t_F), h_FL = eps_prime hbar J / (e mu0 Ms t_F),
 *       eps = P Lambda^2 / ((Lambda^2 + 1) + (Lambda^2 - 1) m.p)
 *  ZL:  u = J P mu_B / (e Ms) along dir (divided by 1 + xi^2 when match_mumax),
 *       tau = [-(1 + alpha xi) m x (m x (u.grad)m) - (xi - alpha) m x (u.grad)m] / (1 + alpha^2)
 * t_F <= 0 selects nz * dz. */
typedef struct mm_torque {
    int kind;                 /* mm_torque_kind */
    double p[3];
    double theta_SH, fl_ratio;
    double P, Lambda, eps_prime;
    double t_F;
    double xi;
    double dir[3];
    int match_mumax;
} mm_torque;

typedef struct mm_stats {
    long long accepted, rejected, attempts;
    long long kernel_launches;  /* kernels of this library launched by the context */
    double t, dt;
} mm_stats;

/* Per-kernel timing collected while profiling is on (mm_set_profiling). */
typedef struct mm_profile_entry {
    char name[32];
    long long launches;
    double total_ms;          /* sum of CUDA-event durations on the context stream */
    double bytes_per_launch;  /* algorithmic bytes of one launch */
} mm_profile_entry;

/* Create a single-instance context (Methods, "Physics and discretization").
 * Allocates device memory, validates the device (compute capability 10.3),
 * computes the FP64 Newell tensor spectrum on the GPU when demag is on.
 * m starts along +z.  Errors: MM_ERR_ARG (sizes <= 0, bad precision or
 * integrator, RK45 or RK4 with T > 0, > 256 materials), MM_ERR_DEVICE,
 * MM_ERR_OOM. */
MM_API mm_status mm_create(const mm_grid* grid, const mm_material* mat,
                           const mm_config* cfg, mm_ctx** out);

/* Create R replicas of possibly different grids sharing one material
 * (Methods, "Replica batching"): state replica-outermost, each replica with
 * its own Philox key (seeds[r], or splitmix64(cfg->seed + r) when seeds is
 * NULL), temperature (mm_set_temperature) and current (mm_set_torque).
 * R = 1 is the single-instance context.  For R > 1: FP32, Heun or
 * Depondt-Mertens, nz = 1 open films sharing one cell size and one uniform
 * material (Ms > 0);
 * nx, ny may differ per replica (sizes of the same shape share one tensor
 * spectrum).  A stage runs as one persistent launch or, in the stacked
 * shape, as per-size-class passes (mm_batch_autotune picks the shape,
 * mm_batch_set_shape sets it; retire/refill runs on both).  Errors:
 * MM_ERR_ARG for any other combination. */
MM_API mm_status mm_create_batch(int R, const mm_grid* grids, const mm_material* mat,
                                 const mm_config* cfg, const uint64_t* seeds, mm_ctx** out);

/* Free the context and every device buffer it owns; NULL is accepted.
 * No passage: boundary convenience (the paper's solver objects are C++
 * values with automatic lifetime). */
MM_API mm_status mm_destroy(mm_ctx* ctx);

/* Run on a caller stream (cudaStream_t, e.g. torch's current stream); NULL
 * returns to the context's own stream.  Cached CUDA graphs are rebuilt.
 * No passage: boundary convenience (stream interop with the caller). */
MM_API mm_status mm_set_stream(mm_ctx* ctx, void* stream);

/* Set / read the magnetisation of one replica (Methods, "Physics and
 * discretization": the unit vector m of Eq. 1 on the x-fastest grid; host
 * float64, 3N, layout [component][z][y][x]).  Page-locked host memory is read / written in place
 * by the conversion kernel (one pass over the host link); pageable memory
 * goes through a device staging buffer (3N doubles, allocated on first use
 * and kept).  Input is renormalised per cell unless its length is already
 * 1 to within a few units in the last place of the context's precision
 * (|m|^2 - 1 within 4.8e-7 in FP32, 8.9e-16 in FP64), in which case it is
 * taken as it is; absent cells and zero vectors are set to zero.  A state
 * read with mm_get_m and written back unchanged is therefore the same bit
 * for bit, and mm_set_m then keeps the integrator's first-same-as-last
 * slope (any changed cell discards it).  Both calls
 * return after the copy has completed (they synchronise the context
 * stream).  Errors: MM_ERR_ARG (bad replica, NULL m), MM_ERR_OOM, MM_ERR_CUDA. */
MM_API mm_status mm_set_m(mm_ctx* ctx, int replica, const double* m);
MM_API mm_status mm_get_m(mm_ctx* ctx, int replica, double* m);

/* Device-pointer variants over all replicas at once (Methods, "Replica
 * batching": replica-outermost, component-major state), in the context's
 * precision (float or double), concatenated replica-outermost in storage
 * order: replicas of one grid size are stored together (sizes in order of
 * first appearance, replicas by index within a size), which is replica
 * order when the replicas come grouped by size.  Ordered on the context
 * stream; no host synchronisation. */
MM_API mm_status mm_set_m_device(mm_ctx* ctx, const void* m_dev);
MM_API mm_status mm_get_m_device(mm_ctx* ctx, void* m_dev);

/* Applied field B (tesla) of the Zeeman term (Methods, "Physics and
 * discretization": H += B/mu0): uniform B[3], or per cell (3N) when
 * B_cell != NULL; B == NULL means zero.  Errors: MM_ERR_ARG (bad replica,
 * per-cell field on a replica-batched context), MM_ERR_OOM, MM_ERR_CUDA. */
MM_API mm_status mm_set_field(mm_ctx* ctx, int replica, const double B[3], const double* B_cell);

/* Strain tensor of the magnetoelastic term (Methods, "Physics and
 * discretization": magnetoelastic anisotropy): eps[6] = xx, yy, zz, xy, xz, yz
 * for every cell, or per cell (eps_cell, 6N doubles component-major) when
 * eps_cell != NULL.  Replica-batched contexts take the uniform form only.
 * Errors: MM_ERR_ARG (both NULL), MM_ERR_OOM. */
MM_API mm_status mm_set_strain(mm_ctx* ctx, const double eps[6], const double* eps_cell);

/* RKKY interlayer exchange (Methods, "Physics and discretization") between
 * layers k1 and k2 (z indices, usually on either side of an Ms = 0 spacer):
 * energy -J m(k1).m(k2) per column area (J in J/m^2, J > 0 favours
 * parallel moments), so a coupled cell sees (J / (mu0 Ms dz)) times its
 * partner's moment where both cells are present.  J = 0 turns the
 * coupling off.  Errors: MM_ERR_ARG (layers out of range or equal),
 * MM_ERR_STATE (replica-batched context). */
MM_API mm_status mm_set_rkky(mm_ctx* ctx, int k1, int k2, double J);

/* Temperature per replica (R values, kelvin) of the thermal field
 * (Methods, "Physics and discretization": stochastic LLG, sigma =
 * sqrt(2 alpha kB T / (mu0^2 Ms V gamma0 dt)); "Replica batching":
 * per-replica T).  Errors: MM_ERR_ARG (NULL, negative T, T > 0 with an
 * integrator other than Heun or Depondt-Mertens), MM_ERR_STATE (while
 * retire/refill owns the temperatures). */
MM_API mm_status mm_set_temperature(mm_ctx* ctx, const double* T);

/* Spin torque of every replica (Methods, "Physics and discretization":
 * spin-orbit, Slonczewski and Zhang-Li torques added in every integrator
 * stage; "Replica batching": per-replica J); J holds R current densities
 * (A/m^2); J == NULL means zero current.  Errors: MM_ERR_ARG (NULL tq,
 * unknown kind, Zhang-Li on a replica-batched context), MM_ERR_STATE
 * (while retire/refill owns the currents). */
MM_API mm_status mm_set_torque(mm_ctx* ctx, const mm_torque* tq, const double* J);

/* Advance n steps (Methods, "Integrators"): n fixed steps (Heun, RK4,
 * Depondt-Mertens), or n accepted adaptive steps (rejected attempts are
 * retried on the device; the step controller runs on the device).
 * Errors: MM_ERR_NONFINITE, MM_ERR_DT_UNDERFLOW (the context stays usable
 * at the last accepted state), MM_ERR_CUDA. */
MM_API mm_status mm_step(mm_ctx* ctx, long n);

/* RK45 or adaptive Depondt-Mertens (Methods, "Integrators") with a
 * prescribed step sequence (no control, every step accepted): replays
 * dts[0..n-1], e.g. the accepted steps of a reference run; the replay
 * itself has no passage (a parity-testing convenience).  Errors:
 * MM_ERR_STATE (fixed-step integrator), MM_ERR_ARG (dts NULL with n > 0,
 * n < 0), then as mm_step. */
MM_API mm_status mm_step_dt(mm_ctx* ctx, const double* dts, long n);

/* Advance to simulated time t_end (Methods, "Integrators"); the last step
 * is clipped to land on it.  Errors as mm_step. */
MM_API mm_status mm_run(mm_ctx* ctx, double t_end);

/* Effective field H of Eq. 1 (Methods, "Physics and discretization") at
 * the current state (A/m, host float64 3N) restricted to the terms in
 * term_mask (MM_TERM_THERMAL uses the current step's noise).  Errors:
 * MM_ERR_ARG (bad replica, NULL H). */
MM_API mm_status mm_get_heff(mm_ctx* ctx, int replica, double* H, unsigned term_mask);

/* Energy per term and total (joules; Results, "A showcase of representative
 * examples": the total energy of the S-state and vortex branches whose
 * exchange/demagnetisation balance the paper compares): E[MM_NENERGY], FP64
 * compensated sums of -1/2 mu0 Ms m.H_term V (Zeeman -mu0 Ms m.H_ext V);
 * E[MM_E_TOTAL] sums every term, those indexed after it included.  Errors:
 * MM_ERR_ARG (bad replica, NULL E). */
MM_API mm_status mm_energy(mm_ctx* ctx, int replica, double* E);

/* Topological charge (Results, "A showcase of representative examples":
 * the relaxed skyrmion charge Q of the D-K phase diagram)
 * Q = (1/4pi) sum m.(dm/dx x dm/dy) dx dy of layer `layer`, or the mean
 * over layers when layer = -1; central differences, one-sided at edges and
 * holes; FP64 compensated sum.  Errors: MM_ERR_ARG (bad replica,
 * layer >= nz or layer < -1, NULL Q). */
MM_API mm_status mm_topo_charge(mm_ctx* ctx, int replica, int layer, double* Q);

/* Mean magnetisation <m> (Results: the average magnetisation the standard
 * problems and relaxation runs report): the average of the unit vectors m
 * over the present cells (Ms > 0) of the replica, or of z-layer `layer`
 * when layer >= 0; FP64 compensated sums of the working-precision state.
 * m_mean: host double[3], written only on success (zeros when no cell of
 * the selection is present).  Errors: MM_ERR_ARG (bad replica, layer >= nz,
 * m_mean NULL), MM_ERR_CUDA. */
MM_API mm_status mm_mean_m(mm_ctx* ctx, int replica, int layer, double* m_mean);

/* Simulated time, current step size and accepted steps of a replica, and
 * the context's step / launch counters.  No passage: boundary convenience.
 * Outputs may be NULL (mm_get_time).  Errors: MM_ERR_ARG (bad replica). */
MM_API mm_status mm_get_time(mm_ctx* ctx, int replica, double* t, double* dt, long long* steps);
MM_API mm_status mm_get_stats(mm_ctx* ctx, mm_stats* st);

/* Checkpoint: m, t, dt, step counters, seeds and the FSAL slope.  With
 * buf == NULL the required size is returned in *nbytes.  No passage:
 * boundary convenience (the paper has no checkpoint); resume is bit-exact
 * because the thermal stream is counter-based (Methods, "Replica
 * batching").  Errors: MM_ERR_ARG (buffer too small, foreign blob, or an
 * integrator record that no run produces: slope slot other than 0 or 6,
 * non-finite t, negative or non-finite dt), checked before anything is
 * copied to the device. */
MM_API mm_status mm_get_state(mm_ctx* ctx, void* buf, size_t* nbytes);
MM_API mm_status mm_set_state(mm_ctx* ctx, const void* buf, size_t nbytes);

/* Thermal noise of one replica at a given step counter (Methods,
 * "Replica batching": counter-based Philox keyed by seed, replica-and-cell
 * index and step): raw Philox4x32-10 words (4N uint32, cell-major) and/or
 * the thermal field (3N A/m) for the context's dt; either output may be
 * NULL. */
MM_API mm_status mm_get_thermal(mm_ctx* ctx, int replica, long long step,
                                uint32_t* raw, double* H_th);

/* Demagnetisation tensor spectrum (Methods, "Physics and discretization":
 * the Newell tensor, zero-padded to 2N) in the stored form: n_out doubles of
 * [ncomp][Pz/2+1][Py/2+1][Px/2+1] (ncomp 6: xx,yy,zz,xy,xz,yz; 4 when nz=1),
 * scaled by -1/(Px Py Pz).  dims_out[0..3] = ncomp, Px, Py, Pz. */
MM_API mm_status mm_get_demag_kernel(mm_ctx* ctx, double* out, size_t n_out, int* dims_out);

/* FP64 Newell tensor (Methods, "Physics and discretization") evaluated on
 * the GPU at count integer displacements
 * ijk[3*q..3*q+2] of cells dx*dy*dz; out[6*q+c] in xx,yy,zz,xy,xz,yz. */
MM_API mm_status mm_newell(long count, const int* ijk, double dx, double dy, double dz, double* out);

/* Retire/refill of batched trials (Results, "Replica batching"): the slots
 * of a replica-batched context (R >= 2 replicas of one grid) run n_trials
 * independent trials.  Trial q has current density J[q] (A/m^2, with the
 * context's torque, mm_set_torque) and temperature T[q] (K), Philox key
 * splitmix64(base_seed + q) and its own step counter (from 0) as the noise
 * counter, and starts from m_init (host float64, [3][ny][nx], renormalised
 * per cell).  After every step a slot whose trial has
 *     mean over cells of m . axis/|axis| <= threshold     (stopped = 1)
 * or has taken max_steps steps (stopped = 0) records the trial's step count
 * and, with refill, starts the next trial not yet begun (a fresh noise
 * stream); otherwise, or when none is left, the slot idles.  A trial's
 * outcome depends on q alone, not on its slot or start step.  Slots start
 * with trials 0 .. min(R, n_trials) - 1 at the current step; mm_step
 * advances every busy slot.  Per-replica temperatures and currents set
 * before are replaced.  Errors: MM_ERR_STATE (single-instance context),
 * MM_ERR_ARG (replicas of different sizes, n_trials < 1, max_steps < 1,
 * NULL tables, negative T, zero axis). */
typedef struct mm_trials {
    long long n_trials;
    const double* J;          /* [n_trials] */
    const double* T;          /* [n_trials] */
    const double* m_init;     /* [3][ny][nx] */
    double axis[3];
    double threshold;
    long long max_steps;
    uint64_t base_seed;
    int refill;               /* 1: a finished slot starts the next trial */
} mm_trials;
MM_API mm_status mm_trials_start(mm_ctx* ctx, const mm_trials* spec);

/* Outcomes so far of the retire/refill trials (Results, "A replica-batched
 * engine for finite-temperature ensembles": switching probability from the
 * trials' stop steps; synchronises the context stream): steps[q] = steps the
 * trial took (-1 while unfinished or not started), stopped[q] = 1 if the
 * stop condition ended it; *done = finished trials.  Any output may be NULL.
 * Errors: MM_ERR_STATE before mm_trials_start. */
MM_API mm_status mm_trials_result(mm_ctx* ctx, long long* steps, int* stopped, long long* done);

/* Launch-shape autotuner of a replica-batched context (Methods, "Replica
 * batching").  Candidates: one persistent launch per stage (threads per CTA
 * x resident CTAs per SM), and the stacked shape (*nt_out = *blocks_out =
 * 0): per size class, the 2-D demag passes and the field + stage kernel
 * over all of the class's replicas at once (not used with retire/refill).
 * Times a few steps for every candidate, keeps the fastest and restores
 * the state (m, t, step counters) afterwards.  When
 * cache_path is non-NULL the choice is read from / appended to that JSON
 * file, keyed by the replica-size histogram.  nt_out / blocks_out may be
 * NULL.  MM_ERR_STATE for single-instance contexts. */
MM_API mm_status mm_batch_autotune(mm_ctx* ctx, const char* cache_path, int* nt_out, int* blocks_out);

/* Set the launch shape of a replica-batched context (Methods, "Replica
 * batching") directly, bypassing the autotuner: nt = 256 or
 * 512 threads per CTA with `blocks` persistent CTAs (1 <= blocks), or
 * nt = 0 for the stacked shape (blocks ignored).  Errors: MM_ERR_STATE
 * (single-instance context), MM_ERR_ARG (other values), MM_ERR_OOM (the
 * stacked shape's per-class buffers). */
MM_API mm_status mm_batch_set_shape(mm_ctx* ctx, int nt, int blocks);

/* Topological charge without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * device memory -- code running while a CUDA graph is captured (a plain
 * cudaMalloc is not allowed there), loops that must never enter the
 * allocator, and hosts whose device memory belongs to another framework's
 * pool.  The caller passes the state m_dev (device, [3][nz][ny][nx] in
 * `precision` 32 = float or 64 = double, every cell present) and the output
 * Q_dev (one device double); the result is the same quantity as
 * mm_topo_charge (layer = -1: mean over layers).  Work is ordered on
 * `stream` (cudaStream_t, NULL = default stream); nothing is synchronised.
 * The only scratch is a fixed 64 KiB file-scope device array (one partial
 * sum per block of 4096 cells) that every GPU loading the library keeps
 * until exit; the first call on a device looks up its address, so make
 * that first call before any stream capture.  Calls share the array:
 * calls that overlap on the GPU race.  No cudaMalloc, cudaFree or
 * allocating library routine is used.  Errors: MM_ERR_ARG for bad
 * arguments (layer >= nz or < -1 included) or more than 16,777,216 cells
 * (4096 blocks) in the reduced range; MM_ERR_STATE, with nothing launched,
 * when a CUDA error from earlier work is already pending on the calling
 * thread (it is left in place, not consumed); MM_ERR_DEVICE / MM_ERR_CUDA
 * for this call's own runtime failures. */
MM_API mm_status mm_topo_charge_noalloc(const void* m_dev, int precision, int nx, int ny, int nz,
                                        double dx, double dy, int layer, double* Q_dev, void* stream);

/* ---- learned demag surrogate (the benchmark's own addition; not in the paper)
 * A 4-layer CNN (3 -> 32 -> 32 -> 32 -> 3 channels, 5x5 kernels, ReLU after
 * layers 1-3) with BF16 operands and FP32 accumulation on the tensor cores
 * maps a magnetisation increment dm = m - m_ref (scaled by c_in) to the demag
 * increment H_demag(dm) / Ms (scaled by c_in); the demag field is linear in
 * m, so between exact FFT evaluations H ~ H_exact(m_ref) + CNN(m - m_ref).
 * Single-instance FP32 nz = 1 contexts with exact demag only. */
typedef struct mm_train_cfg {
    int n_snapshots;   /* exact RK45 snapshots from the current state */
    int snap_every;    /* accepted RK45 steps between snapshots */
    int max_gap;       /* pairs (i, j), 1 <= j - i <= max_gap, give dm = m_j - m_i */
    int crop;          /* training window edge (cells, <= nx, ny) */
    int batch;         /* windows per optimisation step */
    int steps;         /* optimisation steps */
    double lr;         /* Adam learning rate */
    uint64_t seed;     /* window positions and weight initialisation */
} mm_train_cfg;

typedef struct mm_surrogate_stats {
    long long exact_evals;      /* exact FFT demag evaluations while stepping */
    long long surrogate_evals;  /* network evaluations while stepping */
    long long refreshes;        /* exact refreshes of (m_ref, H_ref) */
    int fallback;               /* 1 once the monitored error passed the threshold */
    double last_error;          /* max|H_pred - H_exact| / max|H_exact| at the last refresh */
    double max_error;
    double train_loss;          /* last training loss */
    double c_in;                /* network input scale (input = c_in dm) */
    double c_out;               /* network output scale (output = c_out dH_far / Ms) */
} mm_surrogate_stats;

/* Generate (dm, H_demag(dm)) pairs with the exact FFT path from a relaxation
 * started at the current state (the state is restored afterwards) and train
 * the network with the library's own BF16 forward/backward kernels and Adam.
 * Prediction model between exact refreshes:
 *   H(m) = H_ref - Ms N_near * dm + Ms CNN(c_in dm) / c_out,  dm = m - m_ref,
 * where N_near is the exact Newell tensor on in-plane displacements
 * |dx|, |dy| <= 5 (a fixed convolution) and the network is trained on what
 * it leaves over, c_out (H_demag(dm) + Ms N_near * dm) / Ms, with
 * c_in = 1 / rms(dm) and c_out = 1 / rms of that remainder over the
 * training pairs.  final_loss may be NULL. */
MM_API mm_status mm_surrogate_train(mm_ctx* ctx, const mm_train_cfg* cfg, double* final_loss);

/* k >= 1: every k-th attempted step refreshes (m_ref, H_ref) with the exact
 * demag and first compares the network's prediction at that state with the
 * exact field; above tol (relative, max norm) every later evaluation is exact
 * (fallback).  k = 0 turns the surrogate off. */
MM_API mm_status mm_surrogate_set(mm_ctx* ctx, int k, double tol);
MM_API mm_status mm_surrogate_get_stats(mm_ctx* ctx, mm_surrogate_stats* st);

/* Network parameters as n doubles in layer order (w0 [32][3][5][5], b0,
 * w1 [32][32][5][5], b1, w2, b2, w3 [3][32][5][5], b3; 56099 values).  get
 * or set may be NULL; c_in (in/out, may be NULL) is the input scale; setting
 * weights also sets the output scale c_out to c_in. */
MM_API mm_status mm_surrogate_weights(mm_ctx* ctx, double* get, const double* set, size_t n, double* c_in);

/* Network on host data: x [B][3][H][W] -> y [B][3][H][W] (raw network output),
 * path 0 = tensor-core kernels, 1 = SIMT cross-check kernels. */
MM_API mm_status mm_surrogate_forward(mm_ctx* ctx, int B, int H, int W, const double* x, double* y, int path);

/* One forward + mean-squared-error loss against t + backward pass: loss and
 * the gradient of every parameter (n = 56099, same order as the weights).
 * path 0 = weight gradients on the tensor cores (per-CTA partial sums added
 * in a fixed order, so repeated calls agree bit for bit), 1 = SIMT
 * cross-check kernels (FP32 atomics).  Errors: MM_ERR_ARG (NULL x or t,
 * non-positive sizes, path not 0 or 1), MM_ERR_TIMEOUT (a bounded
 * tensor-core wait ran out; reported once, the context stays usable). */
MM_API mm_status mm_surrogate_grad(mm_ctx* ctx, int B, int H, int W, const double* x, const double* t,
                                   double* loss, double* grad, int path);

/* Per-kernel CUDA-event timing (graphs are bypassed while on).  No passage:
 * boundary convenience (tracing; the paper times whole runs, Methods,
 * "Benchmark protocol").  mm_get_profile: *n_inout in = capacity of out,
 * out = entries written. */
MM_API mm_status mm_set_profiling(mm_ctx* ctx, int on);
MM_API mm_status mm_get_profile(mm_ctx* ctx, mm_profile_entry* out, int* n_inout);

/* Measured arithmetic throughput of the current device: a grid of
 * independent fused multiply-add chains in FP32 (precision 32) or FP64
 * (64), timed with CUDA events on the default stream (about a millisecond);
 * *flops_per_s = 2 x FMAs / s.  No passage: measurement convenience (the
 * denominator of ALU-bound rooflines).  Allocates 2 KB for the duration of
 * the call.  Errors: MM_ERR_ARG (bad precision, NULL), MM_ERR_DEVICE,
 * MM_ERR_OOM, MM_ERR_CUDA. */
MM_API mm_status mm_measure_peak(int precision, double* flops_per_s);

/* Fault injection for tests: 1 = next allocation fails, 2 = poison the
 * state with NaN at the next step, 3 = force dt underflow, 4 = the next
 * evaluation of the surrogate network issues no tensor-core work and polls
 * its accumulator barrier only 1000 times, so the bounded wait runs out with
 * nothing asynchronous in flight (mm_surrogate_forward then returns
 * MM_ERR_TIMEOUT and the context stays usable).  No passage: test
 * convenience.  Errors: MM_ERR_ARG (NULL, fault outside 0..4). */
MM_API mm_status mm_debug_inject(mm_ctx* ctx, int fault);

/* Message of the last failure of ctx (or of the last context-less call
 * when ctx is NULL), and the name of a status code.  No passage: boundary
 * convenience.  The strings stay owned by the library. */
MM_API const char* mm_last_error(const mm_ctx* ctx);
MM_API const char* mm_status_string(mm_status s);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
