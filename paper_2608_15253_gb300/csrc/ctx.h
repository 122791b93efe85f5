// Host-side internals of libmm: the context, its device buffers, the
// per-region material table, launch bookkeeping and the kernel launchers
// each translation unit provides.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <array>
#include <vector>

#include "mm.h"

namespace mm {

constexpr int kMaxRegions = 256;

// Per-region coefficients consumed by the field kernels (working precision).
template <typename T>
struct Region {
    T present;    // 1 if Ms > 0
    T inv_mu0Ms;  // 1/(mu0 Ms), 0 when absent
    T Ms;
    T cg;         // ghost exchange coefficient 2 A_i / (mu0 Ms_i)
    T ratio;      // D / (2 A), 0 when A = 0
    T dmi;        // 2 D / (mu0 Ms)
    T ku;         // 2 Ku1 / (mu0 Ms)
    T ux, uy, uz;
    T alpha;
    T gm;         // gamma0 mu0 / (1 + alpha^2)
    T sigma0;     // sqrt(2 alpha kB / (mu0^2 Ms gamma0)); times sqrt(T/(V dt)) -> A/m
    T inv_Ms;     // 1/Ms, 0 when absent
    T ratio_b;    // bulk DMI: Db / (2 A), 0 when A = 0
    T dmib;       // bulk DMI: 2 Db / (mu0 Ms)
    T kc1, kc2;   // cubic: 2 Kc1 / (mu0 Ms), 2 Kc2 / (mu0 Ms)
    T c1x, c1y, c1z, c2x, c2y, c2z, c3x, c3y, c3z;   // orthonormal cubic axes
    T ks;         // surface: 2 Ks / (mu0 Ms) (divided by dz in the kernel)
    T b1, b2;     // magnetoelastic: 2 B1 / (mu0 Ms), 2 B2 / (mu0 Ms)
};

struct RegionHost {
    double Ms, A, alpha, Ku1, u[3], D, Db;
    double Kc1, Kc2, c1[3], c2[3], Ks, B1, B2;   // uniform over the material
    bool operator==(const RegionHost& o) const {
        return Ms == o.Ms && A == o.A && alpha == o.alpha && Ku1 == o.Ku1 && u[0] == o.u[0] &&
               u[1] == o.u[1] && u[2] == o.u[2] && D == o.D && Db == o.Db;
    }
};

// Device state of the integrator (one per context, read by every kernel of
// an attempt so that whole steps can be replayed from a CUDA graph).
struct DevState {
    double t, dt, dt_eff, t_end;
    double rtol, dt_min, dt_max;
    double err;                 // max-norm error of the last attempt (as a double)
    float err_f;                // float32 accumulation target
    int active;                 // 0: remaining kernels of this attempt are no-ops
    int accept;
    int last_rejected;
    int replay;                 // 1: take dt from replay_dts, always accept
    int status;                 // mm_status raised on the device (sticky)
    int k_first;                // slot index holding k1 (FSAL rotation: 0 or 6)
    int fsal;                   // 1: RK45 (k7 becomes k1 on accept)
    double ctrl_exp;            // step-size exponent: 1/5 (RK45), 1/2 (adaptive Depondt-Mertens)
    long long accepted, rejected, attempts, step;
    long long target;           // stop after this many accepted steps
    long long replay_n;
    const double* replay_dts;
    // dt-scaled tableau of the current attempt in working precision, set once
    // per attempt so that the per-element kernels do no FP64 arithmetic
    float cf32[7][7];           // dt * a_sj
    float ce32[7];              // dt * (b5_j - b4_j)
    double cf64[7][7];
    double ce64[7];
};

struct DemagPlan {
    int on = 0;
    int Px = 0, Py = 0, Pz = 0;   // padded lengths
    int Lh = 0;                   // Px / 2 (complex length of the X transform)
    int Kx = 0, Wk = 0;           // Px/2 + 1 spectrum columns, row pitch
    int PyA = 0;                  // rows per z-plane of the spectrum buffer
    int ncomp = 0;                // 6 (3D) or 4 (nz = 1)
    void* spec = nullptr;         // [3][nz][PyA][Wk] complex
    void* khat = nullptr;         // [ncomp][Pz/2+1][Py/2+1][Wk] real
    void* tw_x = nullptr;         // exp(-2 pi i k / Px), k < Px
    void* tw_y = nullptr;         // exp(-2 pi i k / Py)
    void* tw_z = nullptr;         // exp(-2 pi i k / Pz)
};

struct BatchHost;
struct SurrogateHost;

struct ProfileSlot {
    std::string name;
    long long launches = 0;
    double total_ms = 0.0;
    double bytes = 0.0;
};

}  // namespace mm

struct mm_ctx {
    int prec = 32;              // 32 or 64
    size_t esz = 4;             // bytes per real
    int integrator = MM_RK45;
    unsigned terms = MM_TERM_ALL;
    int R = 1;
    mm_grid grid{};
    long long N = 0;            // cells per replica (single instance)
    mm_config cfg{};
    std::string last_error;

    // material regions
    int nreg = 1;
    int uniform = 1;            // every cell in region 0
    std::vector<mm::RegionHost> regions;
    std::vector<uint8_t> region_of_cell;
    void* d_region = nullptr;   // uint8 per cell (null when uniform)
    void* d_lut = nullptr;      // Region<T>[nreg]
    void* d_cpair = nullptr;    // T[nreg*nreg]: 2 A_ij / (mu0 Ms_i)
    mm::Region<float> r0f{};    // host copies of region 0 (the one material when uniform)
    mm::Region<double> r0d{};
    float c00f = 0.f;           // cpair[0]
    double c00d = 0.0;

    // state buffers (working precision), [3][N] each
    void* d_m = nullptr;        // current state m0
    void* d_mtmp = nullptr;     // stage state
    void* d_k[7] = {};          // stage slopes
    void* d_kslot = nullptr;    // device array of 7 pointers (FSAL rotation)
    void* d_hd = nullptr;       // demag field
    void* d_hbuf = nullptr;     // scratch field (observables)
    void* d_stage = nullptr;    // host-transfer staging, stage_n doubles
    long long stage_n = 0;
    void* d_bcell = nullptr;    // per-cell applied field (A/m) or null
    double Hext[3] = {0, 0, 0}; // uniform applied field (A/m)
    unsigned terms_req = MM_TERM_ALL;   // requested terms; `terms` drops those without parameters
    bool cubic_energy = false;          // field evaluation weighted for the cubic energy
    bool ext_terms = true;              // bulk DMI or a further local term is on: the full field kernels
    double strain[6] = {0, 0, 0, 0, 0, 0};   // uniform strain (magnetoelastic)
    void* d_strain = nullptr;   // per-cell strain [6][N] or null
    bool strain_set = false;
    int rkky_k1 = 0, rkky_k2 = 0;
    double rkky_J = 0.0;        // J/m^2; 0: off
    double Tr = 0.0;            // temperature
    uint64_t seed = 0;          // Philox key of the replica

    // torque
    mm_torque tq{};
    double J = 0.0;

    mm::DevState* d_state = nullptr;
    mm::DevState h_state{};
    double* d_replay = nullptr;
    size_t replay_cap = 0;
    double* d_red = nullptr;    // reduction partials
    int* d_flag = nullptr;      // one device int (mm_set_m: did the state change)
    size_t red_cap = 0;

    mm::DemagPlan dm;

    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    bool k1_valid = false;

    // CUDA graph of a chunk of integrator attempts
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    cudaGraphExec_t graph1 = nullptr;   // one attempt (the remainder of a request)
    long long launches_per_attempt = 0;
    long long launches_per_chunk = 0;

    // replica batching (R > 1): per-replica grids, offsets, keys, T and J
    mm::BatchHost* batch = nullptr;
    std::vector<mm_grid> rgrid;
    std::vector<long long> roff;       // element offset of replica r's [3][ny][nx] block
    std::vector<uint64_t> rkey;
    std::vector<double> rT, rJ;
    long long Ntot = 0;                // cells over all replicas (storage, gaps between size classes included)
    std::vector<std::array<long long, 3>> sblocks;   // per size class: storage offset, packed offset, length

    mm::SurrogateHost* surr = nullptr;  // learned demag surrogate (single instance)

    long long launches = 0;
    bool profiling = false;
    std::vector<mm::ProfileSlot> prof;
    int inject = 0;
};

namespace mm {

mm_status set_error(mm_ctx* c, mm_status s, const std::string& msg);
mm_status cuda_check(mm_ctx* c, cudaError_t e, const char* what);

// Kernel-launch bookkeeping: counts launches and, while profiling, brackets
// the launch with CUDA events on the context stream.
struct LaunchScope {
    mm_ctx* c;
    int slot;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LaunchScope(mm_ctx* c, const char* name, double bytes);
    ~LaunchScope();
};

// demag.cu
mm_status demag_setup(mm_ctx* c);
void demag_free(mm_ctx* c);
void demag_apply(mm_ctx* c, const void* m, void* Hd);   // Hd = H_demag(m)
// FP32 RK45 stage s fused into the X pass: forms m_s = m0 + sum (dt a_sj) k_j
// into d_mtmp while transforming it, then Hd = H_demag(m_s)
bool demag_stage_fusable(const mm_ctx* c);
void demag_apply_stage(mm_ctx* c, int stage, void* Hd);
// FP32: every demag pass but the inverse X pass, for the fused inverse-X +
// field kernel (stage > 0: the RK45 stage state is formed into d_mtmp first)
void demag_apply_partial(mm_ctx* c, const void* m, int stage);
mm_status newell_gpu(long count, const int* ijk, double dx, double dy, double dz, double* out_host);

// conv_split.cu: middle pass for lines split over several threads (FP32)
bool split_conv_supported(int L);
cudaError_t split_conv_setup();
void split_conv_launch_3d(mm_ctx* c, void* spec, const void* khat, int nz, int Py, int Pz, int Kx, int Wk,
                          double bytes);
void split_conv_launch_2d(mm_ctx* c, void* spec, const void* khat, int ny, int Py, int Kx, int Wk,
                          long long comp_stride, long long plane_stride, int n_planes, const char* name,
                          double bytes);
bool ysplit_supported(int L);
void ysplit_launch(mm_ctx* c, bool fwd, void* spec, int nz, int Py, int Kx, int Wk, int n_in, int n_out,
                   const char* name, double bytes);

// field.cu
// MODE_DM1 / MODE_DM2: Depondt-Mertens predictor (out <- rotated m, out2 <-
// Omega) and corrector (out <- m0 rotated by the mean Omega, k1 = Omega_1)
enum FieldMode { MODE_H = 0, MODE_K = 1, MODE_HEUN1 = 2, MODE_HEUN2 = 3, MODE_DM1 = 4, MODE_DM2 = 5 };
void field_launch(mm_ctx* c, int mode, unsigned terms, const void* m, const void* Hd,
                  void* out, void* out2, const void* m0, const void* k1, long long step_override,
                  int gate, int kstage);
void thermal_raw_launch(mm_ctx* c, long long step, uint32_t* d_raw, void* d_h);
// inverse X pass + field kernel in one launch (the demag spectrum of the
// state must be ready); field_c2r_fusable says whether the grid allows it
bool field_c2r_fusable(const mm_ctx* c);
cudaError_t field_c2r_setup();
void field_c2r_launch(mm_ctx* c, int mode, unsigned terms, const void* m, void* out, void* out2, const void* m0,
                      const void* k1, long long step_override, int gate, int kstage);

// batch.cu
BatchHost* batch_new();
void batch_free(BatchHost* b);
mm_status batch_setup(mm_ctx* c, BatchHost* b, const std::vector<mm_grid>& grids, const std::vector<uint64_t>& keys,
                      bool demag);
mm_status batch_upload(mm_ctx* c, BatchHost* b, const std::vector<double>& T, const std::vector<double>& J);
void batch_step(mm_ctx* c, BatchHost* b);
bool batch_is_fused(BatchHost* b);
void batch_macro_steps(mm_ctx* c, BatchHost* b, int nsteps);
mm_status batch_trials_start(mm_ctx* c, BatchHost* b, const mm_trials* sp, long long step_now);
mm_status batch_trials_result(mm_ctx* c, BatchHost* b, long long* steps, int* stopped, long long* done);
bool batch_trials_on(BatchHost* b);
void batch_set_shape(BatchHost* b, int nt, int blocks);
int batch_max_blocks(BatchHost* b);
size_t batch_smem_for(BatchHost* b, int nt);
mm_status demag_setup_for(mm_ctx* c, const mm_grid& g, DemagPlan* out);
void demag_apply_stacked2d(mm_ctx* c, const DemagPlan& p, const float* m, float* Hd, void* S, int nx, int ny, int Rc);
void demag_free_plan(DemagPlan& d);
const DemagPlan& batch_plan(BatchHost* b, int r_cls);
int batch_occupancy(BatchHost* b, int nt);
void batch_get_shape(BatchHost* b, int* nt, int* blocks);
std::string batch_signature(BatchHost* b, unsigned terms);
int batch_class_of(BatchHost* b, int r);

// surrogate.cu
void surrogate_free(mm_ctx* c);
bool surrogate_active(mm_ctx* c);           // this evaluation uses the network
bool surrogate_fallen_back(mm_ctx* c);      // the monitor switched to exact evaluations
void surrogate_count_exact(mm_ctx* c, long long attempts);   // exact attempts after a fallback
void surrogate_invalidate_graph(mm_ctx* c); // drop the captured network attempt
mm_status attempt_graph_launch(mm_ctx* c, cudaGraphExec_t* g, long long* launches);
bool surrogate_stepping(mm_ctx* c);         // surrogate-accelerated stepping is on
void surrogate_apply(mm_ctx* c, const void* m, void* Hd);
mm_status surrogate_block(mm_ctx* c);       // one exact refresh + k-1 network attempts

// integrate.cu
void demag_eval(mm_ctx* c, const void* m, void* Hd);   // exact or surrogate
void heun_batch_begin(mm_ctx* c);
void heun_batch_advance(mm_ctx* c);
void rk45_first_slope(mm_ctx* c);          // k1 = f(m0) into the FSAL slot
void rk45_attempt(mm_ctx* c);               // one attempted DOPRI5 step
void heun_step(mm_ctx* c);
void dm_step(mm_ctx* c);
void dm_adaptive_attempt(mm_ctx* c);                  // one Heun step
void rk4_step(mm_ctx* c);                   // one classical RK4 step

// reduce.cu
void energy_term_launch(mm_ctx* c, const void* m, const void* H, int which, double* d_out2);
void topo_launch(mm_ctx* c, const void* m, int layer, double* d_out2);
void normalize_launch(mm_ctx* c, void* m);

}  // namespace mm
