// Internal declarations of the GB300 dycore library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>
#include <vector>
#include "../../include/icon.h"

namespace icon {

// ---------------------------------------------------------------- constants
// Physical constants and method parameters (the paper fixes none of them).
constexpr double kR = 6.371229e6;        // sphere radius, m
constexpr double kOmega = 7.29212e-5;    // rotation rate, 1/s
constexpr double kGrav = 9.80665;        // m/s^2
constexpr double kRd = 287.04;           // J/kg/K
constexpr double kCpd = 1004.64;         // J/kg/K
constexpr double kCvd = kCpd - kRd;
constexpr double kP0 = 1.0e5;            // Pa
constexpr double kBeta = 0.65;           // vertical off-centring (implicit weight)
constexpr double kCsSmag = 0.15;         // Smagorinsky constant
constexpr double kDivDamp4 = 0.0025;     // default fourth-order divergence damping coefficient

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
#define ICON_CUDA(call)                                                        \
  do {                                                                         \
    cudaError_t _e = (call);                                                   \
    if (_e != cudaSuccess) return ::icon::cuda_fail(_e, #call);                \
  } while (0)

// ---------------------------------------------------------------- kernel kinds and profiling
enum KernelKind {
  K_VERTEX = 0, K_EDGE_VT, K_CELL_KE, K_EDGE_TEND, K_COLUMN,
  K_DIFF_VERTEX, K_DIFF_DIV, K_DIFF_EDGE, K_DIFF_THETA, K_MASS,
  K_MX_VERTEX, K_MX_EDGE, K_MX_CELL_KE, K_MX_EDGE_TEND, K_MX_COLUMN, K_MX_COLUMN_PREP,
  K_MX_DIFF_VERTEX, K_MX_DIFF_EDGE, K_MX_DIFF_THETA, K_ENSEMBLE, K_TRACER, K_DIVDAMP, K_DIFF4, K_TERRAIN,
  K_MX_LEAN, K_MX_LEAN_GATHER, K_KIND_COUNT
};
static_assert(K_KIND_COUNT <= ICON_KIND_COUNT, "kind table");
// When a profile is active on this thread, every launch is bracketed by events.
void prof_begin(cudaStream_t st, int kind);
void prof_end(cudaStream_t st);

// tile over (entity, level) of a stencil kernel: lanes per entity (32 or 16) and block size
struct TileChoice {
  int lanes;
  int block;
};

// ---------------------------------------------------------------- memory
struct Allocator {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*dealloc)(void*, void*) = nullptr;
  void* ctx = nullptr;
};
Allocator current_allocator();
cudaStream_t current_stream();

// A set of device buffers released together with the allocator that made them.
struct DeviceArena {
  Allocator al;
  std::vector<void*> blocks;
  bool failed = false;
  void* get(size_t bytes);           // NULL (and failed = true) on failure
  template <class T> T* get_n(size_t n) { return static_cast<T*>(get(n * sizeof(T))); }
  void release();
};

// ---------------------------------------------------------------- grid
struct Vertical {
  int N = 0;           // full levels
  int ld = 0;          // row stride (elements) of every (entity, level) field
  double z_top = 0, s = 0, z_d = 0;
  std::vector<double> z_h, z_f, dz, dzh, wu, wl, rayleigh, dz2;  // host copies
  std::vector<float> h_f32;                                       // host staging of the FP32 tables
  // device copies (length ld)
  double *d_z_h = nullptr, *d_z_f = nullptr, *d_dz = nullptr, *d_dzh = nullptr,
         *d_wu = nullptr, *d_wl = nullptr, *d_ray = nullptr, *d_dz2 = nullptr;
  float *d_inv_dz32 = nullptr, *d_wu32 = nullptr, *d_wl32 = nullptr, *d_inv_dz2_32 = nullptr;
  double *d_inv_dz = nullptr, *d_inv_dz2 = nullptr, *d_qinv_dz = nullptr;   // 1/dz, 1/dz2, 1/(4 dz)
};

struct GridDev {
  int64_t nc = 0, ne = 0, nv = 0;
  int L = 0;
  // connectivity
  int *c2v = nullptr, *c2e = nullptr, *e2c = nullptr, *e2v = nullptr;
  int *v2e = nullptr, *v2c = nullptr, *vdeg = nullptr, *e2vt = nullptr, *e2q = nullptr;
  // geometry (FP64)
  double *x_c = nullptr, *x_e = nullptr, *x_v = nullptr, *n_e = nullptr, *t_e = nullptr;
  double *l_e = nullptr, *d_e = nullptr, *A_c = nullptr, *A_v = nullptr, *f_e = nullptr;
  double *vt_w = nullptr, *kin_w = nullptr, *lsq_w = nullptr, *L34 = nullptr;
  double *s_ce = nullptr, *s_ve = nullptr;
  // derived coefficient tables
  double *div_w = nullptr;   // [Nc][3]  s_ce * l_e  (divide by A_c afterwards)
  double *rot_w = nullptr;   // [Nv][6]  s_ve * d_e  (divide by A_v afterwards)
  float *vt_w32 = nullptr, *kin_w32 = nullptr, *lsq_w32 = nullptr;
  float *div_w32 = nullptr, *rot_w32 = nullptr;   // mixed precision copies (already / area)
  float *inv_de32 = nullptr, *inv_le32 = nullptr, *f_e32 = nullptr;
  float *l_e32 = nullptr, *n_e32 = nullptr, *t_e32 = nullptr, *L34inv32 = nullptr, *s_ce32 = nullptr;
  double* inv_Ac = nullptr;  // 1 / A_c
  double *div_wa = nullptr, *rot_wa = nullptr;             // s l / A_c, s d / A_v
  double *inv_de = nullptr, *inv_le = nullptr, *inv_L34 = nullptr;
  // tracer transport tables, built on demand (build_tracer_tables)
  int* c2c = nullptr;           // [Nc][3] neighbour across each edge slot
  double* lsq_c = nullptr;      // [Nc][3][3] least-squares gradient weights (3-vectors)
  double* roff = nullptr;       // [Ne][2][3] R (x_e - x_c1), R (x_e - x_c2)
  // per level [3][ld]: 1/(z_f[k-1] - z_f[k+1]) (0 at the top and bottom level),
  // z_h[h] - z_f[h] (donor below), z_h[h] - z_f[h-1] (donor above)
  double* tr_lev = nullptr;
};

}  // namespace icon

struct icon_grid {
  icon::DeviceArena arena;
  icon::GridDev g;
  icon::Vertical vert;
  int root = 2, bisections = 0;
  int device = -1;        // CUDA device the grid's tables live on (current at build time)
};

namespace icon {
// Device buffers of one state. Full-level fields are [n][ld], half-level fields
// [n][ld] with N+1 used entries. "star" holds the predictor state.
// terrain-following levels over topography (FP64 form): z = zeta_h + hs b_h per column
struct TopoDev {
  bool on = false;
  double h0 = 0.0, radius = 0.0;      // Gaussian mountain height and e-folding radius, m
  double* hs = nullptr;               // [Nc] surface height
  double *b = nullptr, *bf = nullptr; // [ld] decay at half and full levels
  double *sn = nullptr, *st = nullptr;   // [Ne] (hs_c2 - hs_c1)/d_e, (hs_v2 - hs_v1)/l_e
  // per cell and level [Nc][ld]: 1/dz, 1/dzh (interior half levels), upper interpolation
  // weight (interior half levels), reference Exner at the full level, dz
  double *inv_dz_c = nullptr, *inv_dzh_c = nullptr, *wu_c = nullptr, *exref_c = nullptr, *dz_c = nullptr;
  // per edge and level [Ne][ld]: upper interpolation weight, 1/(4 dz), dz
  double *wu_e = nullptr, *qinv_dz_e = nullptr, *dz_e = nullptr;
  // per stage [Nc][ld]: contravariant correction wcc and velocity w - wcc (0 at lid and
  // ground) at half levels; Exner perturbation pi - pi_ref and half its vertical
  // derivative at full levels
  double *wcc = nullptr, *wcon = nullptr, *ep = nullptr, *hdpdz = nullptr;
  // mixed-precision states: FP32 copies for the FP32 stencils ([entity][ld]; per edge;
  // per level) and the stage's FP32 contravariant terms (the Exner perturbation is the
  // state's own FP32 shadow, taken against this per-cell reference)
  float *wu_e32 = nullptr, *inv_dz_e32 = nullptr, *dz_e32 = nullptr, *csn32 = nullptr, *bf32 = nullptr;
  float *wu_c32 = nullptr, *inv_dz_c32 = nullptr, *inv_dzh_c32 = nullptr;
  float *wcc32 = nullptr, *wcon32 = nullptr, *hdpdz32 = nullptr;
  // and level-major copies ([k][Nc], N+1 rows) of the column's per-cell tables, which the
  // mixed column reads one column per thread
  double *wu_lm = nullptr, *idz_lm = nullptr, *idzh_lm = nullptr, *exref_lm = nullptr;
};

struct StateDev {
  int precision = ICON_FP64;
  TopoDev topo;
  // prognostics S^n (FP64 in both modes except vn in mixed mode)
  double *vn = nullptr, *w = nullptr, *rho = nullptr, *thv = nullptr, *ex = nullptr;
  float *vn32 = nullptr;
  // predictor state S*
  double *vn_s = nullptr, *w_s = nullptr, *rho_s = nullptr, *thv_s = nullptr, *ex_s = nullptr;
  float *vn32_s = nullptr;
  // tendencies kept from the predictor
  double *Avn0 = nullptr, *Aw0 = nullptr;
  float *Avn0_32 = nullptr, *Aw0_32 = nullptr;
  // step-mean mass fluxes
  double *mflx = nullptr, *wflx = nullptr;
  // scratch (FP64 mode)
  double *zeta = nullptr, *w_v = nullptr, *vt = nullptr, *Ke = nullptr, *Kc = nullptr;
  double *a_e = nullptr, *F = nullptr, *G = nullptr;
  // half the cell weights kappa_ce and s_ce l_e / A_c ([Nc][3]): the FP64 step stores
  // 2 K_e, 2 rho_e vn and 4 rho_e vn theta_e at edges and folds the factors in here
  double *kin_w_h = nullptr, *div_wa_h = nullptr;
  double *uvx = nullptr, *uvy = nullptr, *uvz = nullptr, *divc = nullptr, *Kh = nullptr, *thflx = nullptr;
  // mixed-mode scratch and shadows
  float *zeta32 = nullptr, *wv32 = nullptr, *vt32 = nullptr, *Ke32 = nullptr, *Kc32 = nullptr,
        *ae32 = nullptr, *F32 = nullptr, *G32 = nullptr;
  float *rho32 = nullptr, *thv32 = nullptr, *exp32 = nullptr, *w32 = nullptr;
  float *rho32_s = nullptr, *thv32_s = nullptr, *exp32_s = nullptr, *w32_s = nullptr;
  float *uvx32 = nullptr, *uvy32 = nullptr, *uvz32 = nullptr;
  // mixed mode stores rho, theta_v, Exner, w and wflx level-major ([k][Nc])
  bool level_major = false;
  double *ex_ref = nullptr;           // [ld] reference Exner profile
  // per-level constants of the column solve for the current dtau (mixed mode)
  // FP64 column scratch: tridiagonal rows level-major [h][Nc], update operands [c][ld]
  double *col_lo = nullptr, *col_di = nullptr, *col_up = nullptr, *col_rh = nullptr;
  double *col_rx = nullptr, *col_tx = nullptr, *col_px = nullptr, *col_gm = nullptr;
  double *col_ri = nullptr, *col_mm = nullptr, *col_ws = nullptr, *col_gc = nullptr;
  double* colconst = nullptr;
  // tracers (mixing ratios, FP64 [t][Nc][ld]) and their transport scratch
  int ntr = 0;
  double* q = nullptr;
  double *tr_rho0 = nullptr, *tr_rho1 = nullptr, *tr_W = nullptr;   // [Nc][ld] (rho1, W: mixed only)
  double *tr_gx = nullptr, *tr_gy = nullptr, *tr_gz = nullptr, *tr_V = nullptr, *tr_F = nullptr;
  // frozen parts of the column system shared by predictor and corrector (mixed mode;
  // NULL when they would not fit, then both stages compute them)
  double* fac64 = nullptr;
  double *hdr = nullptr, *hdt = nullptr, *hdw = nullptr, *hdg = nullptr;  // gathered column inputs, level-major
  double* dps = nullptr;      // Thomas scratch, level-major
  float* exref32 = nullptr;   // FP32 copy of the reference Exner profile
  // lean column (mixed precision on flat levels, the default form): gathered stage inputs
  // (dtau D_rho FP64 [k][Nc], its FP32 predictor copy in the same buffer, dtau D_Theta and
  // dtau A_w FP32), the right-hand-side base, elimination values and LU factors [h][Nc],
  // per-level constants and dtau s l / A_c per cell
  double* ln_dr64 = nullptr;
  float *ln_dt32 = nullptr, *ln_aw32 = nullptr, *ln_cp = nullptr, *ln_cf = nullptr;
  double *ln_B = nullptr, *ln_dp = nullptr, *ln_cd = nullptr, *ln_dwa = nullptr;
  float* ln_cw32 = nullptr;   // per cell: FP32 dtau s l / A_c of its three edges, then dtau / A_c
  int ln_hdamp = 0;           // half levels h < ln_hdamp lie in the Rayleigh layer
  // mass reduction partials and the device status word
  double *mass_part = nullptr;
  int mass_nblk = 0;
  unsigned int* status = nullptr;
};
}  // namespace icon

struct icon_state {
  const icon_grid* grid = nullptr;
  icon::DeviceArena arena;
  icon::StateDev s;
  uint64_t seed = 0;
  int case_id = 0;
  // recorded step graph
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  int graph_nsub = 0;
  int graph_kernels = 0;
  cudaStream_t capture_stream = nullptr;
  cudaStream_t graph_stream = nullptr;
  cudaEvent_t done = nullptr;
  // second branch of the recorded mixed step on flat levels of R2B6 and finer grids (the next
  // stage's edge diagnostics beside the column); not created when ICON_STEP_OVERLAP=0
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // stencil tiles (mixed mode): chosen by the autotuner unless forced
  icon::TileChoice tile[ICON_KIND_COUNT] = {};
  bool tile_forced[ICON_KIND_COUNT] = {};
  bool tuned = false;
  // options (icon_state_set_option)
  double divdamp4 = 0.0;        // fourth-order divergence damping coefficient (0: off; set at init)
  double abar = 0.0;            // mean cell area of the (global) grid, m^2: the damping's length scale
  double diff4 = 0.0;           // fourth-order background diffusion coefficient (0: off)
  bool upwind_theta = false;    // heat fluxes with the upwind theta_v
};

namespace icon {
// device side of an ensemble (dycore32.cu)
struct EnsembleDev {
  DeviceArena arena;
  void* members = nullptr;     // MemberDev[64]
  unsigned* bar = nullptr;     // [0] arrivals, [1] generation, [8] status
  int nm = 0, nsub = 0, N = 0, grid_blocks = 0;
  int64_t tot_v = 0, tot_e = 0, tot_c = 0, tot_t = 0;
  bool all_fac = true;         // every member stores its column factors
  bool all_lean = false;       // every member runs the lean column
  bool any_damp = false;       // some member damps the corrector's divergence
  // per-member launches of the lean column's per-level constants and scaled weights
  struct LeanConst {
    int N, ld;
    int64_t nc;
    const double *wu, *wl, *dzh, *dz, *ray, *ex_ref;
    double dtau;
    double* cd;
    float* cf;
    const double *div_wa, *inv_Ac;
    double* dwa;
    float* cw32;
  };
  std::vector<LeanConst> lean_consts;
  long long spin_limit = 1ll << 24;
  int test_skip_barrier = 0;
};
int ensemble_prepare(EnsembleDev& E, icon_state* const* members, int n, const double* dts, int nsub);
int ensemble_launch(EnsembleDev& E, cudaStream_t st, unsigned long long* prof = nullptr, int prof_max = 0);
void autotune_mixed(icon_state* st, double dt, int nsub, cudaStream_t stream);
// a launch shape (sweep unroll, resident blocks per SM) the lean mixed column is built with
bool lean_column_shape_ok(int unroll, int blocks_per_sm);
// the stored-factor column parts of a mixed state (api.cu); false if they do not fit
bool alloc_mixed_factors(icon_state* st);
int selftest_conversions(int64_t n, unsigned* host_fails);
}  // namespace icon

namespace icon {
// grid_build.cu
int build_grid_device(icon_grid* grid, cudaStream_t st);
int build_tracer_tables(icon_grid* grid, cudaStream_t st);
// terrain.cu
constexpr double kTopoDecay = 4000.0;   // SLEVE decay scale, m
constexpr double kTopoTref = 250.0;     // temperature of the reference Exner profile, K
int topo_build(icon_state* st, double h0, double radius, cudaStream_t stream);
void topo_stage(icon_state* st, const double* vn, const double* vt, const double* w, const double* ex,
                cudaStream_t stream);
// mixed-precision states: the same stage terms in FP32 from the FP32 stage shadows
// (exp = Exner - the per-cell reference)
void topo_stage32(icon_state* st, const float* vn, const float* vt, const float* w, const float* exp,
                  cudaStream_t stream);
// tracer.cu
int tracer_alloc(icon_state* st, int ntracers);
void tracer_begin(icon_state* st, cudaStream_t stream);
void tracer_end(icon_state* st, double dt, cudaStream_t stream);
// init.cu
void make_vertical(Vertical& v, int nlev, double top_m, double stretch_s, double damp_m);
int init_state_device(icon_state* st, uint64_t seed, int case_id, const icon_case_params& p,
                      cudaStream_t stream);
// dycore64.cu
void enqueue_step_fp64(icon_state* st, double dt, int nsub, cudaStream_t stream);
void fp64_step_begin(icon_state* st, double dt, int nsub, cudaStream_t stream);
void fp64_step_stage(icon_state* st, double dt, int nsub, bool corr, cudaStream_t stream);
void fp64_step_diffusion(icon_state* st, double dt, cudaStream_t stream);
// dycore32.cu
void enqueue_step_mixed(icon_state* st, double dt, int nsub, cudaStream_t stream);
// mixed-mode state from FP64 fields in [entity][ld] layout (init.cu)
void mixed_cells_from_fp64(icon_state* st, int64_t c0, int64_t n, const double* w, const double* rho,
                           const double* thv, const double* ex, cudaStream_t stream);
void mixed_refresh_shadows(icon_state* st, cudaStream_t stream);
// mass
void enqueue_mass(const icon_state* st, double* d_out, cudaStream_t stream);
int mass_partials_count(int64_t nc);
// scan helper (grid_build.cu)
int exclusive_scan_u32(const unsigned* in, unsigned* out, int64_t n, unsigned* total_dev,
                       DeviceArena& tmp, cudaStream_t st);

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }
}  // namespace icon
