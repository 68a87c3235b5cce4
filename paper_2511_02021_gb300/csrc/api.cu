// C ABI of the dycore library: argument checks, handle lifetimes, device memory
// through the registered allocator, the recorded step graph and host copies.
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include "icon_internal.h"

namespace icon {

static thread_local std::string t_err;
static thread_local cudaStream_t t_stream = nullptr;
static std::mutex g_alloc_mu;
static Allocator g_alloc;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return ICON_ECUDA;
}

// ---------------------------------------------------------------- profiling
struct Prof {
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  int open = -1;
  bool failed = false;
};
static thread_local Prof* t_prof = nullptr;

void prof_begin(cudaStream_t st, int kind) {
  Prof* p = t_prof;
  if (!p || p->failed) return;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) { p->failed = true; return; }
  p->ev.push_back(a);
  p->ev.push_back(b);
  p->kind.push_back(kind);
  p->open = (int)p->kind.size() - 1;
  cudaEventRecord(a, st);
}

void prof_end(cudaStream_t st) {
  Prof* p = t_prof;
  if (!p || p->failed || p->open < 0) return;
  cudaEventRecord(p->ev[2 * p->open + 1], st);
  p->open = -1;
}

static const char* kKindNames[K_KIND_COUNT] = {
    "vertex_curl_wmean", "edge_vt_ke", "cell_ke", "edge_tendency_flux", "column_solve",
    "diff_vertex", "diff_div", "diff_edge", "diff_theta", "global_mass",
    "mx_vertex", "mx_edge_diag", "mx_cell_ke", "mx_edge_tendency_flux", "mx_column_solve", "mx_column_prep",
    "mx_diff_vertex", "mx_diff_edge", "mx_diff_theta", "ensemble_persistent", "tracer_transport", "divergence_damping", "background_diffusion",
    "terrain_metrics", "mx_lean_column", "mx_lean_gather"};

Allocator current_allocator() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc;
}
cudaStream_t current_stream() { return t_stream; }

void* DeviceArena::get(size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (al.alloc) {
    p = al.alloc(bytes, al.ctx);
    if (p) {
      // never use a pointer that is not device memory (a failing allocator callback
      // must not make kernels write through garbage)
      cudaPointerAttributes attr;
      if (cudaPointerGetAttributes(&attr, p) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        p = nullptr;
      }
    }
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) {
    failed = true;
    return nullptr;
  }
  blocks.push_back(p);
  return p;
}

void DeviceArena::release() {
  for (void* p : blocks) {
    if (al.dealloc) al.dealloc(p, al.ctx);
    else cudaFree(p);
  }
  blocks.clear();
}

namespace {

int upload_vertical(icon_grid* grid, cudaStream_t st) {
  Vertical& v = grid->vert;
  DeviceArena& A = grid->arena;
  double** dst[] = {&v.d_z_h, &v.d_z_f, &v.d_dz, &v.d_dzh, &v.d_wu, &v.d_wl, &v.d_ray, &v.d_dz2};
  const std::vector<double>* src[] = {&v.z_h, &v.z_f, &v.dz, &v.dzh, &v.wu, &v.wl, &v.rayleigh, &v.dz2};
  for (int i = 0; i < 8; ++i) {
    *dst[i] = A.get_n<double>(v.ld);
    if (!*dst[i]) { set_error("out of device memory (vertical grid)"); return ICON_ENOMEM; }
    ICON_CUDA(cudaMemcpyAsync(*dst[i], src[i]->data(), sizeof(double) * v.ld, cudaMemcpyHostToDevice, st));
  }
  // FP32 copies for the mixed-precision stencils (kept in the grid, copied synchronously below)
  v.h_f32.assign(4 * (size_t)v.ld, 0.0f);
  for (int k = 0; k < v.N; ++k) v.h_f32[k] = (float)(1.0 / v.dz[k]);
  for (int h = 0; h <= v.N; ++h) {
    v.h_f32[v.ld + h] = (float)v.wu[h];
    v.h_f32[2 * v.ld + h] = (float)v.wl[h];
    v.h_f32[3 * v.ld + h] = (h > 0 && h < v.N) ? (float)(1.0 / v.dz2[h]) : 0.0f;
  }
  // FP64 reciprocals of the layer thicknesses (full levels, the two-layer span, and a
  // quarter of the full-level one, exactly scaled)
  std::vector<double> inv(3 * (size_t)v.ld, 0.0);
  for (int k = 0; k < v.N; ++k) inv[k] = 1.0 / v.dz[k];
  for (int h = 1; h < v.N; ++h) inv[v.ld + h] = 1.0 / v.dz2[h];
  for (int k = 0; k < v.N; ++k) inv[2 * v.ld + k] = 0.25 * inv[k];
  double* di = A.get_n<double>(3 * (size_t)v.ld);
  if (!di) { set_error("out of device memory (vertical grid)"); return ICON_ENOMEM; }
  ICON_CUDA(cudaMemcpy(di, inv.data(), sizeof(double) * 3 * v.ld, cudaMemcpyHostToDevice));
  v.d_inv_dz = di;
  v.d_inv_dz2 = di + v.ld;
  v.d_qinv_dz = di + 2 * v.ld;
  float* f = A.get_n<float>(4 * (size_t)v.ld);
  if (!f) { set_error("out of device memory (vertical grid)"); return ICON_ENOMEM; }
  ICON_CUDA(cudaMemcpyAsync(f, v.h_f32.data(), sizeof(float) * 4 * v.ld, cudaMemcpyHostToDevice, st));
  v.d_inv_dz32 = f;
  v.d_wu32 = f + v.ld;
  v.d_wl32 = f + 2 * v.ld;
  v.d_inv_dz2_32 = f + 3 * v.ld;
  return ICON_OK;
}

struct TableRef {
  const void* ptr;
  size_t elem;
  size_t count;
};

bool table_ref(const icon_grid* grid, int id, TableRef& t) {
  const GridDev& g = grid->g;
  const size_t nc = g.nc, ne = g.ne, nv = g.nv;
  switch (id) {
    case ICON_T_C2V: t = {g.c2v, 4, 3 * nc}; return true;
    case ICON_T_C2E: t = {g.c2e, 4, 3 * nc}; return true;
    case ICON_T_E2C: t = {g.e2c, 4, 2 * ne}; return true;
    case ICON_T_E2V: t = {g.e2v, 4, 2 * ne}; return true;
    case ICON_T_V2E: t = {g.v2e, 4, 6 * nv}; return true;
    case ICON_T_V2C: t = {g.v2c, 4, 6 * nv}; return true;
    case ICON_T_VDEG: t = {g.vdeg, 4, nv}; return true;
    case ICON_T_E2VT: t = {g.e2vt, 4, 5 * ne}; return true;
    case ICON_T_E2Q: t = {g.e2q, 4, 4 * ne}; return true;
    case ICON_G_XC: t = {g.x_c, 8, 3 * nc}; return true;
    case ICON_G_XE: t = {g.x_e, 8, 3 * ne}; return true;
    case ICON_G_XV: t = {g.x_v, 8, 3 * nv}; return true;
    case ICON_G_NE: t = {g.n_e, 8, 3 * ne}; return true;
    case ICON_G_TE: t = {g.t_e, 8, 3 * ne}; return true;
    case ICON_G_LE: t = {g.l_e, 8, ne}; return true;
    case ICON_G_DE: t = {g.d_e, 8, ne}; return true;
    case ICON_G_AC: t = {g.A_c, 8, nc}; return true;
    case ICON_G_AV: t = {g.A_v, 8, nv}; return true;
    case ICON_G_FE: t = {g.f_e, 8, ne}; return true;
    case ICON_G_VTW: t = {g.vt_w, 8, 5 * ne}; return true;
    case ICON_G_KINW: t = {g.kin_w, 8, 3 * nc}; return true;
    case ICON_G_LSQW: t = {g.lsq_w, 8, 18 * nv}; return true;
    case ICON_G_L34: t = {g.L34, 8, ne}; return true;
    case ICON_G_SCE: t = {g.s_ce, 8, 3 * nc}; return true;
    case ICON_G_SVE: t = {g.s_ve, 8, 6 * nv}; return true;
    case ICON_T_C2C: t = {g.c2c, 4, 3 * nc}; return g.c2c != nullptr;
    case ICON_G_LSQC: t = {g.lsq_c, 8, 9 * nc}; return g.lsq_c != nullptr;
    case ICON_G_ROFF: t = {g.roff, 8, 6 * ne}; return g.roff != nullptr;
    default: return false;
  }
}

}  // namespace

// the frozen parts of the column system that the stored-factor form keeps between the
// predictor and the corrector (12 FP64 fields per half level) and its gathered inputs;
// allocated when they take at most a quarter of the device memory (else the column
// recomputes them). Returns true if the state has them afterwards.
bool alloc_mixed_factors(icon_state* st) {
  StateDev& s = st->s;
  if (s.fac64) return true;
  const int64_t nc = st->grid->g.nc;
  const size_t ld0 = (size_t)st->grid->vert.N;
  const size_t fac_bytes = (size_t)nc * (12 + 5) * (ld0 + 1) * 8;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (fac_bytes > total_b / 4) return false;
  DeviceArena& A = st->arena;
  double* p[6];
  const size_t H = (size_t)nc * (ld0 + 1);
  p[0] = A.get_n<double>(H * 12);
  for (int i = 1; i < 6; ++i) p[i] = p[0] ? A.get_n<double>(H) : nullptr;
  if (A.failed) {
    A.failed = false;          // the state stays usable without them
    return false;
  }
  s.fac64 = p[0];
  s.hdr = p[1];
  s.hdt = p[2];
  s.hdw = p[3];
  s.hdg = p[4];
  s.dps = p[5];
  return true;
}

namespace {

// allocate every buffer of a state; returns ICON_ENOMEM (arena then released by the caller)
int alloc_state(icon_state* st, int precision, bool topo) {
  const icon_grid* grid = st->grid;
  const int64_t ld = grid->vert.ld, nc = grid->g.nc, ne = grid->g.ne, nv = grid->g.nv;
  DeviceArena& A = st->arena;
  StateDev& s = st->s;
  s.precision = precision;
  const size_t E = (size_t)(ne * ld), C = (size_t)(nc * ld), V = (size_t)(nv * ld);
  const size_t ld0 = (size_t)grid->vert.N;
  s.mflx = A.get_n<double>(E);
  s.ex_ref = A.get_n<double>(ld);
  s.mass_part = A.get_n<double>(mass_partials_count(nc) + 8);
  s.status = A.get_n<unsigned>(64);
  if (precision == ICON_FP64) {
    s.w = A.get_n<double>(C); s.rho = A.get_n<double>(C); s.thv = A.get_n<double>(C); s.ex = A.get_n<double>(C);
    s.w_s = A.get_n<double>(C); s.rho_s = A.get_n<double>(C); s.thv_s = A.get_n<double>(C);
    s.ex_s = A.get_n<double>(C);
    s.wflx = A.get_n<double>(C);
    s.colconst = A.get_n<double>(8 * (size_t)ld);
    double** col[] = {&s.col_lo, &s.col_di, &s.col_up, &s.col_rh, &s.col_rx,
                      &s.col_tx, &s.col_px, &s.col_gm, &s.col_ri, &s.col_mm, &s.col_ws, &s.col_gc};
    for (double** p : col) *p = A.get_n<double>(C);
    s.vn = A.get_n<double>(E); s.vn_s = A.get_n<double>(E);
    s.Avn0 = A.get_n<double>(E); s.Aw0 = A.get_n<double>(C);
    s.zeta = A.get_n<double>(V); s.w_v = A.get_n<double>(V);
    s.vt = A.get_n<double>(E); s.Ke = A.get_n<double>(E); s.Kc = A.get_n<double>(C);
    s.a_e = A.get_n<double>(E); s.F = A.get_n<double>(E); s.G = A.get_n<double>(E);
    s.kin_w_h = A.get_n<double>(3 * (size_t)nc); s.div_wa_h = A.get_n<double>(3 * (size_t)nc);
    // diffusion scratch reuses substep scratch (they never overlap in time)
    s.Kh = s.vt; s.thflx = s.Ke; s.divc = s.Kc; s.uvx = s.w_v;
    s.uvy = A.get_n<double>(V); s.uvz = A.get_n<double>(V);
  } else {
    // FP64 prognostics level-major [k][Nc]; everything the stencils touch is FP32 [entity][ld]
    s.level_major = true;
    s.w = A.get_n<double>(nc * (ld0 + 1)); s.rho = A.get_n<double>(nc * ld0);
    s.thv = A.get_n<double>(nc * ld0); s.ex = A.get_n<double>(nc * ld0);
    s.wflx = A.get_n<double>(nc * (ld0 + 1));
    s.vn32 = A.get_n<float>(E); s.vn32_s = A.get_n<float>(E); s.Avn0_32 = A.get_n<float>(E);
    s.vt32 = A.get_n<float>(E); s.F32 = A.get_n<float>(E);
    s.G32 = A.get_n<float>(E); s.ae32 = A.get_n<float>(E);
    s.rho32 = A.get_n<float>(C); s.thv32 = A.get_n<float>(C); s.exp32 = A.get_n<float>(C); s.w32 = A.get_n<float>(C);
    s.rho32_s = A.get_n<float>(C); s.thv32_s = A.get_n<float>(C); s.exp32_s = A.get_n<float>(C);
    s.w32_s = A.get_n<float>(C); s.Kc32 = A.get_n<float>(C);
    s.Aw0_32 = A.get_n<float>(nc * (ld0 + 1));
    s.zeta32 = A.get_n<float>(V); s.wv32 = A.get_n<float>(V);
    // the diffusion's vertex vectors reuse buffers that are dead during diffusion
    // (vertex rows Nv*ld fit in cell rows Nc*ld)
    s.uvx32 = s.wv32; s.uvy32 = s.rho32_s; s.uvz32 = s.thv32_s;
    s.colconst = A.get_n<double>(8 * (size_t)ld);
    s.exref32 = A.get_n<float>(ld);
    // the column form: ICON_MIXED_COLUMN = "lean" (default), "stored" (the frozen parts of the
    // column system stored by the predictor for the corrector, when they take at most a
    // quarter of the device memory) or "recompute" (both stages compute them; also selected
    // by ICON_MIXED_RECOMPUTE=1). On terrain-following levels the lean column runs with the
    // cells' own tables (its stored base depends on S^n only; the explicit vertical fluxes,
    // which carry each stage's own contravariant correction, are formed in each stage); the
    // stored form is flat-only (it freezes those fluxes)
    const char* form = getenv("ICON_MIXED_COLUMN");
    const char* force_recompute = getenv("ICON_MIXED_RECOMPUTE");
    bool recompute = force_recompute && force_recompute[0] == '1' && force_recompute[1] == '\0';
    bool stored = false;
    if (form && strcmp(form, "recompute") == 0) recompute = true;
    if (form && strcmp(form, "stored") == 0) stored = true;
    if (!recompute && !stored) {
      const size_t H = (size_t)nc * (ld0 + 1);
      s.ln_dr64 = A.get_n<double>(H);
      s.ln_dt32 = A.get_n<float>(H);
      s.ln_aw32 = A.get_n<float>(H);
      s.ln_B = A.get_n<double>(H);
      s.ln_dp = A.get_n<double>(H);
      s.ln_cp = A.get_n<float>(H);
      s.ln_cd = A.get_n<double>(8 * (size_t)ld);
      s.ln_cf = A.get_n<float>(8 * (size_t)ld);
      s.ln_dwa = A.get_n<double>(3 * (size_t)nc);
      s.ln_cw32 = A.get_n<float>(4 * (size_t)nc);
      int hd = 0;
      for (int h = 0; h <= grid->vert.N; ++h)
        if (grid->vert.rayleigh[h] > 0.0) hd = h + 1;
      s.ln_hdamp = hd;
    } else if (!topo && !recompute) {
      alloc_mixed_factors(st);
    }
  }
  if (A.failed) {
    set_error("out of device memory allocating the state");
    return ICON_ENOMEM;
  }
  return ICON_OK;
}

int sync_status(icon_state* st, cudaStream_t stream) {
  unsigned h = 0;
  ICON_CUDA(cudaMemcpyAsync(&h, st->s.status, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
  ICON_CUDA(cudaStreamSynchronize(stream));
  if (h != 0) {
    ICON_CUDA(cudaMemsetAsync(st->s.status, 0, sizeof(unsigned), stream));
    ICON_CUDA(cudaStreamSynchronize(stream));
    if (h & 2u) {
      set_error("an in-kernel barrier wait ran out (status 0x%x)", h);
      return ICON_ETIMEOUT;
    }
    set_error("non-finite value in the prognostic state (status 0x%x)", h);
    return ICON_ENONFINITE;
  }
  return ICON_OK;
}

void enqueue_step(icon_state* st, double dt, int nsub, cudaStream_t stream) {
  if (st->s.ntr > 0) tracer_begin(st, stream);
  if (st->s.precision == ICON_FP64) enqueue_step_fp64(st, dt, nsub, stream);
  else enqueue_step_mixed(st, dt, nsub, stream);
  if (st->s.ntr > 0) tracer_end(st, dt, stream);
}

// record the graph of one step for (dt, nsub) unless it is already recorded
int record_graph(icon_state* st, double dt, int nsub) {
  if (st->graph && st->graph_dt == dt && st->graph_nsub == nsub) return ICON_OK;
  if (st->s.precision == ICON_MIXED && !st->tuned) {
    cudaStream_t ts = current_stream();
    autotune_mixed(st, dt, nsub, ts);
    ICON_CUDA(cudaGetLastError());
    ICON_CUDA(cudaStreamSynchronize(ts));
  }
  if (st->graph) {
    cudaGraphExecDestroy(st->graph);
    st->graph = nullptr;
  }
  if (!st->capture_stream) ICON_CUDA(cudaStreamCreateWithFlags(&st->capture_stream, cudaStreamNonBlocking));
  const char* ov = getenv("ICON_STEP_OVERLAP");
  if (st->s.precision == ICON_MIXED && !st->s.topo.on && !st->side_stream && !(ov && ov[0] == '0')) {
    ICON_CUDA(cudaStreamCreateWithFlags(&st->side_stream, cudaStreamNonBlocking));
    ICON_CUDA(cudaEventCreateWithFlags(&st->fork_ev, cudaEventDisableTiming));
    ICON_CUDA(cudaEventCreateWithFlags(&st->join_ev, cudaEventDisableTiming));
  }
  cudaGraph_t g = nullptr;
  ICON_CUDA(cudaStreamBeginCapture(st->capture_stream, cudaStreamCaptureModeThreadLocal));
  Prof* saved = t_prof;
  t_prof = nullptr;
  enqueue_step(st, dt, nsub, st->capture_stream);
  t_prof = saved;
  cudaError_t e = cudaStreamEndCapture(st->capture_stream, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
  int nk = 0;
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
  }
  e = cudaGraphInstantiate(&st->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    st->graph = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  st->graph_dt = dt;
  st->graph_nsub = nsub;
  st->graph_kernels = nk;
  return ICON_OK;
}

int launch_step(icon_state* st, double dt, int nsub, cudaStream_t stream) {
  int rc = record_graph(st, dt, nsub);
  if (rc != ICON_OK) return rc;
  ICON_CUDA(cudaGraphLaunch(st->graph, stream));
  return ICON_OK;
}

bool field_ref(const icon_state* st, int id, void** ptr, int* is_f32, int64_t* n, int* nlev, int* lm) {
  const icon_grid* grid = st->grid;
  const StateDev& s = st->s;
  const int N = grid->vert.N;
  *is_f32 = 0;
  *lm = (s.level_major && id != ICON_F_VN && id != ICON_F_MFLX) ? 1 : 0;
  switch (id) {
    case ICON_F_VN:
      *n = grid->g.ne; *nlev = N;
      if (s.precision == ICON_FP64) *ptr = s.vn; else { *ptr = s.vn32; *is_f32 = 1; }
      return true;
    case ICON_F_W: *ptr = s.w; *n = grid->g.nc; *nlev = N + 1; return true;
    case ICON_F_RHO: *ptr = s.rho; *n = grid->g.nc; *nlev = N; return true;
    case ICON_F_THETA_V: *ptr = s.thv; *n = grid->g.nc; *nlev = N; return true;
    case ICON_F_EXNER: *ptr = s.ex; *n = grid->g.nc; *nlev = N; return true;
    case ICON_F_MFLX: *ptr = s.mflx; *n = grid->g.ne; *nlev = N; return true;
    case ICON_F_WFLX: *ptr = s.wflx; *n = grid->g.nc; *nlev = N + 1; return true;
    default: return false;
  }
}

// the device address of pinned (page-locked, mapped) host memory, or NULL for any other
// pointer; the query allocates nothing
const void* mapped_host_ptr(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return attr.type == cudaMemoryTypeHost ? attr.devicePointer : nullptr;
}

// host-order [n][nlev] staging <-> the device layout of a field: mode 0 FP64 rows of
// ld, mode 1 FP32 rows of ld, mode 2 FP64 level-major [k][n]
__global__ void k_unpack(const double* __restrict__ stage, void* __restrict__ dst, int64_t n, int nlev, int ld,
                         int mode) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nlev) return;
  if (mode == 2) {
    const int64_t k = t / n, i = t % n;
    static_cast<double*>(dst)[t] = stage[i * nlev + k];
  } else {
    const int64_t i = t / nlev, k = t % nlev;
    if (mode == 0) static_cast<double*>(dst)[i * ld + k] = stage[t];
    else static_cast<float*>(dst)[i * ld + k] = (float)stage[t];
  }
}
__global__ void k_pack(const void* __restrict__ src, double* __restrict__ stage, int64_t n, int nlev, int ld,
                       int mode) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nlev) return;
  if (mode == 2) {
    const int64_t k = t / n, i = t % n;
    stage[i * nlev + k] = static_cast<const double*>(src)[t];
  } else {
    const int64_t i = t / nlev, k = t % nlev;
    stage[t] = mode == 0 ? static_cast<const double*>(src)[i * ld + k]
                         : (double)static_cast<const float*>(src)[i * ld + k];
  }
}

}  // namespace
}  // namespace icon

using namespace icon;

extern "C" {

int icon_set_allocator(void* (*alloc)(size_t, void*), void (*dealloc)(void*, void*), void* ctx) {
  if ((alloc == nullptr) != (dealloc == nullptr)) {
    set_error("icon_set_allocator: pass both callbacks or neither");
    return ICON_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.dealloc = dealloc;
  g_alloc.ctx = alloc ? ctx : nullptr;
  return ICON_OK;
}

int icon_set_stream(void* cuda_stream) {
  t_stream = static_cast<cudaStream_t>(cuda_stream);
  return ICON_OK;
}

const char* icon_last_error(void) { return t_err.c_str(); }

int icon_grid_build(int root, int bisections, int nlev, icon_grid** out) {
  if (!out) { set_error("icon_grid_build: out is NULL"); return ICON_EINVAL; }
  if (root != 2) { set_error("icon_grid_build: only root 2 is supported (got %d)", root); return ICON_EINVAL; }
  if (bisections < 0 || bisections > 10) {
    set_error("icon_grid_build: bisections must be in 0..10 (got %d)", bisections);
    return ICON_EINVAL;
  }
  if (nlev < 1 || nlev > 256) { set_error("icon_grid_build: nlev must be in 1..256 (got %d)", nlev); return ICON_EINVAL; }
  icon_grid* g = new icon_grid();
  g->root = root;
  g->bisections = bisections;
  g->arena.al = current_allocator();
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    cudaGetLastError();
    g->device = -1;
  }
  make_vertical(g->vert, nlev, -1, -1, -1);
  cudaStream_t st = current_stream();
  int rc = upload_vertical(g, st);
  if (rc == ICON_OK) rc = build_grid_device(g, st);
  if (rc == ICON_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "grid build");
  }
  if (rc != ICON_OK) {
    cudaStreamSynchronize(st);
    g->arena.release();
    delete g;
    return rc;
  }
  *out = g;
  return ICON_OK;
}

int icon_grid_counts(const icon_grid* grid, int64_t* nc, int64_t* ne, int64_t* nv) {
  if (!grid) { set_error("icon_grid_counts: grid is NULL"); return ICON_EINVAL; }
  if (nc) *nc = grid->g.nc;
  if (ne) *ne = grid->g.ne;
  if (nv) *nv = grid->g.nv;
  return ICON_OK;
}

int icon_grid_copy_table(const icon_grid* grid, int table_id, void* host_dst, size_t bytes) {
  if (!grid || !host_dst) { set_error("icon_grid_copy_table: NULL argument"); return ICON_EINVAL; }
  if ((table_id == ICON_T_C2C || table_id == ICON_G_LSQC || table_id == ICON_G_ROFF) && !grid->g.c2c) {
    const int rc = build_tracer_tables(const_cast<icon_grid*>(grid), current_stream());
    if (rc != ICON_OK) return rc;
  }
  TableRef t;
  if (!table_ref(grid, table_id, t)) { set_error("icon_grid_copy_table: unknown table %d", table_id); return ICON_EINVAL; }
  if (bytes != t.elem * t.count) {
    set_error("icon_grid_copy_table: table %d has %zu bytes, got %zu", table_id, t.elem * t.count, bytes);
    return ICON_EINVAL;
  }
  cudaStream_t st = current_stream();
  ICON_CUDA(cudaMemcpyAsync(host_dst, t.ptr, bytes, cudaMemcpyDeviceToHost, st));
  ICON_CUDA(cudaStreamSynchronize(st));
  return ICON_OK;
}

void icon_grid_free(icon_grid* grid) {
  if (!grid) return;
  cudaDeviceSynchronize();
  grid->arena.release();
  delete grid;
}

int icon_state_init_ex(const icon_grid* grid, uint64_t seed, int case_id, const icon_case_params* params,
                       icon_state** out) {
  if (!grid || !out) { set_error("icon_state_init: NULL argument"); return ICON_EINVAL; }
  if (case_id < ICON_CASE_REST || case_id > ICON_CASE_MEMBER) {
    set_error("icon_state_init: unknown case %d", case_id);
    return ICON_EINVAL;
  }
  if (grid->vert.N < 2) { set_error("icon_state_init: the dycore needs nlev >= 2"); return ICON_EINVAL; }
  icon_case_params p;
  p.noise_K = -1.0; p.top_m = -1.0; p.stretch_s = -1.0; p.damp_m = -1.0; p.precision = ICON_FP64; p.member = 0;
  p.topo_height_m = 0.0; p.topo_radius_m = 0.0;
  if (params) p = *params;
  const bool topo = p.topo_height_m != 0.0;
  if (topo && !(p.topo_height_m > 0.0 && p.topo_height_m <= 0.5 * kTopoDecay && p.topo_radius_m >= 1e4)) {
    set_error("icon_state_init: topography needs 0 < height <= %g m and radius >= 1e4 m (got %g, %g)",
              0.5 * kTopoDecay, p.topo_height_m, p.topo_radius_m);
    return ICON_EINVAL;
  }

  if (p.precision != ICON_FP64 && p.precision != ICON_MIXED) {
    set_error("icon_state_init: unknown precision %d", p.precision);
    return ICON_EINVAL;
  }
  if (p.member < 0) { set_error("icon_state_init: member must be >= 0"); return ICON_EINVAL; }
  if ((p.top_m > 0 && p.top_m != grid->vert.z_top) || (p.stretch_s > 0 && p.stretch_s != grid->vert.s) ||
      (p.damp_m > 0 && p.damp_m != grid->vert.z_d)) {
    set_error("icon_state_init: vertical-grid overrides must match the grid's (top %g, s %g, damping base %g)",
              grid->vert.z_top, grid->vert.s, grid->vert.z_d);
    return ICON_EINVAL;
  }
  icon_state* st = new icon_state();
  st->grid = grid;
  st->seed = seed;
  st->case_id = case_id;
  st->divdamp4 = kDivDamp4;
  st->abar = 4.0 * M_PI * kR * kR / (double)grid->g.nc;
  st->arena.al = current_allocator();
  cudaStream_t stream = current_stream();
  int rc = alloc_state(st, p.precision, topo);
  if (rc == ICON_OK) {
    cudaError_t e = cudaMemsetAsync(st->s.status, 0, 64 * sizeof(unsigned), stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync");
  }
  if (rc == ICON_OK && topo) rc = topo_build(st, p.topo_height_m, p.topo_radius_m, stream);
  if (rc == ICON_OK) rc = init_state_device(st, seed, case_id, p, stream);
  if (rc == ICON_OK) {
    cudaError_t e = cudaEventCreateWithFlags(&st->done, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaEventCreate");
  }
  if (rc == ICON_OK) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "state init");
  }
  if (rc != ICON_OK) {
    cudaStreamSynchronize(stream);
    if (st->done) cudaEventDestroy(st->done);
    st->arena.release();
    delete st;
    return rc;
  }
  *out = st;
  return ICON_OK;
}

int icon_state_init(const icon_grid* grid, uint64_t seed, int case_id, icon_state** out) {
  return icon_state_init_ex(grid, seed, case_id, nullptr, out);
}

int icon_dycore_step_async(icon_state* st, double dt, int nsubsteps) {
  if (!st) { set_error("icon_dycore_step: state is NULL"); return ICON_EINVAL; }
  if (!(dt > 0.0) || nsubsteps < 1 || nsubsteps > 64) {
    set_error("icon_dycore_step: need dt > 0 and 1 <= nsubsteps <= 64 (got %g, %d)", dt, nsubsteps);
    return ICON_EINVAL;
  }
  return launch_step(st, dt, nsubsteps, current_stream());
}

int icon_dycore_step(icon_state* st, double dt, int nsubsteps) {
  int rc = icon_dycore_step_async(st, dt, nsubsteps);
  if (rc != ICON_OK) return rc;
  return sync_status(st, current_stream());
}

int icon_state_status(icon_state* st) {
  if (!st) { set_error("icon_state_status: state is NULL"); return ICON_EINVAL; }
  return sync_status(st, current_stream());
}

int icon_global_mass(const icon_state* st, double* out) {
  if (!st || !out) { set_error("icon_global_mass: NULL argument"); return ICON_EINVAL; }
  cudaStream_t stream = current_stream();
  double* d_out = st->s.mass_part + mass_partials_count(st->grid->g.nc);
  enqueue_mass(st, d_out, stream);
  ICON_CUDA(cudaGetLastError());
  double h = 0.0;
  ICON_CUDA(cudaMemcpyAsync(&h, d_out, sizeof(double), cudaMemcpyDeviceToHost, stream));
  ICON_CUDA(cudaStreamSynchronize(stream));
  *out = h;
  return ICON_OK;
}

int icon_global_mass_async(const icon_state* st, double* host_out) {
  if (!st || !host_out) { set_error("icon_global_mass_async: NULL argument"); return ICON_EINVAL; }
  cudaStream_t stream = current_stream();
  double* d_out = st->s.mass_part + mass_partials_count(st->grid->g.nc);
  enqueue_mass(st, d_out, stream);
  ICON_CUDA(cudaGetLastError());
  ICON_CUDA(cudaMemcpyAsync(host_out, d_out, sizeof(double), cudaMemcpyDeviceToHost, stream));
  return ICON_OK;
}

int icon_state_step_kernels(icon_state* st, double dt, int nsubsteps, int* out) {
  if (!st || !out) { set_error("icon_state_step_kernels: NULL argument"); return ICON_EINVAL; }
  if (!(dt > 0.0) || nsubsteps < 1 || nsubsteps > 64) {
    set_error("icon_state_step_kernels: need dt > 0 and 1 <= nsubsteps <= 64");
    return ICON_EINVAL;
  }
  int rc = record_graph(st, dt, nsubsteps);
  if (rc != ICON_OK) return rc;
  *out = st->graph_kernels;
  return ICON_OK;
}

int icon_dycore_step_profile(icon_state* st, double dt, int nsubsteps, double* ms_per_kind, int* launches_per_kind) {
  if (!st || !ms_per_kind || !launches_per_kind) { set_error("icon_dycore_step_profile: NULL argument"); return ICON_EINVAL; }
  if (!(dt > 0.0) || nsubsteps < 1 || nsubsteps > 64) { set_error("icon_dycore_step_profile: bad dt/nsubsteps"); return ICON_EINVAL; }
  cudaStream_t stream = current_stream();
  Prof prof;
  t_prof = &prof;
  enqueue_step(st, dt, nsubsteps, stream);
  t_prof = nullptr;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  int rc = ICON_OK;
  if (e != cudaSuccess) rc = cuda_fail(e, "icon_dycore_step_profile");
  if (rc == ICON_OK && prof.failed) { set_error("icon_dycore_step_profile: event creation failed"); rc = ICON_ECUDA; }
  if (rc == ICON_OK) {
    for (size_t i = 0; i < prof.kind.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, prof.ev[2 * i], prof.ev[2 * i + 1]);
      ms_per_kind[prof.kind[i]] += ms;
      launches_per_kind[prof.kind[i]] += 1;
    }
  }
  for (cudaEvent_t ev : prof.ev) cudaEventDestroy(ev);
  if (rc != ICON_OK) return rc;
  return sync_status(st, stream);
}

int icon_selftest(long long n, unsigned* failures) {
  if (!failures || n < 1) { set_error("icon_selftest: bad argument"); return ICON_EINVAL; }
  return selftest_conversions(n, failures);
}

const char* icon_kernel_kind_name(int kind) {
  if (kind < 0 || kind >= K_KIND_COUNT) return nullptr;
  return kKindNames[kind];
}

int icon_state_copy_field(const icon_state* st, int field_id, double* host_dst, size_t count) {
  if (!st || !host_dst) { set_error("icon_state_copy_field: NULL argument"); return ICON_EINVAL; }
  void* ptr;
  int f32, nlev, lm;
  int64_t n;
  if (!field_ref(st, field_id, &ptr, &f32, &n, &nlev, &lm)) {
    set_error("icon_state_copy_field: unknown field %d", field_id);
    return ICON_EINVAL;
  }
  if (count != (size_t)(n * nlev)) {
    set_error("icon_state_copy_field: field %d has %lld elements, got %zu", field_id, (long long)(n * nlev), count);
    return ICON_EINVAL;
  }
  // pack into host order on the device, then one contiguous transfer; into pinned host
  // memory of a row-layout field the pack kernel writes the host buffer directly (the GPU
  // reaches page-locked host memory over the CPU-GPU link: one pass, no staging copy)
  const int ld = st->grid->vert.ld;
  cudaStream_t stream = current_stream();
  if (!lm) {
    void* hd = const_cast<void*>(mapped_host_ptr(host_dst));
    if (hd) {
      k_pack<<<blocks_for(n * nlev, 256), 256, 0, stream>>>(ptr, static_cast<double*>(hd), n, nlev, ld,
                                                           f32 ? 1 : 0);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) return cuda_fail(e, "icon_state_copy_field");
      return ICON_OK;
    }
  }
  DeviceArena tmp;
  tmp.al = st->arena.al;
  double* stage = tmp.get_n<double>((size_t)n * nlev);
  if (!stage) { set_error("icon_state_copy_field: out of device memory"); return ICON_ENOMEM; }
  k_pack<<<blocks_for(n * nlev, 256), 256, 0, stream>>>(ptr, stage, n, nlev, ld, lm ? 2 : (f32 ? 1 : 0));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_dst, stage, sizeof(double) * n * nlev, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  tmp.release();
  if (e != cudaSuccess) return cuda_fail(e, "icon_state_copy_field");
  return ICON_OK;
}

int icon_state_set_field(icon_state* st, int field_id, const double* host_src, size_t count) {
  if (!st || !host_src) { set_error("icon_state_set_field: NULL argument"); return ICON_EINVAL; }
  if (field_id < ICON_F_VN || field_id > ICON_F_EXNER) {
    set_error("icon_state_set_field: field %d is not a prognostic field", field_id);
    return ICON_EINVAL;
  }
  void* ptr;
  int f32, nlev, lm;
  int64_t n;
  field_ref(st, field_id, &ptr, &f32, &n, &nlev, &lm);
  if (count != (size_t)(n * nlev)) {
    set_error("icon_state_set_field: field %d has %lld elements, got %zu", field_id, (long long)(n * nlev), count);
    return ICON_EINVAL;
  }
  // one contiguous transfer into a staging buffer, then unpack into the device layout; from
  // pinned host memory into a row-layout field the unpack kernel reads the host buffer directly
  const int ld = st->grid->vert.ld;
  cudaStream_t stream = current_stream();
  if (!lm) {
    const void* hs = mapped_host_ptr(host_src);
    if (hs) {
      k_unpack<<<blocks_for(n * nlev, 256), 256, 0, stream>>>(static_cast<const double*>(hs), ptr, n, nlev, ld,
                                                             f32 ? 1 : 0);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) return cuda_fail(e, "icon_state_set_field");
      return ICON_OK;
    }
  }
  DeviceArena tmp;
  tmp.al = st->arena.al;
  double* stage = tmp.get_n<double>((size_t)n * nlev);
  if (!stage) { set_error("icon_state_set_field: out of device memory"); return ICON_ENOMEM; }
  cudaError_t e = cudaMemcpyAsync(stage, host_src, sizeof(double) * n * nlev, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) {
    k_unpack<<<blocks_for(n * nlev, 256), 256, 0, stream>>>(stage, ptr, n, nlev, ld, lm ? 2 : (f32 ? 1 : 0));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && lm) {
    mixed_refresh_shadows(st, stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  tmp.release();
  if (e != cudaSuccess) return cuda_fail(e, "icon_state_set_field");
  return ICON_OK;
}

int icon_state_tiling(const icon_state* st, int kind, int* lanes, int* block) {
  if (!st || !lanes || !block || kind < 0 || kind >= ICON_KIND_COUNT) {
    set_error("icon_state_tiling: bad argument");
    return ICON_EINVAL;
  }
  *lanes = st->tile[kind].lanes;
  *block = st->tile[kind].block;
  return ICON_OK;
}

int icon_state_set_tiling(icon_state* st, int kind, int lanes, int block) {
  if (!st || kind < 0 || kind >= ICON_KIND_COUNT) { set_error("icon_state_set_tiling: bad argument"); return ICON_EINVAL; }
  if (lanes != 0 && kind == K_MX_LEAN) {
    if (!lean_column_shape_ok(lanes, block)) {
      set_error("icon_state_set_tiling: the lean column takes (unroll, blocks per SM) (2, 9), (2, 10), (2, 8), (2, 12) or (2, 6)");
      return ICON_EINVAL;
    }
  } else if (lanes != 0 && ((lanes != 8 && lanes != 16 && lanes != 32) ||
                            (block != 64 && block != 128 && block != 256 && block != 512))) {
    set_error("icon_state_set_tiling: lanes must be 8, 16 or 32 and block 64, 128, 256 or 512");
    return ICON_EINVAL;
  }
  st->tile[kind] = TileChoice{lanes, lanes ? block : 0};
  st->tile_forced[kind] = lanes != 0;
  if (lanes == 0) st->tuned = false;
  if (st->graph) {
    cudaGraphExecDestroy(st->graph);
    st->graph = nullptr;
  }
  return ICON_OK;
}

int icon_state_precision(const icon_state* st, int* out) {
  if (!st || !out) { set_error("icon_state_precision: NULL argument"); return ICON_EINVAL; }
  *out = st->s.precision;
  return ICON_OK;
}

void icon_state_free(icon_state* st) {
  if (!st) return;
  cudaDeviceSynchronize();
  if (st->graph) cudaGraphExecDestroy(st->graph);
  if (st->capture_stream) cudaStreamDestroy(st->capture_stream);
  if (st->side_stream) cudaStreamDestroy(st->side_stream);
  if (st->fork_ev) cudaEventDestroy(st->fork_ev);
  if (st->join_ev) cudaEventDestroy(st->join_ev);
  if (st->done) cudaEventDestroy(st->done);
  st->arena.release();
  delete st;
}

}  // extern "C"

// ---------------------------------------------------------------- ensemble
struct icon_ensemble {
  std::vector<icon_state*> members;
  icon::EnsembleDev E;
  std::vector<double> dts;
  int nsub = 0;
  bool prepared = false;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t capture_stream = nullptr;
  unsigned long long* prof = nullptr;   // phase stamps of icon_ensemble_step_profile
  int prof_cap = 0;
};

extern "C" {

int icon_state_add_tracers(icon_state* st, int ntracers) {
  if (!st) { set_error("icon_state_add_tracers: state is NULL"); return ICON_EINVAL; }
  if (ntracers < 1 || ntracers > 8) { set_error("icon_state_add_tracers: need 1..8 tracers"); return ICON_EINVAL; }
  if (st->s.ntr != 0) { set_error("icon_state_add_tracers: the state already has tracers"); return ICON_EINVAL; }
  const int rc = tracer_alloc(st, ntracers);
  if (rc != ICON_OK) return rc;
  if (st->graph) {                      // the step's graph now has to transport them too
    cudaGraphExecDestroy(st->graph);
    st->graph = nullptr;
  }
  return ICON_OK;
}

int icon_state_set_option(icon_state* st, int option, double value) {
  if (!st) { set_error("icon_state_set_option: state is NULL"); return ICON_EINVAL; }
  if (option == ICON_OPT_DIVDAMP4) {
    if (!(value >= 0.0 && value <= 0.05)) {
      set_error("icon_state_set_option: divergence damping coefficient %g outside [0, 0.05]", value);
      return ICON_EINVAL;
    }
    st->divdamp4 = value;
  } else if (option == ICON_OPT_DIFF4) {
    if (!(value >= 0.0 && value <= 0.01)) {
      set_error("icon_state_set_option: background diffusion coefficient %g outside [0, 0.01]", value);
      return ICON_EINVAL;
    }
    st->diff4 = value;
  } else if (option == ICON_OPT_UPWIND_THETA) {
    if (value != 0.0 && value != 1.0) {
      set_error("icon_state_set_option: upwind theta takes 0 or 1, got %g", value);
      return ICON_EINVAL;
    }
    st->upwind_theta = value == 1.0;
  } else {
    set_error("icon_state_set_option: unknown option %d", option);
    return ICON_EINVAL;
  }
  if (st->graph) {                      // the step's graph changes with the option
    cudaGraphExecDestroy(st->graph);
    st->graph = nullptr;
  }
  return ICON_OK;
}

int icon_state_tracers(const icon_state* st, int* out) {
  if (!st || !out) { set_error("icon_state_tracers: NULL argument"); return ICON_EINVAL; }
  *out = st->s.ntr;
  return ICON_OK;
}

static int tracer_copy(icon_state* st, int t, double* host, size_t count, bool to_host) {
  const char* fn = to_host ? "icon_state_copy_tracer" : "icon_state_set_tracer";
  if (!st || !host) { set_error("%s: NULL argument", fn); return ICON_EINVAL; }
  if (t < 0 || t >= st->s.ntr) { set_error("%s: tracer %d of %d", fn, t, st->s.ntr); return ICON_EINVAL; }
  const int64_t nc = st->grid->g.nc;
  const int N = st->grid->vert.N, ld = st->grid->vert.ld;
  if (count != (size_t)(nc * N)) {
    set_error("%s: a tracer has %lld elements, got %zu", fn, (long long)(nc * N), count);
    return ICON_EINVAL;
  }
  double* dev = st->s.q + (size_t)t * nc * ld;
  cudaStream_t stream = current_stream();
  cudaError_t e = to_host ? cudaMemcpy2DAsync(host, sizeof(double) * N, dev, sizeof(double) * ld, sizeof(double) * N,
                                              nc, cudaMemcpyDeviceToHost, stream)
                          : cudaMemcpy2DAsync(dev, sizeof(double) * ld, host, sizeof(double) * N, sizeof(double) * N,
                                              nc, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return ICON_OK;
}

int icon_state_set_tracer(icon_state* st, int t, const double* host_src, size_t count) {
  return tracer_copy(st, t, const_cast<double*>(host_src), count, false);
}

int icon_state_copy_tracer(const icon_state* st, int t, double* host_dst, size_t count) {
  return tracer_copy(const_cast<icon_state*>(st), t, host_dst, count, true);
}

int icon_ensemble_create(icon_state* const* members, int n, icon_ensemble** out) {
  if (!members || !out || n < 1 || n > 64) { set_error("icon_ensemble_create: need 1..64 members"); return ICON_EINVAL; }
  for (int i = 0; i < n; ++i) {
    if (!members[i]) { set_error("icon_ensemble_create: member %d is NULL", i); return ICON_EINVAL; }
    if (members[i]->s.precision != ICON_MIXED) {
      set_error("icon_ensemble_create: members must be mixed-precision states");
      return ICON_EINVAL;
    }
    if (members[i]->diff4 != 0.0 || members[i]->upwind_theta) {
      set_error("icon_ensemble_create: the persistent ensemble has the divergence damping but not the other step "
                "options (member %d sets one)", i);
      return ICON_EINVAL;
    }
    if (members[i]->s.ntr != 0) {
      set_error("icon_ensemble_create: the persistent ensemble does not transport tracers (member %d has some)", i);
      return ICON_EINVAL;
    }
    if (members[i]->s.topo.on) {
      set_error("icon_ensemble_create: the persistent ensemble runs on flat levels only (member %d has topography)", i);
      return ICON_EINVAL;
    }
    if (members[i]->grid->vert.N != members[0]->grid->vert.N || members[i]->grid->vert.N > 96) {
      set_error("icon_ensemble_create: members must share one level count of at most 96");
      return ICON_EINVAL;
    }
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) { set_error("icon_ensemble_create: member %d repeats member %d", i, j); return ICON_EINVAL; }
  }
  icon_ensemble* e = new icon_ensemble();
  e->members.assign(members, members + n);
  e->E.arena.al = current_allocator();
  *out = e;
  return ICON_OK;
}

int icon_ensemble_set_option(icon_ensemble* ens, int option, long long value) {
  if (!ens) { set_error("icon_ensemble_set_option: ensemble is NULL"); return ICON_EINVAL; }
  if (option == ICON_ENS_SPIN_LIMIT && value > 0) ens->E.spin_limit = value;
  else if (option == ICON_ENS_TEST_SKIP_BARRIER && (value == 0 || value == 1)) ens->E.test_skip_barrier = (int)value;
  else { set_error("icon_ensemble_set_option: bad option %d or value %lld", option, value); return ICON_EINVAL; }
  if (ens->graph) {
    cudaGraphExecDestroy(ens->graph);
    ens->graph = nullptr;
  }
  return ICON_OK;
}

int icon_ensemble_step(icon_ensemble* ens, const double* dt_per_member, int nsubsteps, int nsteps) {
  if (!ens || !dt_per_member || nsteps < 0 || nsubsteps < 1 || nsubsteps > 64) {
    set_error("icon_ensemble_step: bad arguments");
    return ICON_EINVAL;
  }
  const int n = (int)ens->members.size();
  for (int i = 0; i < n; ++i)
    if (!(dt_per_member[i] > 0.0)) { set_error("icon_ensemble_step: dt of member %d must be > 0", i); return ICON_EINVAL; }
  cudaStream_t stream = current_stream();
  std::vector<double> dts(dt_per_member, dt_per_member + n);
  if (!ens->prepared || dts != ens->dts || nsubsteps != ens->nsub) {
    int rc = ensemble_prepare(ens->E, ens->members.data(), n, dts.data(), nsubsteps);
    if (rc != ICON_OK) return rc;
    ens->prepared = true;
    ens->dts = dts;
    ens->nsub = nsubsteps;
    if (ens->graph) {
      cudaGraphExecDestroy(ens->graph);
      ens->graph = nullptr;
    }
  }
  if (!ens->graph) {
    // one step: reset the barrier words, then the cooperative persistent launch
    if (!ens->capture_stream) ICON_CUDA(cudaStreamCreateWithFlags(&ens->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    ICON_CUDA(cudaStreamBeginCapture(ens->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(ens->E.bar, 0, 8 * sizeof(unsigned), ens->capture_stream);
    int rc = e == cudaSuccess ? ensemble_launch(ens->E, ens->capture_stream) : cuda_fail(e, "cudaMemsetAsync");
    cudaError_t e2 = cudaStreamEndCapture(ens->capture_stream, &g);
    if (rc != ICON_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture (ensemble)");
    e = cudaGraphInstantiate(&ens->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { ens->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate (ensemble)"); }
  }
  ICON_CUDA(cudaMemsetAsync(ens->E.bar + 8, 0, sizeof(unsigned), stream));
  for (int s = 0; s < nsteps; ++s) ICON_CUDA(cudaGraphLaunch(ens->graph, stream));
  unsigned h = 0;
  ICON_CUDA(cudaMemcpyAsync(&h, ens->E.bar + 8, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
  ICON_CUDA(cudaStreamSynchronize(stream));
  int worst = ICON_OK;
  for (int i = 0; i < n; ++i) {
    int rc = sync_status(ens->members[i], stream);
    if (rc != ICON_OK) worst = rc;
  }
  if (h & 2u) {
    ICON_CUDA(cudaMemsetAsync(ens->E.bar, 0, 16 * sizeof(unsigned), stream));
    ICON_CUDA(cudaStreamSynchronize(stream));
    set_error("icon_ensemble_step: a grid-barrier wait ran out; the members' states are not valid");
    return ICON_ETIMEOUT;
  }
  return worst;
}

static const char* kEnsPhaseNames[ICON_ENS_PHASE_COUNT] = {
    "zero", "vertex", "edge_diag", "cell_ke", "edge_tend", "dd_div", "dd_lap",
    "dd_edge", "gather", "column", "corr_update", "diff_vertex", "diff_edge", "diff_theta"};

const char* icon_ensemble_phase_name(int phase) {
  if (phase < 0 || phase >= ICON_ENS_PHASE_COUNT) return nullptr;
  return kEnsPhaseNames[phase];
}

int icon_ensemble_step_profile(icon_ensemble* ens, const double* dt_per_member, int nsubsteps, double* ms_per_phase,
                               int* count_per_phase) {
  if (!ens || !dt_per_member || !ms_per_phase || !count_per_phase || nsubsteps < 1 || nsubsteps > 64) {
    set_error("icon_ensemble_step_profile: bad arguments");
    return ICON_EINVAL;
  }
  const int n = (int)ens->members.size();
  for (int i = 0; i < n; ++i)
    if (!(dt_per_member[i] > 0.0)) { set_error("icon_ensemble_step_profile: dt of member %d must be > 0", i); return ICON_EINVAL; }
  std::vector<double> dts(dt_per_member, dt_per_member + n);
  if (!ens->prepared || dts != ens->dts || nsubsteps != ens->nsub) {
    int rc = ensemble_prepare(ens->E, ens->members.data(), n, dts.data(), nsubsteps);
    if (rc != ICON_OK) return rc;
    ens->prepared = true;
    ens->dts = dts;
    ens->nsub = nsubsteps;
    if (ens->graph) {
      cudaGraphExecDestroy(ens->graph);
      ens->graph = nullptr;
    }
  }
  // barriers per step: 1 + nsub x 2 stages x (at most 10) + 2, and the start and end stamps
  const int cap = 8 + 20 * nsubsteps;
  if (!ens->prof || ens->prof_cap < cap) {
    ens->prof = ens->E.arena.get_n<unsigned long long>(2 * (size_t)cap);
    if (!ens->prof) { set_error("icon_ensemble_step_profile: out of device memory"); return ICON_ENOMEM; }
    ens->prof_cap = cap;
  }
  cudaStream_t stream = current_stream();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ICON_CUDA(cudaEventCreate(&e0));
  ICON_CUDA(cudaEventCreate(&e1));
  ICON_CUDA(cudaMemsetAsync(ens->prof, 0, sizeof(unsigned long long) * 2 * cap, stream));
  ICON_CUDA(cudaMemsetAsync(ens->E.bar, 0, 16 * sizeof(unsigned), stream));
  ICON_CUDA(cudaEventRecord(e0, stream));
  int rc = ensemble_launch(ens->E, stream, ens->prof, cap);
  ICON_CUDA(cudaEventRecord(e1, stream));
  std::vector<unsigned long long> h(2 * (size_t)cap);
  unsigned bar_status = 0;
  ICON_CUDA(cudaMemcpyAsync(h.data(), ens->prof, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, stream));
  ICON_CUDA(cudaMemcpyAsync(&bar_status, ens->E.bar + 8, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
  ICON_CUDA(cudaStreamSynchronize(stream));
  float total = 0.f;
  cudaEventElapsedTime(&total, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != ICON_OK) return rc;
  if (bar_status & 2u) {
    ICON_CUDA(cudaMemsetAsync(ens->E.bar, 0, 16 * sizeof(unsigned), stream));
    ICON_CUDA(cudaStreamSynchronize(stream));
    set_error("icon_ensemble_step_profile: a grid-barrier wait ran out; the members' states are not valid");
    return ICON_ETIMEOUT;
  }
  // stamps: (kind, ns) pairs, the first the start (kind ICON_ENS_PHASE_COUNT), the last
  // block 0's end of the final phase
  int ns = 0;
  while (ns < cap && h[2 * ns + 1] != 0) ++ns;
  double used = 0.0;
  for (int i = 1; i < ns; ++i) {
    const int kind = (int)h[2 * i];
    const double ms = (double)(h[2 * i + 1] - h[2 * i - 1]) * 1e-6;
    if (i == ns - 1) break;                            // the last phase: closed below
    if (kind >= 0 && kind < ICON_ENS_PHASE_COUNT) {
      ms_per_phase[kind] += ms;
      count_per_phase[kind] += 1;
      used += ms;
    }
  }
  if (ns >= 2) {
    const int kind = (int)h[2 * (ns - 1)];
    if (kind >= 0 && kind < ICON_ENS_PHASE_COUNT) {
      ms_per_phase[kind] += total - used > 0.0 ? total - used : 0.0;
      count_per_phase[kind] += 1;
    }
  }
  int worst = ICON_OK;
  for (int i = 0; i < n; ++i) {
    int r = sync_status(ens->members[i], stream);
    if (r != ICON_OK) worst = r;
  }
  return worst;
}

void icon_ensemble_free(icon_ensemble* ens) {
  if (!ens) return;
  cudaDeviceSynchronize();
  if (ens->graph) cudaGraphExecDestroy(ens->graph);
  if (ens->capture_stream) cudaStreamDestroy(ens->capture_stream);
  ens->E.arena.release();
  delete ens;
}

}  // extern "C"
