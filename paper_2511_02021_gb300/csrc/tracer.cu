// Tracer transport with the dycore step's mean mass fluxes (FP64, sm_103a).
//
// The paper's atmosphere carries water, CO2 and ozone tracers (Sec. "Overview of the
// Problem"); it prints no transport scheme. This is a flux-form, second-order,
// mass-consistent step (Miura-type) for mixing ratios q, run after every dycore step
// with that step's substep-averaged FP64 mass fluxes M (edge-levels, c1 -> c2) and W
// (half levels, upward):
//   gradient   g_c = sum_s G_cs (q_nb(c,s) - q_c), least-squares weights G (grid table)
//   edge value donor cd = c1 if M >= 0 else c2; rho_e = (rho_c1 + rho_c2)/2 of the
//              step's initial density; v_n = M / rho_e; v_t = (sum_j W_ej M_j) / rho_e
//              with the dycore's tangential weights; q_e = q_cd + g_cd . (R (x_e - x_cd)
//              - dt/2 (v_n n_e + v_t t_e))
//   half level donor level kd = h if W >= 0 (below) else h - 1; centred slope s_kd;
//              w_h = W / rho_ic; q_h = q_kd + s_kd (z_h - z_kd - dt/2 w_h); no flux
//              through the lid and the ground
//   update     q' = (rho^n q - dt [(1/A_c) sum_s s_ce l_e M q_e + (W q)_k - (W q)_{k+1}) / dz_k])
//              / rho^{n+1}
// With the dycore's fluxes rho^{n+1} = rho^n - dt div(M, W) to rounding, so a uniform
// tracer stays uniform and tracer mass is conserved. Three warp-per-entity kernels with
// lanes over levels per tracer: cell (gradient and vertical fluxes), edge (horizontal
// fluxes), cell (update, in place). Densities and W are read in the [cell][level]
// layout; a mixed-precision state's level-major FP64 fields are transposed first.
// On terrain-following levels (the TOPO instances) M carries the layer thickness dz_e
// and W is contravariant: v_n = M / (rho_e dz_e), each cell's own spacings and weights
// in the vertical reconstruction, and the update divides both flux divergences by the
// cell's dz.
#include "icon_internal.h"
#include "recip64.h"

namespace icon {
namespace {

constexpr int kTrWarps = 8;

struct TrArgs {
  int64_t nc, ne;
  int N, ld;
  const int *c2e, *e2c, *c2c, *e2vt;
  const double *lsq_c, *roff, *n_e, *t_e, *vt_w, *div_wa;
  const double *inv_dz, *wu, *wl, *lev;     // lev: [3][ld] slope 1/(dz), offsets below / above
  const double *rho0, *rho1, *W, *M;        // [c][ld], [c][ld], [c][ld] (half levels), [e][ld]
  const double *t_dz_c, *t_inv_dz_c, *t_wu_c, *t_dz_e;   // terrain-following levels, [entity][ld]
  double* q;                                // [c][ld], updated in place
  double *gx, *gy, *gz, *V, *F;
  unsigned* status;
  double dt;
};

__device__ inline int64_t tr_warp() {
  return (int64_t)blockIdx.x * kTrWarps + (threadIdx.x >> 5);
}

__device__ inline bool tr_finite(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// least-squares gradient at full levels; vertical flux W q_h at half levels
template <bool TOPO>
__global__ void __launch_bounds__(256) k_tr_cell(TrArgs a) {
  const int64_t c = tr_warp();
  if (c >= a.nc) return;
  const int lane = threadIdx.x & 31, N = a.N, ld = a.ld;
  const int64_t o = c * ld;
  int64_t nb[3];
  double G[3][3];
  for (int s = 0; s < 3; ++s) {
    nb[s] = (int64_t)a.c2c[3 * c + s] * ld;
    for (int j = 0; j < 3; ++j) G[s][j] = a.lsq_c[9 * c + 3 * s + j];
  }
  const double* __restrict__ q = a.q;
  for (int k = lane; k < N; k += 32) {
    const double qk = q[o + k];
    const double d0 = q[nb[0] + k] - qk, d1 = q[nb[1] + k] - qk, d2 = q[nb[2] + k] - qk;
    a.gx[o + k] = (G[0][0] * d0 + G[1][0] * d1) + G[2][0] * d2;
    a.gy[o + k] = (G[0][1] * d0 + G[1][1] * d1) + G[2][1] * d2;
    a.gz[o + k] = (G[0][2] * d0 + G[1][2] * d1) + G[2][2] * d2;
  }
  const double hdt = 0.5 * a.dt;
  for (int h = lane; h <= N; h += 32) {
    double flux = 0.0;
    if (h >= 1 && h < N) {
      const double W = a.W[o + h];
      const bool up = W >= 0.0;
      const int kd = up ? h : h - 1;
      double sd = 0.0, rho_ic, off;
      if constexpr (TOPO) {
        // zf_{k-1} - zf_{k+1} = dz_{k-1}/2 + dz_k + dz_{k+1}/2; z_h - zf of the donor = +-dz/2
        const double* dz = a.t_dz_c + o;
        if (kd >= 1 && kd + 1 < N)
          sd = (q[o + kd - 1] - q[o + kd + 1]) * recip64((0.5 * dz[kd - 1] + dz[kd]) + 0.5 * dz[kd + 1]);
        const double wu = a.t_wu_c[o + h];
        rho_ic = wu * a.rho0[o + h - 1] + (1.0 - wu) * a.rho0[o + h];
        off = up ? 0.5 * dz[h] : -0.5 * dz[h - 1];
      } else {
        sd = (kd >= 1 && kd + 1 < N) ? (q[o + kd - 1] - q[o + kd + 1]) * a.lev[kd] : 0.0;
        rho_ic = a.wu[h] * a.rho0[o + h - 1] + a.wl[h] * a.rho0[o + h];
        off = up ? a.lev[ld + h] : a.lev[2 * ld + h];
      }
      const double wh = W * recip64(rho_ic);
      flux = W * (q[o + kd] + sd * (off - hdt * wh));
    }
    a.V[o + h] = flux;
  }
}

// horizontal flux M q_e at edge-levels
template <bool TOPO>
__global__ void __launch_bounds__(256) k_tr_edge(TrArgs a) {
  const int64_t e = tr_warp();
  if (e >= a.ne) return;
  const int lane = threadIdx.x & 31, N = a.N, ld = a.ld;
  const int64_t o = e * ld;
  const int64_t c1 = (int64_t)a.e2c[2 * e] * ld, c2 = (int64_t)a.e2c[2 * e + 1] * ld;
  const double nx = a.n_e[3 * e], ny = a.n_e[3 * e + 1], nz = a.n_e[3 * e + 2];
  const double tx = a.t_e[3 * e], ty = a.t_e[3 * e + 1], tz = a.t_e[3 * e + 2];
  double r1[3], r2[3], wt[5];
  int64_t S[5];
  for (int j = 0; j < 3; ++j) {
    r1[j] = a.roff[6 * e + j];
    r2[j] = a.roff[6 * e + 3 + j];
  }
  for (int j = 0; j < 5; ++j) {
    S[j] = (int64_t)a.e2vt[5 * e + j] * ld;
    wt[j] = a.vt_w[5 * e + j];
  }
  const double hdt = 0.5 * a.dt;
  for (int k = lane; k < N; k += 32) {
    const double M = a.M[o + k];
    const bool up = M >= 0.0;
    const int64_t cd = (up ? c1 : c2) + k;
    double rho_e = 0.5 * (a.rho0[c1 + k] + a.rho0[c2 + k]);
    if constexpr (TOPO) rho_e *= a.t_dz_e[o + k];
    const double r = recip64(rho_e);
    double Mt = 0.0;
    for (int j = 0; j < 5; ++j) Mt += wt[j] * a.M[S[j] + k];
    const double vn = M * r, vt = Mt * r;
    const double ox = (up ? r1[0] : r2[0]) - hdt * (vn * nx + vt * tx);
    const double oy = (up ? r1[1] : r2[1]) - hdt * (vn * ny + vt * ty);
    const double oz = (up ? r1[2] : r2[2]) - hdt * (vn * nz + vt * tz);
    const double qe = a.q[cd] + ((a.gx[cd] * ox + a.gy[cd] * oy) + a.gz[cd] * oz);
    a.F[o + k] = M * qe;
  }
}

// flux-form update of the mixing ratio, in place
template <bool TOPO>
__global__ void __launch_bounds__(256) k_tr_update(TrArgs a) {
  const int64_t c = tr_warp();
  if (c >= a.nc) return;
  const int lane = threadIdx.x & 31, N = a.N, ld = a.ld;
  const int64_t o = c * ld;
  int64_t E[3];
  double dw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)a.c2e[3 * c + s] * ld;
    dw[s] = a.div_wa[3 * c + s];
  }
  bool bad = false;
  for (int k = lane; k < N; k += 32) {
    const double div = (dw[0] * a.F[E[0] + k] + dw[1] * a.F[E[1] + k]) + dw[2] * a.F[E[2] + k];
    double tend;
    if constexpr (TOPO) tend = (div + (a.V[o + k] - a.V[o + k + 1])) * a.t_inv_dz_c[o + k];
    else tend = div + (a.V[o + k] - a.V[o + k + 1]) * a.inv_dz[k];
    const double qn = (a.rho0[o + k] * a.q[o + k] - a.dt * tend) * recip64(a.rho1[o + k]);
    a.q[o + k] = qn;
    bad |= !tr_finite(qn);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, 1u);
}

// level-major [k][n] (nlev levels) -> [n][ld]
__global__ void k_tr_lm_to_rm(const double* __restrict__ a, double* __restrict__ b, int64_t n, int nlev, int ld) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nlev) return;
  const int64_t k = t / n, i = t % n;
  b[i * ld + k] = a[t];
}

}  // namespace

int tracer_alloc(icon_state* st, int ntracers) {
  icon_grid* grid = const_cast<icon_grid*>(st->grid);
  int rc = build_tracer_tables(grid, current_stream());
  if (rc != ICON_OK) return rc;
  StateDev& s = st->s;
  DeviceArena& A = st->arena;
  const size_t C = (size_t)grid->g.nc * grid->vert.ld, E = (size_t)grid->g.ne * grid->vert.ld;
  double* q = A.get_n<double>(C * ntracers);
  double* rho0 = A.get_n<double>(C);
  double* gx = A.get_n<double>(C);
  double* gy = A.get_n<double>(C);
  double* gz = A.get_n<double>(C);
  double* V = A.get_n<double>(C);
  double* F = A.get_n<double>(E);
  double *rho1 = nullptr, *W = nullptr;
  if (s.level_major) {
    rho1 = A.get_n<double>(C);
    W = A.get_n<double>(C);
  }
  if (A.failed) {
    set_error("out of device memory allocating %d tracers", ntracers);
    return ICON_ENOMEM;
  }
  cudaStream_t stream = current_stream();
  ICON_CUDA(cudaMemsetAsync(q, 0, sizeof(double) * C * ntracers, stream));
  ICON_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * C, stream));
  ICON_CUDA(cudaStreamSynchronize(stream));
  s.q = q; s.tr_rho0 = rho0; s.tr_gx = gx; s.tr_gy = gy; s.tr_gz = gz; s.tr_V = V; s.tr_F = F;
  s.tr_rho1 = rho1; s.tr_W = W;
  s.ntr = ntracers;
  return ICON_OK;
}

// before the substeps: keep the step's initial density in the [cell][level] layout
void tracer_begin(icon_state* st, cudaStream_t stream) {
  StateDev& s = st->s;
  const icon_grid* grid = st->grid;
  const int64_t nc = grid->g.nc;
  const int N = grid->vert.N, ld = grid->vert.ld;
  prof_begin(stream, K_TRACER);
  if (s.level_major)
    k_tr_lm_to_rm<<<blocks_for(nc * N, 256), 256, 0, stream>>>(s.rho, s.tr_rho0, nc, N, ld);
  else
    cudaMemcpyAsync(s.tr_rho0, s.rho, sizeof(double) * nc * ld, cudaMemcpyDeviceToDevice, stream);
  prof_end(stream);
}

// after the step: transport every tracer with the step's mean fluxes
void tracer_end(icon_state* st, double dt, cudaStream_t stream) {
  StateDev& s = st->s;
  const icon_grid* grid = st->grid;
  const GridDev& g = grid->g;
  const Vertical& v = grid->vert;
  const int64_t nc = g.nc;
  TrArgs a;
  a.nc = nc; a.ne = g.ne; a.N = v.N; a.ld = v.ld;
  a.c2e = g.c2e; a.e2c = g.e2c; a.c2c = g.c2c; a.e2vt = g.e2vt;
  a.lsq_c = g.lsq_c; a.roff = g.roff; a.n_e = g.n_e; a.t_e = g.t_e; a.vt_w = g.vt_w; a.div_wa = g.div_wa;
  a.inv_dz = v.d_inv_dz; a.wu = v.d_wu; a.wl = v.d_wl; a.lev = g.tr_lev;
  a.rho0 = s.tr_rho0;
  a.M = s.mflx;
  const TopoDev& T = s.topo;
  a.t_dz_c = T.dz_c; a.t_inv_dz_c = T.inv_dz_c; a.t_wu_c = T.wu_c; a.t_dz_e = T.dz_e;
  a.gx = s.tr_gx; a.gy = s.tr_gy; a.gz = s.tr_gz; a.V = s.tr_V; a.F = s.tr_F;
  a.status = s.status;
  a.dt = dt;
  prof_begin(stream, K_TRACER);
  if (s.level_major) {
    k_tr_lm_to_rm<<<blocks_for(nc * v.N, 256), 256, 0, stream>>>(s.rho, s.tr_rho1, nc, v.N, v.ld);
    k_tr_lm_to_rm<<<blocks_for(nc * (v.N + 1), 256), 256, 0, stream>>>(s.wflx, s.tr_W, nc, v.N + 1, v.ld);
    a.rho1 = s.tr_rho1;
    a.W = s.tr_W;
  } else {
    a.rho1 = s.rho;
    a.W = s.wflx;
  }
  const unsigned nbc = blocks_for(nc, kTrWarps), nbe = blocks_for(g.ne, kTrWarps);
  for (int t = 0; t < s.ntr; ++t) {
    a.q = s.q + (size_t)t * nc * v.ld;
    if (T.on) {
      k_tr_cell<true><<<nbc, 256, 0, stream>>>(a);
      k_tr_edge<true><<<nbe, 256, 0, stream>>>(a);
      k_tr_update<true><<<nbc, 256, 0, stream>>>(a);
    } else {
      k_tr_cell<false><<<nbc, 256, 0, stream>>>(a);
      k_tr_edge<false><<<nbe, 256, 0, stream>>>(a);
      k_tr_update<false><<<nbc, 256, 0, stream>>>(a);
    }
  }
  prof_end(stream);
}

}  // namespace icon
