// FP64 dynamical-core step ("plain method"): predictor-corrector substeps with
// a vertically implicit w/Exner column solve, then Smagorinsky diffusion.
//
// The paper states that ICON's dynamical core is a nonhydrostatic solver on the
// icosahedral-triangular C grid (Sec. "Current State of the Art"), that it is
// memory-bandwidth bound and dominated by index lookups on triangles, hexagons
// and 12 pentagons (Sec. "Separation of Concerns"), and that all data stay on
// the GPU (Sec. "Innovations Realized"). It gives no discretisation; the one
// computed here, on fields stored level-contiguous ([entity][ld], full level k =
// 0..N-1 top to bottom, half level h = 0..N with w = 0 at h = 0 and h = N), is:
//
//   O1 gradient   (psi_c2 - psi_c1) / d_e
//   O2 divergence (1/A_c) sum_e s_ce l_e u_e
//   O3 curl       (1/A_v) sum_e s_ve d_e vn_e           (counter-clockwise about v)
//   O4 vt         sum_j W_ej vn_j over 5 edges (Perot)
//   O5 K_c        sum_e kappa_ce (vn^2 + vt^2)/2
//   A_vn = -(K_c2 - K_c1)/d_e + ((zeta_v1 + zeta_v2)/2 + f_e) vt - wbar_e dvn/dz
//   A_w  = -sum_e kappa_ce [vn_ie dw/dn + vt_ie dw_v/dt] - w (w_{h-1} - w_{h+1})/(z_{h-1} - z_{h+1})
//   predictor vn* = vn + dtau (A_vn - cpd thv_e dpi/dn), column(S^n, vn*, A_w)
//   corrector vn' = vn + dtau ((A_vn0 + A_vn*)/2 - cpd thv_e* dpi*/dn),
//             column(S^n, vn', (A_w0 + A_w*)/2) with fluxes from S*
//   column: explicit predictors of rho, rho*theta_v, Exner, w with off-centring
//   beta = 0.65, tridiagonal system in w at interior half levels (Thomas,
//   no pivoting), Rayleigh damping, then back-substituted rho, Theta, Exner.
//   diffusion: K_h = cs^2 l d sqrt(D_T^2 + D_S^2) from least-squares vertex
//   velocities, vn += dt K_h L(vn), flux-form theta_v diffusion, Exner adjusted
//   at constant density.
//
// Mapping: one warp per entity (edge, cell or vertex) with lanes over levels, so
// every neighbour index is loaded once per entity and every gathered neighbour
// row is a coalesced, aligned segment; the implicit column solve runs its
// level-parallel parts the same way and only its Thomas recurrence one thread per
// column (see "column solve" below). The summation order of every stencil follows
// the operator definitions (fixed neighbour order), so results do not depend on the
// launch shape.
// FP64 division issues about eight FP64-pipe instructions on this GPU, so every
// division by a geometric or per-level constant is a multiplication by a
// precomputed reciprocal (area factors folded into the stencil weights); the
// column's three quotients per level (pi/Theta, the Thomas pivot, Theta/rho) use
// the Newton-Raphson reciprocal of recip64.h.
#include <cmath>
#include "icon_internal.h"
#include "recip64.h"

namespace icon {
namespace {

constexpr int kWarpsPerBlock = 8;

struct Geo64 {
  int64_t nc, ne, nv;
  int N, ld;
  const int *c2e, *e2c, *e2v, *v2e, *v2c, *vdeg, *e2vt, *e2q;
  const double *div_wa, *rot_wa, *inv_Ac, *vt_w, *kin_w, *lsq_w, *inv_de, *inv_le, *l_e, *d_e, *f_e, *inv_L34;
  const double *n_e, *t_e, *s_ce;
  const double *wu, *wl, *inv_dz, *inv_dz2, *qinv_dz;
  const double* cc;                        // per-level constants for the current dtau
  const double *kin_w_h, *div_wa_h;        // half the cell weights (state tables, [Nc][3])
  // terrain-following levels (the TOPO kernel variants; see terrain.cu): per-edge normal
  // slope factor, full-level decay, per-entity tables [entity][ld], and the stage's
  // contravariant correction, contravariant velocity, Exner perturbation and half its
  // vertical derivative
  const double *t_sn, *t_bf, *t_wu_e, *t_qinv_dz_e, *t_dz_e;
  const double *t_wu_c, *t_inv_dz_c, *t_inv_dzh_c, *t_wcc, *t_wcon, *t_ep, *t_hdpdz;
};

// per-level constants of the column solve for one dtau, [8][ld] (same layout as the
// mixed path): wu, wl, dtau beta cpd / dzh, (1 - beta) cpd / dzh, 1/(1 + dtau r),
// dtau beta / dz, dtau (1 - beta) / dz, unused
enum { C_WU = 0, C_WL, C_CA, C_CX, C_DAMP, C_DTBDZ, C_DT1BDZ, C_COUNT };

__global__ void k_colconst64(int N, int ld, const double* __restrict__ wu, const double* __restrict__ wl,
                             const double* __restrict__ dzh, const double* __restrict__ dz,
                             const double* __restrict__ ray, double dtau, double* __restrict__ cc) {
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    const bool interior = i > 0 && i < N;
    cc[C_WU * ld + i] = i <= N ? wu[i] : 0.0;
    cc[C_WL * ld + i] = i <= N ? wl[i] : 0.0;
    cc[C_CA * ld + i] = interior ? dtau * kBeta * kCpd / dzh[i] : 0.0;
    cc[C_CX * ld + i] = interior ? (1.0 - kBeta) * kCpd / dzh[i] : 0.0;
    cc[C_DAMP * ld + i] = i <= N ? 1.0 / (1.0 + dtau * ray[i]) : 1.0;
    cc[C_DTBDZ * ld + i] = i < N ? dtau * kBeta / dz[i] : 0.0;
    cc[C_DT1BDZ * ld + i] = i < N ? dtau * (1.0 - kBeta) / dz[i] : 0.0;
  }
}

// finiteness from the exponent bits (integer pipe; a floating-point compare would
// take an FP64-pipe slot)
__device__ inline bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// The warp-per-entity FP64 kernels are held to 64 registers (4 blocks of 8 warps per SM):
// they are bound by the FP64 pipe, and the extra warps hide more load latency than the few
// spilled registers of the rows kernel cost (R2B6/90 step 97.5 -> 94.4 ms).
__device__ inline int64_t warp_entity() {
  return (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
}

// zeta_v (full levels) and w_v (half levels)
__global__ void __launch_bounds__(256, 4) k_vertex(Geo64 G, const double* __restrict__ vn, const double* __restrict__ w,
                                                double* __restrict__ zeta, double* __restrict__ w_v) {
  const int64_t v = warp_entity();
  if (v >= G.nv) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[6], C[6];
  double rw[6];
  for (int j = 0; j < 6; ++j) {
    E[j] = (int64_t)G.v2e[6 * v + j] * ld;
    C[j] = (int64_t)G.v2c[6 * v + j] * ld;
    rw[j] = G.rot_wa[6 * v + j];
  }
  const int deg = G.vdeg[v];
  const double inv_deg = deg == 6 ? 1.0 / 6.0 : 1.0 / 5.0;
  for (int k = lane; k < G.N; k += 32) {
    double acc = 0.0;
    for (int j = 0; j < 6; ++j) acc += rw[j] * vn[E[j] + k];
    zeta[v * ld + k] = acc;
  }
  for (int h = lane; h <= G.N; h += 32) {
    double acc = 0.0;
    for (int j = 0; j < 5; ++j) acc += w[C[j] + h];
    acc += (deg == 6) ? w[C[5] + h] : 0.0;
    w_v[v * ld + h] = acc * inv_deg;
  }
}

// vt (Perot) and 2 K_e = vn^2 + vt^2 at edges (the 1/2 is folded into k_cell_ke's weights)
__global__ void __launch_bounds__(256) k_edge_vt(Geo64 G, const double* __restrict__ vn, double* __restrict__ vt,
                                                 double* __restrict__ Ke) {
  const int64_t e = warp_entity();
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t S[5];
  double W[5];
  for (int j = 0; j < 5; ++j) {
    S[j] = (int64_t)G.e2vt[5 * e + j] * ld;
    W[j] = G.vt_w[5 * e + j];
  }
  for (int k = lane; k < G.N; k += 32) {
    double acc = 0.0;
    for (int j = 0; j < 5; ++j) acc += W[j] * vn[S[j] + k];
    const double v0 = vn[e * ld + k];
    vt[e * ld + k] = acc;
    Ke[e * ld + k] = fma(v0, v0, acc * acc);
  }
}

// K_c at cells (from 2 K_e)
__global__ void __launch_bounds__(256) k_cell_ke(Geo64 G, const double* __restrict__ Ke, double* __restrict__ Kc) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[3];
  double kw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    kw[s] = G.kin_w_h[3 * c + s];
  }
  for (int k = lane; k < G.N; k += 32) {
    double acc = 0.0;
    for (int s = 0; s < 3; ++s) acc += kw[s] * Ke[E[s] + k];
    Kc[c * ld + k] = acc;
  }
}

struct EdgeArgs {
  const double *vn, *w, *rho, *thv, *ex;   // stage state (S^n or S*)
  const double *vt, *Kc, *zeta, *w_v;      // diagnostics of the stage state
  const double* vn_base;                   // vn^n
  double* vn_out;                          // vn* or vn^{n+1} (may alias vn_base)
  double* Avn0;                            // stored (predictor) or read (corrector)
  double *F, *G, *a_e, *mflx;
  double dtau, inv_nsub;
  double hinv_nsub;                        // inv_nsub / 2 (set on the host)
  double hdtau;                            // dtau / 2 (set on the host)
  int corrector;
  int skip_flux;                           // fluxes formed after divergence damping instead
  int upwind_theta;                        // heat flux with the upwind theta_v (option)
};

// vn tendency and update, horizontal mass/heat fluxes, edge part of w advection.
// FP64-pipe bound, so the kernel minimises FP64 warp instructions: one pass over the
// half levels in windows of 31 (lane l of a window holds half level h = base + l and,
// for l < 31, full level k = h), each half-level interpolant and cell-pair sum formed
// once and handed to the lane below with a shuffle, factors of 1/2 folded into
// exactly-scaled constants, and the per-edge constants cpd / d_e hoisted.
//
// TOPO (terrain-following levels): per-edge interpolation weights, the contravariant
// vertical velocity w - wcc (zero at lid and ground) in the vertical advection of vn,
// the metric correction of the pressure gradient on pi' = pi - pi_ref,
//   (pi'_c2 - pi'_c1)/d_e - sn_e bf_k (d pi'/dz at c1 and c2)/2,
// and mass fluxes through layers of thickness dz_e; w - wcc, pi' and d pi'/dz come from
// the stage's k_topo_cell.
template <bool TOPO, bool UT>
__global__ void __launch_bounds__(256, 4) k_edge_tend(Geo64 G, EdgeArgs a) {
  const int64_t e = warp_entity();
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld, N = G.N;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld;
  const int64_t v1 = (int64_t)G.e2v[2 * e] * ld, v2 = (int64_t)G.e2v[2 * e + 1] * ld;
  const int64_t eo = e * ld;
  const double ide = G.inv_de[e], ile = G.inv_le[e], fe = G.f_e[e];
  // the factors 1/2 of theta_e = (t1 + t2)/2 and rho_e = (rho1 + rho2)/2 are folded into
  // these constants (and the column's divergence weights), exact scalings by powers of two
  const double hcide = 0.5 * (kCpd * ide);
  const double hcsne = TOPO ? 0.5 * (kCpd * G.t_sn[e]) : 0.0;
  // flat levels: the pressure-gradient term enters vn through one multiply-add with
  // -dtau cpd / (2 d_e), and the advective part through dtau (predictor) or dtau / 2
  const double ndhcide = -(a.dtau * hcide);
  const double hinv_nsub = a.hinv_nsub;
  const double* __restrict__ vn = a.vn + eo;
  const double* __restrict__ vt = a.vt + eo;
  const double dtau = a.dtau;
  for (int base = 0; base <= N; base += 31) {
    const int h = base + lane;
    const bool hv = h <= N;                    // a half level of this column
    const bool kv = lane < 31 && h < N;        // a full level owned by this lane
    // half-level interpolation weights: f(0) = f[0], f(N) = f[N-1], linear between
    const int hl = h > 0 ? (h - 1 < N - 1 ? h - 1 : N - 1) : 0;
    const int hu = h < N ? h : N - 1;
    double wa, wb;
    if (TOPO) {
      wa = (h == 0) ? 0.0 : (h >= N ? 1.0 : G.t_wu_e[eo + h]);
      wb = (h == 0) ? 1.0 : (h >= N ? 0.0 : 1.0 - wa);
    } else {
      wa = (h == 0) ? 0.0 : (h >= N ? 1.0 : G.wu[h]);
      wb = (h == 0) ? 1.0 : (h >= N ? 0.0 : G.wl[h]);
    }
    double vie = 0.0, tie = 0.0, sw = 0.0, dw = 0.0, dwv = 0.0;
    if (hv) {
      vie = wa * vn[hl] + wb * vn[hu];
      tie = wa * vt[hl] + wb * vt[hu];
      const double w1 = a.w[c1 + h], w2 = a.w[c2 + h];
      if (TOPO)
        sw = G.t_wcon[c1 + h] + G.t_wcon[c2 + h];        // 0 at the lid and the ground
      else
        sw = w1 + w2;
      dw = w2 - w1;
      dwv = a.w_v[v2 + h] - a.w_v[v1 + h];
    }
    const double vie_up = __shfl_down_sync(0xffffffffu, vie, 1);   // half level h + 1
    const double sw_up = __shfl_down_sync(0xffffffffu, sw, 1);
    if (hv && lane < 31) a.a_e[eo + h] = (vie * dw) * ide + (tie * dwv) * ile;
    if (kv) {
      const int k = h;
      // advective tendency: -grad K + (zeta + f) vt - wbar dvn/dz, with
      // wbar = (sum of the four w) / 4 and the 1/4 folded into the level constant
      const double zs = a.zeta[v1 + k] + a.zeta[v2 + k];
      const double dK = a.Kc[c2 + k] - a.Kc[c1 + k];
      const double T = fma(-dK, ide, fma(0.5, zs, fe) * vt[k]);
      const double A = fma(-((sw + sw_up) * (vie - vie_up)), TOPO ? G.t_qinv_dz_e[eo + k] : G.qinv_dz[k], T);
      const double t1 = a.thv[c1 + k], t2 = a.thv[c2 + k];
      const double th_s = t1 + t2;                     // 2 theta_e
      double vnew;
      if (TOPO) {
        const double corr = (hcsne * G.t_bf[k]) * (G.t_hdpdz[c1 + k] + G.t_hdpdz[c2 + k]);
        const double pg = th_s * fma(G.t_ep[c2 + k] - G.t_ep[c1 + k], hcide, -corr);
        if (a.corrector) {
          vnew = fma(dtau, fma(0.5, a.Avn0[eo + k] + A, -pg), a.vn_base[eo + k]);
        } else {
          vnew = fma(dtau, A - pg, a.vn_base[eo + k]);
          a.Avn0[eo + k] = A;
        }
      } else {
        const double tdx = th_s * (a.ex[c2 + k] - a.ex[c1 + k]);
        if (a.corrector) {
          vnew = fma(ndhcide, tdx, fma(a.hdtau, a.Avn0[eo + k] + A, a.vn_base[eo + k]));
        } else {
          vnew = fma(ndhcide, tdx, fma(dtau, A, a.vn_base[eo + k]));
          a.Avn0[eo + k] = A;
        }
      }
      a.vn_out[eo + k] = vnew;
      if (a.skip_flux) continue;
      // F = 2 rho_e vn and G = 4 rho_e vn theta_e (exactly; the column weights carry 1/2)
      double F = (a.rho[c1 + k] + a.rho[c2 + k]) * vnew;
      if (TOPO) F *= G.t_dz_e[eo + k];
      a.F[eo + k] = F;
      if constexpr (UT) a.G[eo + k] = F * (2.0 * (vnew >= 0.0 ? t1 : t2));     // upwind theta_v (option)
      else a.G[eo + k] = F * th_s;
      if (a.corrector) a.mflx[eo + k] = fma(F, hinv_nsub, a.mflx[eo + k]);
    }
  }
}

// ---------------------------------------------------------------- divergence damping (option)
// Fourth-order divergence damping of the corrector's vn^{n+1} before its fluxes are formed:
// vn -= c4 Abar^2 grad(div(grad(div vn))), Abar the mean cell area (an ICON option; the
// paper prints none). Cell divergence, cell Laplacian of it, then the edge update together
// with the corrector's mass and heat fluxes and the step-mean mass flux.
__global__ void __launch_bounds__(256, 4) k_dd_div(Geo64 G, const double* __restrict__ vn, double* __restrict__ D) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[3];
  double dw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    dw[s] = G.div_wa[3 * c + s];
  }
  for (int k = lane; k < G.N; k += 32) D[c * ld + k] = (dw[0] * vn[E[0] + k] + dw[1] * vn[E[1] + k]) + dw[2] * vn[E[2] + k];
}

__global__ void __launch_bounds__(256, 4) k_dd_lap(Geo64 G, const double* __restrict__ D, double* __restrict__ L) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t A[3], B[3];
  double wt[3];
  for (int s = 0; s < 3; ++s) {
    const int e = G.c2e[3 * c + s];
    A[s] = (int64_t)G.e2c[2 * e] * ld;
    B[s] = (int64_t)G.e2c[2 * e + 1] * ld;
    wt[s] = G.div_wa[3 * c + s] * G.inv_de[e];
  }
  for (int k = lane; k < G.N; k += 32)
    L[c * ld + k] = (wt[0] * (D[B[0] + k] - D[A[0] + k]) + wt[1] * (D[B[1] + k] - D[A[1] + k])) +
                    wt[2] * (D[B[2] + k] - D[A[2] + k]);
}

struct DDArgs {
  const double *L, *rho, *thv;             // Laplacian of the divergence, stage state S*
  double *vn, *F, *G, *mflx;
  const double* dz_e;                      // layer thickness at edges (terrain-following), or NULL
  double scale, inv_nsub;                  // c4 Abar^2
  int upwind_theta;
};

__global__ void __launch_bounds__(256, 4) k_dd_edge(Geo64 G, DDArgs a) {
  const int64_t e = warp_entity();
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld, eo = e * ld;
  const double s = a.scale * G.inv_de[e];
  for (int k = lane; k < G.N; k += 32) {
    const double vn = a.vn[eo + k] - s * (a.L[c2 + k] - a.L[c1 + k]);
    a.vn[eo + k] = vn;
    double F = (a.rho[c1 + k] + a.rho[c2 + k]) * vn;      // 2 rho_e vn, as k_edge_tend
    if (a.dz_e) F *= a.dz_e[eo + k];
    a.F[eo + k] = F;
    const double t1 = a.thv[c1 + k], t2 = a.thv[c2 + k];
    a.G[eo + k] = F * (a.upwind_theta ? (vn >= 0.0 ? t1 + t1 : t2 + t2) : t1 + t2);
    a.mflx[eo + k] = fma(F, 0.5 * a.inv_nsub, a.mflx[eo + k]);
  }
}

// ---------------------------------------------------------------- column solve
//
// The vertically implicit update of every column in three launches:
//   k_col_rows   one warp per cell, lanes over levels: everything that is parallel
//                over the levels (half-level interpolants, horizontal divergences,
//                explicit predictors, the linearised state equation, the w predictor
//                and, in the predictor, the tridiagonal row of every interior half
//                level, which depends on S^n only and serves both stages). Rows go out
//                level-major for the solve; the operands of the final update stay in
//                the cell's own rows.
//   k_col_thomas one thread per column: the Thomas recurrence on level-major rows
//                (coalesced across the warp; the corrector substitutes with the
//                predictor's factors), Rayleigh damping; the solution w goes to ws.
//   k_col_update one warp per cell, lanes over levels: the implicit parts of rho,
//                Theta and pi, theta_v = Theta / rho, the step-mean vertical mass flux.
// Only the recurrence is sequential in the level; keeping it apart lets the rest run
// with coalesced, level-contiguous loads instead of one thread walking a column.
struct ColArgs {
  const double *rho, *thv, *ex, *w;        // S^n [c][ld]
  const double* w_stage;                   // w of the stage state (vertical part of A_w)
  const double *F, *G, *a_e;               // edge fluxes and w-advection edge terms
  double* Aw0;                             // stored (predictor) or read (corrector)
  double *lo, *di, *up, *rh;               // tridiagonal rows, level-major [h][Nc], h = 1..N-1
  double* ws;                              // the damped solution w^{n+1}, level-major [h][Nc]
  double *rx, *tx, *px, *gm;               // rho*, Theta*, pi* (explicit parts), gamma: [c][ld]
  double* gc;                              // (Rd/cvd) pi / Theta of S^n: [c][ld]
  double *ri, *mm;                         // half-level rho and rho theta_v of S^n: [c][ld]
  double *rho_o, *thv_o, *ex_o, *w_o;      // S* or S^{n+1} (may alias S^n)
  double* wflx;
  unsigned* status;
  double dtau, inv_nsub;
  double hdtau;                            // dtau / 2 (set on the host: a kernel would recompute it per use)
  double b_new, b_old;                     // beta / nsub, (1 - beta) / nsub
  int corrector;
};

// windows of 31 levels: lane l holds full level k = base + l and the half level above
// it (h = k); lane 31 only supplies the half level below lane 30's full level.
// TOPO (terrain-following levels): each cell's own spacings and interpolation weights,
// thickness-weighted horizontal fluxes (already carrying dz_e) divided by the cell's dz,
// the explicit vertical fluxes with the contravariant (1 - beta) w - wcc, and the
// vertical advection of w with w - wcc.
template <bool TOPO>
__global__ void __launch_bounds__(256, 4) k_col_rows(Geo64 G, ColArgs a) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld, N = G.N;
  const int64_t o = c * ld, nc = G.nc;
  const double* __restrict__ cc = G.cc;
  int64_t E[3];
  double dw[3], kw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    dw[s] = G.div_wa_h[3 * c + s];         // the edge fluxes are 2 rho_e vn and 4 rho_e vn theta_e
    kw[s] = G.kin_w[3 * c + s];
  }
  const double dtau = a.dtau, hdtau = a.hdtau, rcv = kRd / kCvd;
  double gam_c = 0.0, px_c = 0.0, M_c = 0.0;          // carried: full / half level base - 1
  for (int base = 0; base <= N; base += 31) {
    const int k = base + lane;
    const bool hv = k <= N;                            // half level k exists
    const bool kv = lane < 31 && k < N;                // full level k owned here
    double rho = 0.0, thv = 0.0, ex = 0.0, rho_m = 0.0, thv_m = 0.0, ex_m = 0.0;
    if (k < N) { rho = a.rho[o + k]; thv = a.thv[o + k]; ex = a.ex[o + k]; }
    if (k >= 1 && k <= N) { rho_m = a.rho[o + k - 1]; thv_m = a.thv[o + k - 1]; ex_m = a.ex[o + k - 1]; }
    // half-level interpolants of S^n: rho_ic and M = rho_ic theta_ic
    double ri = 0.0, ti = 0.0;
    if (k == 0) { ri = rho; ti = thv; }
    else if (k == N) { ri = rho_m; ti = thv_m; }
    else if (k < N) {
      if constexpr (TOPO) {
        const double wu = G.t_wu_c[o + k], wl = 1.0 - wu;
        ri = wu * rho_m + wl * rho;
        ti = wu * thv_m + wl * thv;
      } else {
        const double wu = cc[C_WU * ld + k], wl = cc[C_WL * ld + k];
        ri = wu * rho_m + wl * rho;
        ti = wu * thv_m + wl * thv;
      }
    }
    const double M = ri * ti;
    const double wk = hv ? a.w[o + k] : 0.0;
    // TOPO: explicit part of the contravariant velocity at interior half levels
    const double ve = (TOPO && k >= 1 && k < N) ? (1.0 - kBeta) * wk - G.t_wcc[o + k] : 0.0;
    const double ri1 = __shfl_down_sync(0xffffffffu, ri, 1);      // half level k + 1
    const double M1 = __shfl_down_sync(0xffffffffu, M, 1);
    const double w1 = __shfl_down_sync(0xffffffffu, wk, 1);
    double ve1 = 0.0;
    if constexpr (TOPO) ve1 = __shfl_down_sync(0xffffffffu, ve, 1);
    double gam = 0.0, px = 0.0;
    if (kv) {
      // explicit predictors at full level k
      // Dr: the mass-flux divergence; Dt2: twice the heat-flux divergence
      double Dr = 0.0, Dt2 = 0.0;
      for (int s = 0; s < 3; ++s) Dr += dw[s] * a.F[E[s] + k];
      for (int s = 0; s < 3; ++s) Dt2 += dw[s] * a.G[E[s] + k];
      const double Th = rho * thv;
      double rx, tx;
      if constexpr (TOPO) {
        const double idz = G.t_inv_dz_c[o + k];
        rx = rho - (dtau * ((Dr + ri * ve) - ri1 * ve1)) * idz;
        tx = Th - (dtau * ((0.5 * Dt2 + M * ve) - M1 * ve1)) * idz;
      } else {
        const double dt1 = cc[C_DT1BDZ * ld + k];
        rx = (rho - dtau * Dr) - dt1 * (ri * wk - ri1 * w1);
        tx = (Th - hdtau * Dt2) - dt1 * (M * wk - M1 * w1);
      }
      // the state-equation factor of S^n: formed by the predictor, read back by the corrector
      double g;
      if (!a.corrector) {
        g = (rcv * ex) * recip64(Th);
        a.gc[o + k] = g;
      } else {
        g = a.gc[o + k];
      }
      px = ex + g * (tx - Th);
      a.rx[o + k] = rx;
      a.tx[o + k] = tx;
      a.px[o + k] = px;
      if (!a.corrector) {
        if constexpr (TOPO) gam = g * (dtau * kBeta * G.t_inv_dz_c[o + k]);
        else gam = g * cc[C_DTBDZ * ld + k];
        a.gm[o + k] = gam;
      }
    }
    if (hv && lane < 31 && !a.corrector) {
      a.ri[o + k] = ri;
      a.mm[o + k] = M;
    }
    // full level and half level above: from the lane above, or carried for lane 0
    double gam_m = __shfl_up_sync(0xffffffffu, gam, 1);
    double px_m = __shfl_up_sync(0xffffffffu, px, 1);
    double M_m = __shfl_up_sync(0xffffffffu, M, 1);
    if (lane == 0) { gam_m = gam_c; px_m = px_c; M_m = M_c; }
    if (kv && k >= 1) {
      // row of interior half level h = k: w predictor and the implicit coupling
      const int h = k;
      double hadv = 0.0;
      for (int s = 0; s < 3; ++s) hadv += kw[s] * a.a_e[E[s] + h];
      const double ws = a.w_stage[o + h];
      double Aw;
      if constexpr (TOPO)
        Aw = -hadv - G.t_wcon[o + h] * (a.w_stage[o + h - 1] - a.w_stage[o + h + 1]) * (0.5 * G.t_inv_dzh_c[o + h]);
      else
        Aw = -hadv - ws * (a.w_stage[o + h - 1] - a.w_stage[o + h + 1]) * G.inv_dz2[h];
      if (a.corrector) Aw = 0.5 * (a.Aw0[o + h] + Aw);
      else a.Aw0[o + h] = Aw;
      const double th_ic = ti;
      double w_x, aa;
      if constexpr (TOPO) {
        const double idzh = G.t_inv_dzh_c[o + h];
        w_x = wk + dtau * ((Aw - ((1.0 - kBeta) * kCpd * idzh) * th_ic * (ex_m - ex)) - kGrav);
        aa = (dtau * kBeta * kCpd * idzh) * th_ic;
      } else {
        w_x = wk + dtau * ((Aw - cc[C_CX * ld + h] * th_ic * (ex_m - ex)) - kGrav);
        aa = cc[C_CA * ld + h] * th_ic;
      }
      const int64_t i = (int64_t)h * nc + c;
      if (!a.corrector) {
        const double P = aa * gam_m, Q = aa * gam;
        a.lo[i] = -P * M_m;
        a.di[i] = fma(P + Q, M, 1.0);
        a.up[i] = -Q * M1;
      }
      a.rh[i] = w_x - aa * (px_m - px);
    }
    gam_c = __shfl_sync(0xffffffffu, gam, 30);
    px_c = __shfl_sync(0xffffffffu, px, 30);
    M_c = __shfl_sync(0xffffffffu, M, 30);
  }
}

// Thomas recurrence per column on the level-major rows; the next row is loaded before
// the current one is stored so that its loads overlap the recurrence. The matrix depends on
// S^n only (rho_ic, theta_ic and the state-equation factor of the substep's start), so it is
// the same in both stages: the predictor factors it, keeping the sub-diagonal, storing
// 1 / pivot over the diagonal and up / pivot over the super-diagonal, and the corrector only
// substitutes its own right-hand side (the same operations on the same values as a second
// factorisation, so the results are unchanged). The damped solution goes to ws.
__global__ void __launch_bounds__(128) k_col_thomas(Geo64 G, ColArgs a) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= G.nc) return;
  const int N = G.N, ld = G.ld;
  if (N < 2) return;
  const int64_t nc = G.nc;
  const double* __restrict__ cc = G.cc;
  const double* __restrict__ lo = a.lo;
  double* __restrict__ di = a.di;
  double* __restrict__ up = a.up;
  double* __restrict__ rh = a.rh;
  double* __restrict__ ws = a.ws;
  double dp = 0.0;
  if (!a.corrector) {
    double cp = 0.0;
    double l = lo[nc + c], d = di[nc + c], u = up[nc + c], r = rh[nc + c];
    for (int h = 1; h < N; ++h) {
      double ln = 0.0, dn = 0.0, un = 0.0, rn = 0.0;
      if (h + 1 < N) {
        const int64_t j = (int64_t)(h + 1) * nc + c;
        ln = lo[j]; dn = di[j]; un = up[j]; rn = rh[j];
      }
      const double q = recip64(h == 1 ? d : d - l * cp);
      cp = u * q;
      dp = (h == 1 ? r : r - l * dp) * q;
      const int64_t i = (int64_t)h * nc + c;
      di[i] = q;
      up[i] = cp;
      rh[i] = dp;
      l = ln; d = dn; u = un; r = rn;
    }
  } else {
    double l = lo[nc + c], q = di[nc + c], r = rh[nc + c];
    for (int h = 1; h < N; ++h) {
      double ln = 0.0, qn = 0.0, rn = 0.0;
      if (h + 1 < N) {
        const int64_t j = (int64_t)(h + 1) * nc + c;
        ln = lo[j]; qn = di[j]; rn = rh[j];
      }
      dp = (h == 1 ? r : r - l * dp) * q;
      rh[(int64_t)h * nc + c] = dp;
      l = ln; q = qn; r = rn;
    }
  }
  // back substitution
  double x = dp;
  ws[(int64_t)(N - 1) * nc + c] = x * cc[C_DAMP * ld + N - 1];
  for (int h = N - 2; h >= 1; --h) {
    const int64_t i = (int64_t)h * nc + c;
    x = rh[i] - up[i] * x;
    ws[i] = x * cc[C_DAMP * ld + h];
  }
}

// TOPO: each cell's dz, the contravariant step-mean vertical flux, and the ground w of
// the stage (its wcc, so that w - wcc = 0 there)
template <bool TOPO>
__global__ void __launch_bounds__(256) k_col_update(Geo64 G, ColArgs a) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld, N = G.N;
  const int64_t o = c * ld, nc = G.nc;
  const double* __restrict__ cc = G.cc;
  bool bad = false;
  for (int base = 0; base < N; base += 31) {
    const int k = base + lane;
    // w^{n+1} (damped) at half level k; zero at the top and the bottom
    const double wn = (k >= 1 && k < N) ? a.ws[(int64_t)k * nc + c] : 0.0;
    const double ri = k <= N ? a.ri[o + k] : 0.0;
    const double M = k <= N ? a.mm[o + k] : 0.0;
    const double wn1 = __shfl_down_sync(0xffffffffu, wn, 1);
    const double ri1 = __shfl_down_sync(0xffffffffu, ri, 1);
    const double M1 = __shfl_down_sync(0xffffffffu, M, 1);
    if (lane < 31 && k < N) {
      const double q = M * wn - M1 * wn1;
      const double r = ri * wn - ri1 * wn1;
      const double dtb = TOPO ? a.dtau * kBeta * G.t_inv_dz_c[o + k] : cc[C_DTBDZ * ld + k];
      const double Th_n = a.tx[o + k] - dtb * q;
      const double ex_n = a.px[o + k] - a.gm[o + k] * q;
      const double rho_n = a.rx[o + k] - dtb * r;
      const double thv_n = Th_n * recip64(rho_n);
      if (a.corrector) {
        // (beta wn + (1 - beta) wold - wcc) / nsub with the weights divided on the host
        const double wold = a.w[o + k];
        double wc = fma(a.b_new, wn, a.b_old * wold);
        if (TOPO) wc = fma(-a.inv_nsub, G.t_wcc[o + k], wc);
        a.wflx[o + k] = fma(ri, wc, a.wflx[o + k]);
      }
      a.rho_o[o + k] = rho_n;
      a.thv_o[o + k] = thv_n;
      a.ex_o[o + k] = ex_n;
      a.w_o[o + k] = wn;
      bad |= !finite_bits(thv_n) || !finite_bits(wn) || !finite_bits(ex_n);
    }
  }
  if (lane == 0) a.w_o[o + N] = TOPO ? G.t_wcc[o + N] : 0.0;
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, 1u);
}

// ---------------------------------------------------------------- diffusion
__global__ void __launch_bounds__(256, 4) k_diff_vertex(Geo64 G, const double* __restrict__ vn, double* __restrict__ ux,
                                                     double* __restrict__ uy, double* __restrict__ uz,
                                                     double* __restrict__ zeta) {
  const int64_t v = warp_entity();
  if (v >= G.nv) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[6];
  for (int j = 0; j < 6; ++j) E[j] = (int64_t)G.v2e[6 * v + j] * ld;
  const double* lw = G.lsq_w + 18 * v;
  const double* rw = G.rot_wa + 6 * v;
  for (int k = lane; k < G.N; k += 32) {
    double x = 0.0, y = 0.0, z = 0.0, r = 0.0;
    for (int j = 0; j < 6; ++j) {
      const double q = vn[E[j] + k];
      x += lw[3 * j] * q;
      y += lw[3 * j + 1] * q;
      z += lw[3 * j + 2] * q;
      r += rw[j] * q;
    }
    ux[v * ld + k] = x;
    uy[v * ld + k] = y;
    uz[v * ld + k] = z;
    zeta[v * ld + k] = r;
  }
}

__global__ void __launch_bounds__(256) k_diff_div(Geo64 G, const double* __restrict__ vn, double* __restrict__ divc) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[3];
  double dw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    dw[s] = G.div_wa[3 * c + s];
  }
  for (int k = lane; k < G.N; k += 32) {
    double acc = 0.0;
    for (int s = 0; s < 3; ++s) acc += dw[s] * vn[E[s] + k];
    divc[c * ld + k] = acc;
  }
}

__device__ inline double dot3(double ax, double ay, double az, const double* b) {
  return (ax * b[0] + ay * b[1]) + az * b[2];
}

// fourth-order background diffusion (option): L1 = L(vn) at edges, then the divergence
// and curl of L1 for the second Laplacian in k_diff_edge
__global__ void __launch_bounds__(256, 4) k_bd_lap(Geo64 G, const double* __restrict__ zeta,
                                                const double* __restrict__ divc, double* __restrict__ L1) {
  const int64_t e = warp_entity();
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld;
  const int64_t v1 = (int64_t)G.e2v[2 * e] * ld, v2 = (int64_t)G.e2v[2 * e + 1] * ld;
  const double ile = G.inv_le[e], ide = G.inv_de[e];
  for (int k = lane; k < G.N; k += 32)
    L1[e * ld + k] = (divc[c2 + k] - divc[c1 + k]) * ide - (zeta[v2 + k] - zeta[v1 + k]) * ile;
}

__global__ void __launch_bounds__(256, 4) k_bd_curl(Geo64 G, const double* __restrict__ L1, double* __restrict__ zeta1) {
  const int64_t v = warp_entity();
  if (v >= G.nv) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[6];
  double rw[6];
  for (int j = 0; j < 6; ++j) {
    E[j] = (int64_t)G.v2e[6 * v + j] * ld;
    rw[j] = G.rot_wa[6 * v + j];
  }
  for (int k = lane; k < G.N; k += 32) {
    double r = 0.0;
    for (int j = 0; j < 6; ++j) r += rw[j] * L1[E[j] + k];
    zeta1[v * ld + k] = r;
  }
}

struct BDArgs {
  const double *D1, *zeta1;                // divergence and curl of L(vn); NULL: no background diffusion
  double scale;                            // c Abar^2
};

__global__ void __launch_bounds__(256, 4) k_diff_edge(Geo64 G, double* __restrict__ vn, const double* __restrict__ ux,
                                                   const double* __restrict__ uy, const double* __restrict__ uz,
                                                   const double* __restrict__ zeta, const double* __restrict__ divc,
                                                   const double* __restrict__ thv, double* __restrict__ Kh_out,
                                                   double* __restrict__ thflx, double dt, BDArgs bd) {
  const int64_t e = warp_entity();
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t Q[4];
  for (int j = 0; j < 4; ++j) Q[j] = (int64_t)G.e2q[4 * e + j] * ld;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld;
  const int64_t v1 = (int64_t)G.e2v[2 * e] * ld, v2 = (int64_t)G.e2v[2 * e + 1] * ld;
  const double* n = G.n_e + 3 * e;
  const double* t = G.t_e + 3 * e;
  const double le = G.l_e[e], de = G.d_e[e], i34 = G.inv_L34[e], ile = G.inv_le[e], ide = G.inv_de[e];
  const double cs2ld = (kCsSmag * kCsSmag) * (le * de);
  for (int k = lane; k < G.N; k += 32) {
    const double d34x = ux[Q[3] + k] - ux[Q[2] + k], d34y = uy[Q[3] + k] - uy[Q[2] + k],
                 d34z = uz[Q[3] + k] - uz[Q[2] + k];
    const double d12x = ux[Q[1] + k] - ux[Q[0] + k], d12y = uy[Q[1] + k] - uy[Q[0] + k],
                 d12z = uz[Q[1] + k] - uz[Q[0] + k];
    const double DT = dot3(d34x, d34y, d34z, n) * i34 - dot3(d12x, d12y, d12z, t) * ile;
    const double DS = dot3(d34x, d34y, d34z, t) * i34 + dot3(d12x, d12y, d12z, n) * ile;
    const double Kh = cs2ld * sqrt(DT * DT + DS * DS);
    const double lap = (divc[c2 + k] - divc[c1 + k]) * ide - (zeta[v2 + k] - zeta[v1 + k]) * ile;
    double vnew = vn[e * ld + k] + dt * Kh * lap;
    if (bd.D1) {
      const double lap2 = (bd.D1[c2 + k] - bd.D1[c1 + k]) * ide - (bd.zeta1[v2 + k] - bd.zeta1[v1 + k]) * ile;
      vnew -= bd.scale * lap2;
    }
    vn[e * ld + k] = vnew;
    Kh_out[e * ld + k] = Kh;
    thflx[e * ld + k] = (le * Kh) * (thv[c2 + k] - thv[c1 + k]) * ide;
  }
}

__global__ void __launch_bounds__(256) k_diff_theta(Geo64 G, const double* __restrict__ thflx, double* __restrict__ thv,
                                                    double* __restrict__ ex, double dt) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[3];
  double sg[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    sg[s] = G.s_ce[3 * c + s];
  }
  const double dtA = dt * G.inv_Ac[c];
  for (int k = lane; k < G.N; k += 32) {
    double acc = 0.0;
    for (int s = 0; s < 3; ++s) acc += sg[s] * thflx[E[s] + k];
    const double dth = dtA * acc;
    const double th = thv[c * ld + k];
    ex[c * ld + k] = ex[c * ld + k] * (1.0 + ((kRd / kCvd) * dth) * recip64(th));
    thv[c * ld + k] = th + dth;
  }
}

Geo64 make_geo(const icon_grid* grid, const double* cc) {
  const GridDev& g = grid->g;
  const Vertical& v = grid->vert;
  Geo64 G;
  G.nc = g.nc; G.ne = g.ne; G.nv = g.nv; G.N = v.N; G.ld = v.ld;
  G.c2e = g.c2e; G.e2c = g.e2c; G.e2v = g.e2v; G.v2e = g.v2e; G.v2c = g.v2c; G.vdeg = g.vdeg;
  G.e2vt = g.e2vt; G.e2q = g.e2q;
  G.div_wa = g.div_wa; G.rot_wa = g.rot_wa; G.inv_Ac = g.inv_Ac; G.vt_w = g.vt_w; G.kin_w = g.kin_w;
  G.lsq_w = g.lsq_w; G.inv_de = g.inv_de; G.inv_le = g.inv_le; G.l_e = g.l_e; G.d_e = g.d_e; G.f_e = g.f_e;
  G.inv_L34 = g.inv_L34; G.n_e = g.n_e; G.t_e = g.t_e; G.s_ce = g.s_ce;
  G.wu = v.d_wu; G.wl = v.d_wl; G.inv_dz = v.d_inv_dz; G.inv_dz2 = v.d_inv_dz2; G.qinv_dz = v.d_qinv_dz;
  G.cc = cc;
  G.kin_w_h = G.div_wa_h = nullptr;
  G.t_sn = G.t_bf = G.t_wu_e = G.t_qinv_dz_e = G.t_dz_e = nullptr;
  G.t_wu_c = G.t_inv_dz_c = G.t_inv_dzh_c = G.t_wcc = G.t_wcon = G.t_ep = G.t_hdpdz = nullptr;
  return G;
}

void launch_column(const Geo64& G, const ColArgs& a, bool topo, cudaStream_t st) {
  const unsigned nbc = blocks_for(G.nc, kWarpsPerBlock);
  if (topo) k_col_rows<true><<<nbc, 256, 0, st>>>(G, a);
  else k_col_rows<false><<<nbc, 256, 0, st>>>(G, a);
  k_col_thomas<<<blocks_for(G.nc, 128), 128, 0, st>>>(G, a);
  if (topo) k_col_update<true><<<nbc, 256, 0, st>>>(G, a);
  else k_col_update<false><<<nbc, 256, 0, st>>>(G, a);
}

}  // namespace

namespace {

Geo64 state_geo(const icon_state* st) {
  const StateDev& s = st->s;
  Geo64 G = make_geo(st->grid, s.colconst);
  G.kin_w_h = s.kin_w_h;
  G.div_wa_h = s.div_wa_h;
  const TopoDev& T = s.topo;
  if (T.on) {
    G.t_sn = T.sn; G.t_bf = T.bf; G.t_wu_e = T.wu_e; G.t_qinv_dz_e = T.qinv_dz_e; G.t_dz_e = T.dz_e;
    G.t_wu_c = T.wu_c; G.t_inv_dz_c = T.inv_dz_c; G.t_inv_dzh_c = T.inv_dzh_c;
    G.t_wcc = T.wcc; G.t_wcon = T.wcon; G.t_ep = T.ep; G.t_hdpdz = T.hdpdz;
  }
  return G;
}

}  // namespace

// the parts of one FP64 step, in the order enqueue_step_fp64 issues them; a decomposed
// domain issues them for every part with halo exchanges between the stages
void fp64_step_begin(icon_state* st, double dt, int nsub, cudaStream_t stream) {
  StateDev& s = st->s;
  const Vertical& vg = st->grid->vert;
  const double dtau = dt / nsub;
  k_colconst64<<<1, 128, 0, stream>>>(vg.N, vg.ld, vg.d_wu, vg.d_wl, vg.d_dzh, vg.d_dz, vg.d_ray, dtau, s.colconst);
  cudaMemsetAsync(s.mflx, 0, sizeof(double) * st->grid->g.ne * vg.ld, stream);
  cudaMemsetAsync(s.wflx, 0, sizeof(double) * st->grid->g.nc * vg.ld, stream);
}

void fp64_step_stage(icon_state* st, double dt, int nsub, bool corr, cudaStream_t stream) {
  StateDev& s = st->s;
  const Geo64 G = state_geo(st);
  const TopoDev& T = s.topo;
  const bool topo = T.on;
  const double dtau = dt / nsub;
  const unsigned nbv = blocks_for(G.nv, kWarpsPerBlock), nbe = blocks_for(G.ne, kWarpsPerBlock),
                 nbc = blocks_for(G.nc, kWarpsPerBlock);
  const double* vn_st = corr ? s.vn_s : s.vn;
  const double* w_st = corr ? s.w_s : s.w;
  const double* rho_st = corr ? s.rho_s : s.rho;
  const double* thv_st = corr ? s.thv_s : s.thv;
  const double* ex_st = corr ? s.ex_s : s.ex;
  prof_begin(stream, K_VERTEX);
  k_vertex<<<nbv, 256, 0, stream>>>(G, vn_st, w_st, s.zeta, s.w_v);
  prof_end(stream);
  prof_begin(stream, K_EDGE_VT);
  k_edge_vt<<<nbe, 256, 0, stream>>>(G, vn_st, s.vt, s.Ke);
  prof_end(stream);
  prof_begin(stream, K_CELL_KE);
  k_cell_ke<<<nbc, 256, 0, stream>>>(G, s.Ke, s.Kc);
  prof_end(stream);
  if (topo) topo_stage(st, vn_st, s.vt, w_st, ex_st, stream);
  EdgeArgs ea;
  ea.vn = vn_st; ea.w = w_st; ea.rho = rho_st; ea.thv = thv_st; ea.ex = ex_st;
  ea.vt = s.vt; ea.Kc = s.Kc; ea.zeta = s.zeta; ea.w_v = s.w_v;
  ea.vn_base = s.vn;
  ea.vn_out = corr ? s.vn : s.vn_s;
  ea.Avn0 = s.Avn0;
  ea.F = s.F; ea.G = s.G; ea.a_e = s.a_e; ea.mflx = s.mflx;
  ea.dtau = dtau; ea.inv_nsub = 1.0 / nsub; ea.corrector = corr;
  ea.hinv_nsub = 0.5 / nsub;
  ea.hdtau = 0.5 * dtau;
  const bool damp = corr && st->divdamp4 > 0.0;
  ea.skip_flux = damp ? 1 : 0;
  ea.upwind_theta = st->upwind_theta ? 1 : 0;
  prof_begin(stream, K_EDGE_TEND);
  if (topo) {
    if (ea.upwind_theta) k_edge_tend<true, true><<<nbe, 256, 0, stream>>>(G, ea);
    else k_edge_tend<true, false><<<nbe, 256, 0, stream>>>(G, ea);
  } else {
    if (ea.upwind_theta) k_edge_tend<false, true><<<nbe, 256, 0, stream>>>(G, ea);
    else k_edge_tend<false, false><<<nbe, 256, 0, stream>>>(G, ea);
  }
  prof_end(stream);
  if (damp) {
    // Kc and the column's update-operand scratch are free until the column runs
    const double abar = st->abar;
    DDArgs da;
    da.L = s.col_rx; da.rho = rho_st; da.thv = thv_st;
    da.vn = s.vn; da.F = s.F; da.G = s.G; da.mflx = s.mflx;
    da.dz_e = topo ? T.dz_e : nullptr;
    da.scale = st->divdamp4 * abar * abar; da.inv_nsub = 1.0 / nsub;
    da.upwind_theta = st->upwind_theta ? 1 : 0;
    prof_begin(stream, K_DIVDAMP);
    k_dd_div<<<nbc, 256, 0, stream>>>(G, s.vn, s.Kc);
    k_dd_lap<<<nbc, 256, 0, stream>>>(G, s.Kc, s.col_rx);
    k_dd_edge<<<nbe, 256, 0, stream>>>(G, da);
    prof_end(stream);
  }
  ColArgs ca;
  ca.rho = s.rho; ca.thv = s.thv; ca.ex = s.ex; ca.w = s.w;
  ca.w_stage = w_st;
  ca.F = s.F; ca.G = s.G; ca.a_e = s.a_e;
  ca.Aw0 = s.Aw0;
  ca.lo = s.col_lo; ca.di = s.col_di; ca.up = s.col_up; ca.rh = s.col_rh; ca.ws = s.col_ws;
  ca.rx = s.col_rx; ca.tx = s.col_tx; ca.px = s.col_px; ca.gm = s.col_gm;
  ca.ri = s.col_ri; ca.mm = s.col_mm; ca.gc = s.col_gc;
  ca.rho_o = corr ? s.rho : s.rho_s;
  ca.thv_o = corr ? s.thv : s.thv_s;
  ca.ex_o = corr ? s.ex : s.ex_s;
  ca.w_o = corr ? s.w : s.w_s;
  ca.wflx = s.wflx;
  ca.status = s.status;
  ca.dtau = dtau; ca.inv_nsub = 1.0 / nsub; ca.corrector = corr;
  ca.hdtau = 0.5 * dtau;
  ca.b_new = kBeta / nsub;
  ca.b_old = (1.0 - kBeta) / nsub;
  prof_begin(stream, K_COLUMN);
  launch_column(G, ca, topo, stream);
  prof_end(stream);
}

void fp64_step_diffusion(icon_state* st, double dt, cudaStream_t stream) {
  StateDev& s = st->s;
  const Geo64 G = state_geo(st);
  const unsigned nbv = blocks_for(G.nv, kWarpsPerBlock), nbe = blocks_for(G.ne, kWarpsPerBlock),
                 nbc = blocks_for(G.nc, kWarpsPerBlock);
  prof_begin(stream, K_DIFF_VERTEX);
  k_diff_vertex<<<nbv, 256, 0, stream>>>(G, s.vn, s.uvx, s.uvy, s.uvz, s.zeta);
  prof_end(stream);
  prof_begin(stream, K_DIFF_DIV);
  k_diff_div<<<nbc, 256, 0, stream>>>(G, s.vn, s.divc);
  prof_end(stream);
  BDArgs bd;
  bd.D1 = nullptr; bd.zeta1 = nullptr; bd.scale = 0.0;
  if (st->diff4 > 0.0) {
    // scratch that is dead during diffusion: a_e (edges), two column-scratch cell arrays
    const double abar = st->abar;
    prof_begin(stream, K_DIFF4);
    k_bd_lap<<<nbe, 256, 0, stream>>>(G, s.zeta, s.divc, s.a_e);
    k_bd_curl<<<nbv, 256, 0, stream>>>(G, s.a_e, s.col_di);
    k_diff_div<<<nbc, 256, 0, stream>>>(G, s.a_e, s.col_lo);
    prof_end(stream);
    bd.D1 = s.col_lo; bd.zeta1 = s.col_di; bd.scale = st->diff4 * abar * abar;
  }
  prof_begin(stream, K_DIFF_EDGE);
  k_diff_edge<<<nbe, 256, 0, stream>>>(G, s.vn, s.uvx, s.uvy, s.uvz, s.zeta, s.divc, s.thv, s.Kh, s.thflx, dt, bd);
  prof_end(stream);
  prof_begin(stream, K_DIFF_THETA);
  k_diff_theta<<<nbc, 256, 0, stream>>>(G, s.thflx, s.thv, s.ex, dt);
  prof_end(stream);
}

void enqueue_step_fp64(icon_state* st, double dt, int nsub, cudaStream_t stream) {
  fp64_step_begin(st, dt, nsub, stream);
  for (int it = 0; it < nsub; ++it)
    for (int stage = 0; stage < 2; ++stage) fp64_step_stage(st, dt, nsub, stage == 1, stream);
  fp64_step_diffusion(st, dt, stream);
}

}  // namespace icon
