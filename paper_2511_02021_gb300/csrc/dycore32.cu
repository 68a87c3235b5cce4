// Mixed-precision dynamical-core step: FP32 horizontal stencils and advection,
// FP64 vertically implicit w/Exner solve, FP64 rho / Theta / Exner prognostic
// updates, FP64 mass-flux accumulation and FP64 mass integral.
//
// Same discretisation as the FP64 step (operators O1-O7, predictor-corrector
// substeps with off-centring beta = 0.65, Thomas solve, Rayleigh damping,
// Smagorinsky diffusion); what changes is the precision of each quantity and
// the data layout:
//
//  * vn and every stencil temporary are FP32, stored level-contiguous
//    ([entity][ld]) so that the lanes of a warp gather whole neighbour rows.
//  * rho, theta_v, Exner and w are FP64 prognostics stored level-major ([k][Nc]):
//    only the thread-per-column solve reads and writes them, and in this layout
//    its loads and stores are coalesced across the 32 columns of a warp. FP32
//    shadows ([Nc][ld]: rho, theta_v, Exner - Exner_ref(z), w) feed the stencils.
//  * FP64 is used where the method needs it: the hydrostatic-cancellation terms
//    (the explicit w predictor and a_k (pi_{k-1} - pi_k) in the right-hand side),
//    the tridiagonal system and its solution, the rho / Theta / Exner updates of
//    S^{n+1}, the horizontal mass-flux divergence (the FP32 edge mass fluxes
//    rho_e vn weighted by FP64 s l / A_c and summed in FP64, so that the two cells of
//    an edge use the same value, the global mass is conserved to rounding and the
//    step-mean mass flux reproduces the density change exactly) and the accumulated
//    mass fluxes. Coefficients that only multiply small increments (the linearised
//    state equation factor (Rd/cvd) pi/Theta) are FP32.
//  * The predictor writes the provisional state S* only as FP32 shadows: S* is
//    consumed by FP32 stencils, while the corrector's column uses coefficients
//    frozen at S^n. After the FP64 back substitution, the predictor forms those
//    shadows' implicit increments in FP32.
//
// Every kernel body is a per-item device function (one entity for the stencils,
// one column for the solve) shared by the per-state kernels and by the persistent
// ensemble kernel. The stencil kernels take the number of lanes per entity (32 or
// 16: one or two entities per warp) and the block size from the autotuner; each
// output is computed by one lane with a fixed summation order, so the results do
// not depend on the tile shape.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include "icon_internal.h"
#include "fastconv.h"
#include "recip64.h"

namespace icon {
namespace {

constexpr float kRcvF = (float)(kRd / kCvd);

struct MxGeo {
  int64_t nc, ne, nv;
  int N, ld;
  const int *c2e, *e2c, *e2v, *v2e, *v2c, *vdeg, *e2vt, *e2q;
  const float *div_w32, *rot_w32, *vt_w32, *kin_w32, *lsq_w32, *inv_de32, *inv_le32, *f_e32, *l_e32;
  const float *n_e32, *t_e32, *L34inv32, *s_ce32;
  const double* inv_Ac;                    // 1 / A_c (FP64)
  const double* div_wa;                    // [Nc][3] s_ce l_e / A_c (FP64)
  const double *dz, *dzh, *wu, *wl, *dz2, *ray, *ex_ref;
  const float *inv_dz32, *wu32, *wl32, *inv_dz2_32;
};

// ---------------------------------------------------------------- stencil items (lanes over levels)

// O3 curl (full levels) and the vertex mean of w (half levels)
template <int LPE>
__device__ inline void mx_vertex_item(const MxGeo& G, const float* __restrict__ vn, const float* __restrict__ w,
                                      float* __restrict__ zeta, float* __restrict__ w_v, int64_t v, int lane) {
  const int ld = G.ld;
  int64_t E[6], C[6];
  float rw[6];
  for (int j = 0; j < 6; ++j) {
    E[j] = (int64_t)G.v2e[6 * v + j] * ld;
    C[j] = (int64_t)G.v2c[6 * v + j] * ld;
    rw[j] = G.rot_w32[6 * v + j];
  }
  const int deg = G.vdeg[v];
  const float inv_deg = 1.0f / (float)deg;
  for (int k = lane; k < G.N; k += LPE) {
    float acc = 0.f;
    for (int j = 0; j < 6; ++j) acc += rw[j] * vn[E[j] + k];
    zeta[v * ld + k] = acc;
  }
  for (int h = lane; h <= G.N; h += LPE) {
    float acc = 0.f;
    for (int j = 0; j < 5; ++j) acc += w[C[j] + h];
    if (deg == 6) acc += w[C[5] + h];
    w_v[v * ld + h] = acc * inv_deg;
  }
}

// O4 vt
template <int LPE>
__device__ inline void mx_edge_diag_item(const MxGeo& G, const float* __restrict__ vn, float* __restrict__ vt,
                                         int64_t e, int lane) {
  const int ld = G.ld;
  int64_t S[5];
  float W[5];
  for (int j = 0; j < 5; ++j) {
    S[j] = (int64_t)G.e2vt[5 * e + j] * ld;
    W[j] = G.vt_w32[5 * e + j];
  }
  for (int k = lane; k < G.N; k += LPE) {
    float acc = 0.f;
    for (int j = 0; j < 5; ++j) acc += W[j] * vn[S[j] + k];
    vt[e * ld + k] = acc;
  }
}

// O5 K_c = sum_e kappa_ce (vn_e^2 + vt_e^2)/2
template <int LPE>
__device__ inline void mx_cell_ke_item(const MxGeo& G, const float* __restrict__ vn, const float* __restrict__ vt,
                                       float* __restrict__ Kc, int64_t c, int lane) {
  const int ld = G.ld;
  int64_t E[3];
  float kw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    kw[s] = G.kin_w32[3 * c + s];
  }
  for (int k = lane; k < G.N; k += LPE) {
    float acc = 0.f;
    for (int s = 0; s < 3; ++s) {
      const float a = vn[E[s] + k], b = vt[E[s] + k];
      acc += kw[s] * (0.5f * (a * a + b * b));
    }
    Kc[c * ld + k] = acc;
  }
}

struct MxEdgeArgs {
  const float *vn, *w, *rho, *thv, *exp;   // stage state (FP32 shadows; exp = Exner - Exner_ref)
  const float *vt, *Kc, *zeta, *w_v;
  const float* vn_base;
  float* vn_out;
  float* Avn0;
  float *phi, *gth, *a_e;                  // rho_e vn, l_e rho_e vn theta_e, w-advection edge term
  double* mflx;
  float dtau;
  double inv_nsub;
  int corrector;
  int skip_flux;                           // fluxes formed after divergence damping instead
  int upwind_theta;                        // heat flux with the upwind theta_v (option)
  // terrain-following levels (TOPO instances only; see terrain.cu): per-edge weights,
  // 1/dz and dz ([Ne][ld]), cpd times the normal slope factor per edge, the full-level
  // decay, and the stage's w - wcc and half of d(pi')/dz at cells ([Nc][ld])
  const float *t_wu_e, *t_inv_dz_e, *t_dz_e, *t_csn, *t_bf, *t_wcon, *t_hdpdz;
};

// vn tendency and update, horizontal flux integrals, edge part of the w advection.
// One pass over the half levels in windows of LPE - 1: lane l of an entity's lane
// group holds half level h = base + l and, except the last lane, full level k = h;
// each half-level interpolant and cell-pair sum of w is formed once and passed to the
// lane below with a shuffle (only the group's own lanes take part, so the two halves
// of a warp may serve different entities). TOPO (terrain-following levels): per-edge
// interpolation weights, w - wcc in the vertical advection, the metric correction of the
// pressure gradient (exp is then against the per-cell reference), fluxes through dz_e.
// HOIST: read the arguments the level loop uses once, the outputs through restrict pointers
// (the per-state kernels: 5.6 -> 5.3 ms per R2B6/90 mixed step); the persistent ensemble
// keeps them in its shared-memory slot and reads them there, which its 64-register budget
// takes better (hoisted, its edge phase spilled and slowed from 55 to 79 ms per step)
template <int LPE, bool TOPO = false, bool HOIST = true>
__device__ inline void mx_edge_tend_item(const MxGeo& G, const MxEdgeArgs& a, int64_t e, int lane) {
  const int ld = G.ld, N = G.N;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld;
  const int64_t v1 = (int64_t)G.e2v[2 * e] * ld, v2 = (int64_t)G.e2v[2 * e + 1] * ld;
  const float ide = G.inv_de32[e], ile = G.inv_le32[e], fe = G.f_e32[e], le = G.l_e32[e];
  const float cide = (float)kCpd * ide;
  const float csn = TOPO ? a.t_csn[e] : 0.0f;
  const int64_t o = e * ld;
  const float* __restrict__ vn = a.vn + o;
  const float* __restrict__ vt = a.vt + o;
  const float* __restrict__ w = a.w;
  const float* __restrict__ wv = a.w_v;
  const float* __restrict__ zeta = a.zeta;
  const float* __restrict__ Kc = a.Kc;
  const float* __restrict__ thv = a.thv;
  const float* __restrict__ exq = a.exp;
  const float* __restrict__ rho = a.rho;
  // the arguments the level loop uses (vn_base, Avn0 and vn_out may be one buffer, updated
  // element by element)
  const float* __restrict__ wu32 = G.wu32;
  const float* __restrict__ wl32 = G.wl32;
  const float* __restrict__ idz32 = G.inv_dz32;
  float* __restrict__ ae_o = a.a_e + o;
  const float* vnb_o = a.vn_base + o;
  float* avn_o = a.Avn0 + o;
  float* vout_o = a.vn_out + o;
  float* __restrict__ phi_o = a.phi + o;
  float* __restrict__ gth_o = a.gth + o;
  double* __restrict__ mflx_o = a.mflx + o;
  const bool corr = a.corrector != 0, skip = a.skip_flux != 0, upw = a.upwind_theta != 0;
  const float dtau = a.dtau;
  const double inv_nsub = a.inv_nsub;
  static_assert(LPE == 8 || LPE == 16 || LPE == 32, "lane groups of 8, 16 or 32");
  const unsigned seg = LPE == 32 ? 0xffffffffu : (((1u << LPE) - 1u) << (threadIdx.x & (32 - LPE)));
#pragma unroll 2   // two windows' loads in flight (the kernel is bound by load latency)
  for (int base = 0; base <= N; base += LPE - 1) {
    const int h = base + lane;
    const bool hv = h <= N;
    const int hl = h > 0 ? (h - 1 < N - 1 ? h - 1 : N - 1) : 0;
    const int hu = h < N ? h : N - 1;
    const bool inner = h > 0 && h < N;
    float wa, wb;
    if constexpr (TOPO) {
      wa = inner ? a.t_wu_e[o + h] : (h == 0 ? 0.0f : 1.0f);
      wb = inner ? 1.0f - wa : (h == 0 ? 1.0f : 0.0f);
    } else {
      wa = inner ? (HOIST ? wu32 : G.wu32)[h] : (h == 0 ? 0.0f : 1.0f);
      wb = inner ? (HOIST ? wl32 : G.wl32)[h] : (h == 0 ? 1.0f : 0.0f);
    }
    float vie = 0.f, tie = 0.f, sw = 0.f, dw = 0.f, dwv = 0.f;
    if (hv) {
      vie = wa * vn[hl] + wb * vn[hu];
      tie = wa * vt[hl] + wb * vt[hu];
      const float w1 = w[c1 + h], w2 = w[c2 + h];
      if constexpr (TOPO) sw = a.t_wcon[c1 + h] + a.t_wcon[c2 + h];     // 0 at the lid and the ground
      else sw = w1 + w2;
      dw = w2 - w1;
      dwv = wv[v2 + h] - wv[v1 + h];
    }
    const float vie_up = __shfl_down_sync(seg, vie, 1, LPE);
    const float sw_up = __shfl_down_sync(seg, sw, 1, LPE);
    if (!hv || lane == LPE - 1) continue;
    if constexpr (HOIST) ae_o[h] = vie * dw * ide + tie * dwv * ile;
    else a.a_e[o + h] = vie * dw * ide + tie * dwv * ile;
    if (h == N) continue;
    const int k = h;
    const float wbar = 0.25f * (sw + sw_up);
    const float zeta_e = 0.5f * (zeta[v1 + k] + zeta[v2 + k]);
    const float A = -(Kc[c2 + k] - Kc[c1 + k]) * ide + (zeta_e + fe) * vt[k] -
                    wbar * (vie - vie_up) * (TOPO ? a.t_inv_dz_e[o + k] : (HOIST ? idz32 : G.inv_dz32)[k]);
    const float t1 = thv[c1 + k], t2 = thv[c2 + k];
    const float th_e = 0.5f * (t1 + t2);
    float pg;
    if constexpr (TOPO)
      pg = th_e * ((exq[c2 + k] - exq[c1 + k]) * cide - (csn * a.t_bf[k]) * (a.t_hdpdz[c1 + k] + a.t_hdpdz[c2 + k]));
    else
      pg = th_e * ((exq[c2 + k] - exq[c1 + k]) * cide);
    float vnew;
    if constexpr (HOIST) {
      if (corr) {
        vnew = vnb_o[k] + dtau * (0.5f * (avn_o[k] + A) - pg);
      } else {
        vnew = vnb_o[k] + dtau * (A - pg);
        avn_o[k] = A;
      }
      vout_o[k] = vnew;
      if (skip) continue;
    } else {
      if (a.corrector) {
        vnew = a.vn_base[o + k] + a.dtau * (0.5f * (a.Avn0[o + k] + A) - pg);
      } else {
        vnew = a.vn_base[o + k] + a.dtau * (A - pg);
        a.Avn0[o + k] = A;
      }
      a.vn_out[o + k] = vnew;
      if (a.skip_flux) continue;
    }
    float F = 0.5f * (rho[c1 + k] + rho[c2 + k]) * vnew;
    if constexpr (TOPO) F *= a.t_dz_e[o + k];
    if constexpr (HOIST) {
      phi_o[k] = F;
      gth_o[k] = (le * F) * (upw ? (vnew >= 0.0f ? t1 : t2) : th_e);
      if (corr) mflx_o[k] += f32_to_f64(F) * inv_nsub;
    } else {
      a.phi[o + k] = F;
      a.gth[o + k] = (le * F) * (a.upwind_theta ? (vnew >= 0.0f ? t1 : t2) : th_e);
      if (a.corrector) a.mflx[o + k] += f32_to_f64(F) * a.inv_nsub;
    }
  }
}

// fourth-order divergence damping of the corrector's vn^{n+1} (option), FP32 like the other
// stencils: cell divergence, its cell Laplacian, then the edge update with the corrector's
// fluxes (the same expressions as the edge tendency) and the FP64 step-mean mass flux
__device__ inline void mx_dd_div_item(const MxGeo& G, const float* __restrict__ vn, float* __restrict__ D, int64_t c,
                                      int lane) {
  const int ld = G.ld;
  int64_t E[3];
  float dw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    dw[s] = G.div_w32[3 * c + s];
  }
  for (int k = lane; k < G.N; k += 32) D[c * ld + k] = dw[0] * vn[E[0] + k] + dw[1] * vn[E[1] + k] + dw[2] * vn[E[2] + k];
}

__global__ void __launch_bounds__(256) k_mx_dd_div(MxGeo G, const float* __restrict__ vn, float* __restrict__ D) {
  const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c < G.nc) mx_dd_div_item(G, vn, D, c, threadIdx.x & 31);
}

__device__ inline void mx_dd_lap_item(const MxGeo& G, const float* __restrict__ D, float* __restrict__ L, int64_t c,
                                      int lane) {
  const int ld = G.ld;
  int64_t A[3], B[3];
  float wt[3];
  for (int s = 0; s < 3; ++s) {
    const int e = G.c2e[3 * c + s];
    A[s] = (int64_t)G.e2c[2 * e] * ld;
    B[s] = (int64_t)G.e2c[2 * e + 1] * ld;
    wt[s] = G.div_w32[3 * c + s] * G.inv_de32[e];
  }
  for (int k = lane; k < G.N; k += 32)
    L[c * ld + k] = wt[0] * (D[B[0] + k] - D[A[0] + k]) + wt[1] * (D[B[1] + k] - D[A[1] + k]) +
                    wt[2] * (D[B[2] + k] - D[A[2] + k]);
}

__global__ void __launch_bounds__(256) k_mx_dd_lap(MxGeo G, const float* __restrict__ D, float* __restrict__ L) {
  const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c < G.nc) mx_dd_lap_item(G, D, L, c, threadIdx.x & 31);
}

struct MxDDArgs {
  const float *L, *rho, *thv;
  const float* dz_e;                       // layer thickness at edges (terrain-following), or NULL
  float *vn, *phi, *gth;
  double* mflx;
  float scale;                             // c4 Abar^2
  double inv_nsub;
  int upwind_theta;
};

__device__ inline void mx_dd_edge_item(const MxGeo& G, const MxDDArgs& a, int64_t e, int lane) {
  const int ld = G.ld;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld, o = e * ld;
  const float sc = a.scale * G.inv_de32[e], le = G.l_e32[e];
  for (int k = lane; k < G.N; k += 32) {
    const float vn = a.vn[o + k] - sc * (a.L[c2 + k] - a.L[c1 + k]);
    a.vn[o + k] = vn;
    float F = 0.5f * (a.rho[c1 + k] + a.rho[c2 + k]) * vn;
    if (a.dz_e) F *= a.dz_e[o + k];
    a.phi[o + k] = F;
    const float t1 = a.thv[c1 + k], t2 = a.thv[c2 + k];
    a.gth[o + k] = (le * F) * (a.upwind_theta ? (vn >= 0.0f ? t1 : t2) : 0.5f * (t1 + t2));
    a.mflx[o + k] += f32_to_f64(F) * a.inv_nsub;
  }
}

__global__ void __launch_bounds__(256) k_mx_dd_edge(MxGeo G, MxDDArgs a) {
  const int64_t e = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (e < G.ne) mx_dd_edge_item(G, a, e, threadIdx.x & 31);
}

// diffusion: least-squares vertex velocity and O3 curl of vn
template <int LPE>
__device__ inline void mx_diff_vertex_item(const MxGeo& G, const float* __restrict__ vn, float* __restrict__ ux,
                                           float* __restrict__ uy, float* __restrict__ uz, float* __restrict__ zeta,
                                           int64_t v, int lane) {
  const int ld = G.ld;
  int64_t E[6];
  for (int j = 0; j < 6; ++j) E[j] = (int64_t)G.v2e[6 * v + j] * ld;
  const float* lw = G.lsq_w32 + 18 * v;
  const float* rw = G.rot_w32 + 6 * v;
  float L[18], R[6];
  for (int j = 0; j < 18; ++j) L[j] = lw[j];
  for (int j = 0; j < 6; ++j) R[j] = rw[j];
  for (int k = lane; k < G.N; k += LPE) {
    float x = 0.f, y = 0.f, z = 0.f, r = 0.f;
    for (int j = 0; j < 6; ++j) {
      const float q = vn[E[j] + k];
      x += L[3 * j] * q;
      y += L[3 * j + 1] * q;
      z += L[3 * j + 2] * q;
      r += R[j] * q;
    }
    ux[v * ld + k] = x;
    uy[v * ld + k] = y;
    uz[v * ld + k] = z;
    zeta[v * ld + k] = r;
  }
}

// diffusion: O2 divergence of vn
template <int LPE>
__device__ inline void mx_diff_div_item(const MxGeo& G, const float* __restrict__ vn, float* __restrict__ divc,
                                        int64_t c, int lane) {
  const int ld = G.ld;
  int64_t E[3];
  float dw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    dw[s] = G.div_w32[3 * c + s];
  }
  for (int k = lane; k < G.N; k += LPE) divc[c * ld + k] = dw[0] * vn[E[0] + k] + dw[1] * vn[E[1] + k] + dw[2] * vn[E[2] + k];
}

// diffusion: Smagorinsky K_h, vn += dt K_h L(vn), theta_v flux
template <int LPE>
__device__ inline void mx_diff_edge_item(const MxGeo& G, float* __restrict__ vn, const float* __restrict__ ux,
                                         const float* __restrict__ uy, const float* __restrict__ uz,
                                         const float* __restrict__ zeta, const float* __restrict__ divc,
                                         const float* __restrict__ thv, float* __restrict__ thflx, float dt, int64_t e,
                                         int lane, const float* __restrict__ D1 = nullptr,
                                         const float* __restrict__ zeta1 = nullptr, float bd_scale = 0.0f) {
  const int ld = G.ld;
  int64_t Q[4];
  for (int j = 0; j < 4; ++j) Q[j] = (int64_t)G.e2q[4 * e + j] * ld;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld;
  const int64_t v1 = (int64_t)G.e2v[2 * e] * ld, v2 = (int64_t)G.e2v[2 * e + 1] * ld;
  const float nx = G.n_e32[3 * e], ny = G.n_e32[3 * e + 1], nz = G.n_e32[3 * e + 2];
  const float tx = G.t_e32[3 * e], ty = G.t_e32[3 * e + 1], tz = G.t_e32[3 * e + 2];
  const float ide = G.inv_de32[e], ile = G.inv_le32[e], i34 = G.L34inv32[e], le = G.l_e32[e];
  const float cs2ld = (float)(kCsSmag * kCsSmag) * le / ide;
  for (int k = lane; k < G.N; k += LPE) {
    const float ax = ux[Q[3] + k] - ux[Q[2] + k], ay = uy[Q[3] + k] - uy[Q[2] + k], az = uz[Q[3] + k] - uz[Q[2] + k];
    const float bx = ux[Q[1] + k] - ux[Q[0] + k], by = uy[Q[1] + k] - uy[Q[0] + k], bz = uz[Q[1] + k] - uz[Q[0] + k];
    const float DT = (ax * nx + ay * ny + az * nz) * i34 - (bx * tx + by * ty + bz * tz) * ile;
    const float DS = (ax * tx + ay * ty + az * tz) * i34 + (bx * nx + by * ny + bz * nz) * ile;
    const float Kh = cs2ld * sqrtf(DT * DT + DS * DS);
    const float lap = (divc[c2 + k] - divc[c1 + k]) * ide - (zeta[v2 + k] - zeta[v1 + k]) * ile;
    float vnew = vn[e * ld + k] + dt * Kh * lap;
    if (D1) {                              // fourth-order background diffusion (option)
      const float lap2 = (D1[c2 + k] - D1[c1 + k]) * ide - (zeta1[v2 + k] - zeta1[v1 + k]) * ile;
      vnew -= bd_scale * lap2;
    }
    vn[e * ld + k] = vnew;
    thflx[e * ld + k] = le * Kh * (thv[c2 + k] - thv[c1 + k]) * ide;
  }
}

// fourth-order background diffusion (option), FP32: L1 = L(vn) at edges, then the curl
// (vertices) and divergence (cells) of L1 for the second Laplacian in the edge item
__global__ void __launch_bounds__(256) k_mx_bd_lap(MxGeo G, const float* __restrict__ zeta,
                                                   const float* __restrict__ divc, float* __restrict__ L1) {
  const int64_t e = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld;
  const int64_t v1 = (int64_t)G.e2v[2 * e] * ld, v2 = (int64_t)G.e2v[2 * e + 1] * ld;
  const float ide = G.inv_de32[e], ile = G.inv_le32[e];
  for (int k = lane; k < G.N; k += 32)
    L1[e * ld + k] = (divc[c2 + k] - divc[c1 + k]) * ide - (zeta[v2 + k] - zeta[v1 + k]) * ile;
}

__global__ void __launch_bounds__(256) k_mx_bd_curldiv(MxGeo G, const float* __restrict__ L1, float* __restrict__ zeta1,
                                                       float* __restrict__ D1) {
  const int64_t item = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31, ld = G.ld;
  if (item < G.nv) {
    const int64_t v = item;
    int64_t E[6];
    float rw[6];
    for (int j = 0; j < 6; ++j) {
      E[j] = (int64_t)G.v2e[6 * v + j] * ld;
      rw[j] = G.rot_w32[6 * v + j];
    }
    for (int k = lane; k < G.N; k += 32) {
      float r = 0.0f;
      for (int j = 0; j < 6; ++j) r += rw[j] * L1[E[j] + k];
      zeta1[v * ld + k] = r;
    }
  } else if (item < G.nv + G.nc) {
    mx_diff_div_item<32>(G, L1, D1, item - G.nv, lane);
  }
}

// ---------------------------------------------------------------- column items (one thread per column)

// per-level constants of the column solve for one dtau, FP64 [8][ld]:
// wu, wl, dtau beta cpd / dzh, (1 - beta) cpd / dzh, 1/(1 + dtau r), dtau beta / dz,
// dtau (1 - beta) / dz, Exner_ref
enum { CC_WU = 0, CC_WL, CC_CA, CC_CX, CC_DAMP, CC_DTBDZ, CC_DT1BDZ, CC_EXREF, CC_COUNT };

__global__ void k_mx_colconst(int N, int ld, const double* __restrict__ wu, const double* __restrict__ wl,
                              const double* __restrict__ dzh, const double* __restrict__ dz,
                              const double* __restrict__ ray, const double* __restrict__ ex_ref, double dtau,
                              double* __restrict__ cc) {
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    const bool interior = i > 0 && i < N;
    cc[CC_WU * ld + i] = i <= N ? wu[i] : 0.0;
    cc[CC_WL * ld + i] = i <= N ? wl[i] : 0.0;
    cc[CC_CA * ld + i] = interior ? dtau * kBeta * kCpd / dzh[i] : 0.0;
    cc[CC_CX * ld + i] = interior ? (1.0 - kBeta) * kCpd / dzh[i] : 0.0;
    cc[CC_DAMP * ld + i] = i <= N ? 1.0 / (1.0 + dtau * ray[i]) : 1.0;
    cc[CC_DTBDZ * ld + i] = i < N ? dtau * kBeta / dz[i] : 0.0;
    cc[CC_DT1BDZ * ld + i] = i < N ? dtau * (1.0 - kBeta) / dz[i] : 0.0;
    cc[CC_EXREF * ld + i] = i < N ? ex_ref[i] : 0.0;
  }
}

struct MxColArgs {
  // FP64 prognostics S^n, level-major [k][Nc]
  double *rho, *thv, *ex, *w;
  double* wflx;                            // level-major [h][Nc]
  // FP32 inputs
  const float *phi, *gth, *a_e;            // [Ne][ld]: rho_e vn, l_e rho_e vn theta_e, w-advection term
  const float* w_stage;                    // [Nc][ld] w shadow of the stage state
  float* Aw0;                              // level-major [h][Nc]
  // FP32 shadows written by this stage, [Nc][ld]
  float *rho32, *thv32, *exp32, *w32;
  const double* cc;                        // per-level constants for this dtau
  // parts of the column system frozen at S^n, written by the predictor and read by the
  // corrector (NULL: both stages compute them); level-major [field][level][Nc]
  double* fac64;
  // per-stage horizontal inputs of the column gathered by k_mx_gather_tile, level-major:
  // FP64 mass-flux divergence, FP32 heat-flux divergence, FP32 w-advection tendency
  // (already averaged with the predictor's in the corrector), and the Thomas scratch
  double* hdr;
  double* hdt;
  double* hdw;
  double* hdg;                             // predictor only: g = (Rd/cvd) pi/Theta of S^n
  const float *rho32n, *thv32n, *exp32n;   // FP32 shadows of S^n (for g)
  const float* exref32;
  double* dps;
  unsigned* status;
  double dtau, inv_nsub;
  // terrain-following levels (TOPO instances only): each cell's weights, 1/dz, 1/dzh and
  // reference Exner (FP64, level-major [k][Nc]), and the stage's FP32 wcc and w - wcc ([Nc][ld])
  const double *t_wu_lm, *t_idz_lm, *t_idzh_lm, *t_exref_lm;
  const float *t_wcc, *t_wcon;
};

__device__ inline bool finite64(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// the vertically implicit update of one column; CORR selects predictor (shadows of S*
// only) or corrector (FP64 S^{n+1} in place, shadows of S^{n+1}, vertical mass flux).
// TOPO (terrain-following levels): each cell's spacings and weights, the thickness-
// weighted horizontal divergences over the cell's dz, the explicit vertical fluxes with
// the contravariant (1 - beta) w - wcc, the vertical advection of w with w - wcc, the
// contravariant step-mean vertical flux, and the ground w of the stage (its wcc).
template <int NMAX, bool CORR, bool TOPO = false>
__device__ inline void mx_column_item(const MxGeo& G, const MxColArgs& a, int64_t c) {
  const int N = G.N, ld = G.ld;
  const int64_t nc = G.nc;
  const double dtau = a.dtau;
  const double* __restrict__ cc = a.cc;
  const int64_t o = c * ld;
#define LM(p, k) (p)[(int64_t)(k) * nc + c]
  int64_t E[3];
  float sg[3], kw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    sg[s] = G.s_ce32[3 * c + s];
    kw[s] = G.kin_w32[3 * c + s];
  }
  const double invA = G.inv_Ac[c];
  const float invA32 = (float)invA;
  const float dtau32 = (float)dtau;
  const double dwa[3] = {G.div_wa[3 * c], G.div_wa[3 * c + 1], G.div_wa[3 * c + 2]};

  double rho_ic[NMAX + 1], M[NMAX + 1], Thx[NMAX], exx[NMAX], rhox[NMAX], cp[NMAX], dp[NMAX];
  float gam[NMAX];
  // half-level interpolants of S^n
  double rho_m = LM(a.rho, 0), thv_m = LM(a.thv, 0);
  rho_ic[0] = rho_m;
  M[0] = rho_m * thv_m;
  for (int k = 1; k < N; ++k) {
    const double rho = LM(a.rho, k), thv = LM(a.thv, k);
    double wu, wl;
    if constexpr (TOPO) {
      wu = LM(a.t_wu_lm, k);
      wl = 1.0 - wu;
    } else {
      wu = cc[CC_WU * ld + k];
      wl = cc[CC_WL * ld + k];
    }
    const double ri = wu * rho_m + wl * rho;
    rho_ic[k] = ri;
    M[k] = ri * (wu * thv_m + wl * thv);
    rho_m = rho;
    thv_m = thv;
  }
  rho_ic[N] = rho_m;
  M[N] = rho_m * thv_m;
  // explicit predictors at full levels
  for (int k = 0; k < N; ++k) {
    // horizontal divergences: rho in FP64 from the FP32 mass fluxes (the values the
    // step-mean mass flux accumulates, so tracer transport sees the same divergence)
    const double Dr = (dwa[0] * f32_to_f64(a.phi[E[0] + k]) + dwa[1] * f32_to_f64(a.phi[E[1] + k])) +
                      dwa[2] * f32_to_f64(a.phi[E[2] + k]);
    const float Dt = (sg[0] * a.gth[E[0] + k] + sg[1] * a.gth[E[1] + k] + sg[2] * a.gth[E[2] + k]) * invA32;
    const double rho = LM(a.rho, k), thv = LM(a.thv, k), ex = LM(a.ex, k);
    const double w0 = LM(a.w, k), w1 = LM(a.w, k + 1);
    const double Th = rho * thv;
    double thx;
    float gfac;
    if constexpr (TOPO) {
      const double idz = LM(a.t_idz_lm, k);
      const double ve0 = k >= 1 ? (1.0 - kBeta) * w0 - f32_to_f64(a.t_wcc[o + k]) : 0.0;
      const double ve1 = k + 1 < N ? (1.0 - kBeta) * w1 - f32_to_f64(a.t_wcc[o + k + 1]) : 0.0;
      rhox[k] = rho - (dtau * ((Dr + rho_ic[k] * ve0) - rho_ic[k + 1] * ve1)) * idz;
      thx = Th - (f32_to_f64(dtau32 * Dt) + dtau * (M[k] * ve0 - M[k + 1] * ve1)) * idz;
      gfac = f64_to_f32(dtau * kBeta * idz);
    } else {
      const double dt1 = cc[CC_DT1BDZ * ld + k];
      rhox[k] = rho - dtau * Dr - dt1 * (rho_ic[k] * w0 - rho_ic[k + 1] * w1);
      thx = Th - f32_to_f64(dtau32 * Dt) - dt1 * (M[k] * w0 - M[k + 1] * w1);
      gfac = f64_to_f32(cc[CC_DTBDZ * ld + k]);
    }
    Thx[k] = thx;
    const float g = kRcvF * (f64_to_f32(ex) / f64_to_f32(Th));
    exx[k] = ex + f32_to_f64(g) * (thx - Th);
    gam[k] = g * gfac;
  }
  // tridiagonal system at interior half levels, Thomas forward sweep
  double thv_m1 = LM(a.thv, 0), ex_m1 = LM(a.ex, 0);
  for (int h = 1; h < N; ++h) {
    const float hadv = kw[0] * a.a_e[E[0] + h] + kw[1] * a.a_e[E[1] + h] + kw[2] * a.a_e[E[2] + h];
    const float ws = a.w_stage[o + h];
    const double idzh = TOPO ? LM(a.t_idzh_lm, h) : 0.0;
    float Aw;
    if constexpr (TOPO)
      Aw = -hadv - a.t_wcon[o + h] * (a.w_stage[o + h - 1] - a.w_stage[o + h + 1]) * f64_to_f32(0.5 * idzh);
    else
      Aw = -hadv - ws * (a.w_stage[o + h - 1] - a.w_stage[o + h + 1]) * G.inv_dz2_32[h];
    if (CORR) Aw = 0.5f * (LM(a.Aw0, h) + Aw);
    else LM(a.Aw0, h) = Aw;
    const double thv_h = LM(a.thv, h), ex_h = LM(a.ex, h);
    double th_ic, cx, ca;
    if constexpr (TOPO) {
      const double wu = LM(a.t_wu_lm, h);
      th_ic = wu * thv_m1 + (1.0 - wu) * thv_h;
      cx = (1.0 - kBeta) * kCpd * idzh;
      ca = dtau * kBeta * kCpd * idzh;
    } else {
      th_ic = cc[CC_WU * ld + h] * thv_m1 + cc[CC_WL * ld + h] * thv_h;
      cx = cc[CC_CX * ld + h];
      ca = cc[CC_CA * ld + h];
    }
    const double wx = LM(a.w, h) + dtau * (f32_to_f64(Aw) - cx * th_ic * (ex_m1 - ex_h) - kGrav);
    const double aa = ca * th_ic;
    const double gm = f32_to_f64(gam[h - 1]), gk = f32_to_f64(gam[h]);
    const double lower = -aa * gm * M[h - 1];
    const double diag = 1.0 + aa * (gm + gk) * M[h];
    const double upper = -aa * gk * M[h + 1];
    const double rhs = wx - aa * (exx[h - 1] - exx[h]);
    const int i = h - 1;
    if (i == 0) {
      const double r = recip64(diag);
      cp[0] = upper * r;
      dp[0] = rhs * r;
    } else {
      const double r = recip64(diag - lower * cp[i - 1]);
      cp[i] = upper * r;
      dp[i] = (rhs - lower * dp[i - 1]) * r;
    }
    thv_m1 = thv_h;
    ex_m1 = ex_h;
  }
  for (int i = N - 3; i >= 0; --i) dp[i] = dp[i] - cp[i] * dp[i + 1];
  // updates
  double wn_prev = 0.0;
  bool ok = true;
  for (int k = 0; k < N; ++k) {
    const int h1 = k + 1;
    const double wn1 = (h1 < N) ? dp[h1 - 1] * cc[CC_DAMP * ld + h1] : 0.0;
    const double dtb = TOPO ? dtau * kBeta * LM(a.t_idz_lm, k) : cc[CC_DTBDZ * ld + k];
    const double exref = TOPO ? LM(a.t_exref_lm, k) : cc[CC_EXREF * ld + k];
    if (CORR) {
      const double q = M[k] * wn_prev - M[k + 1] * wn1;
      const double r = rho_ic[k] * wn_prev - rho_ic[k + 1] * wn1;
      const double Th_n = Thx[k] - dtb * q;
      const double ex_n = exx[k] - f32_to_f64(gam[k]) * q;
      const double rho_n = rhox[k] - dtb * r;
      const double thv_n = Th_n * recip64(rho_n);
      const double wold = LM(a.w, k);
      double wc = kBeta * wn_prev + (1.0 - kBeta) * wold;
      if constexpr (TOPO) wc -= k >= 1 ? f32_to_f64(a.t_wcc[o + k]) : 0.0;
      LM(a.wflx, k) += rho_ic[k] * wc * a.inv_nsub;
      LM(a.rho, k) = rho_n;
      LM(a.thv, k) = thv_n;
      LM(a.ex, k) = ex_n;
      LM(a.w, k) = wn_prev;
      a.thv32[o + k] = f64_to_f32(thv_n);
      a.rho32[o + k] = f64_to_f32(rho_n);
      a.exp32[o + k] = f64_to_f32(ex_n - exref);
      ok = ok && finite64(thv_n) && finite64(ex_n) && finite64(wn_prev);
    } else {
      // provisional state: FP32 shadows formed in FP32 from the FP64 solve (as in the
      // stored-factor path)
      const float wf = f64_to_f32(wn_prev), wf1 = f64_to_f32(wn1), dtb32 = f64_to_f32(dtb);
      const float q = f64_to_f32(M[k]) * wf - f64_to_f32(M[k + 1]) * wf1;
      const float r = f64_to_f32(rho_ic[k]) * wf - f64_to_f32(rho_ic[k + 1]) * wf1;
      const float Th_n = f64_to_f32(Thx[k]) - dtb32 * q;
      const float exp_n = f64_to_f32(exx[k] - exref) - gam[k] * q;
      const float rho_n = f64_to_f32(rhox[k]) - dtb32 * r;
      const float thv_n = Th_n / rho_n;
      a.thv32[o + k] = thv_n;
      a.rho32[o + k] = rho_n;
      a.exp32[o + k] = exp_n;
      ok = ok && isfinite(thv_n) && isfinite(exp_n) && finite64(wn_prev);
    }
    a.w32[o + k] = f64_to_f32(wn_prev);
    wn_prev = wn1;
  }
  if constexpr (TOPO) {
    // ground: no flux through it; w there is the stage's terrain-following value
    a.w32[o + N] = a.t_wcc[o + N];
    if (CORR) LM(a.w, N) = f32_to_f64(a.t_wcc[o + N]);
  } else {
    a.w32[o + N] = 0.0f;
    if (CORR) {
      LM(a.wflx, N) += rho_ic[N] * ((1.0 - kBeta) * LM(a.w, N)) * a.inv_nsub;
      LM(a.w, N) = 0.0;
    }
  }
  if (!ok) atomicOr(a.status, 1u);
#undef LM
}

// ---- column solve with the frozen parts stored by the predictor and reused by the corrector
//
// The tridiagonal matrix, its LU factors, the explicit (1 - beta) vertical fluxes and the
// hydrostatic part of the w predictor depend only on S^n and dtau, which both stages
// share. The predictor computes them once, in a single downward sweep that also
// eliminates its own right-hand side, and stores them level-major; the corrector reads
// them and only forms its right-hand side, substitutes and updates. FP64 instructions
// per cell-level (ncu): 43 in the predictor and 29 in the corrector, against 48 and 65
// when both stages compute everything.
enum { F_LO = 0, F_RP, F_CP, F_WX, F_AA, F_M, F_RI, F_RX, F_TX, F_PX, F_GD, F_GAM, F_COUNT64 };  // FP64 [f][h][Nc]

template <int NMAX, bool CORR>
__device__ inline void mx_column_fac_item(const MxGeo& G, const MxColArgs& a, int64_t c) {
  const int N = G.N, ld = G.ld;
  const int64_t nc = G.nc, o = c * ld, H = N + 1;
  const double dtau = a.dtau;
  const double* __restrict__ cc = a.cc;
  double* __restrict__ fac = a.fac64;
  double* __restrict__ dps = a.dps;
  const double* __restrict__ hdr = a.hdr;
  const double* __restrict__ hdt = a.hdt;
  const double* __restrict__ hdw = a.hdw;
#define LM(p, k) (p)[(int64_t)(k) * nc + c]
#define F64(f, k) fac[((int64_t)(f) * H + (k)) * nc + c]
  if (!CORR) {
    // ---- predictor: one downward sweep; at step j half level j becomes known, which
    // completes full level j-1 and the tridiagonal row of half level j-1
    const double* __restrict__ rhoS = a.rho;
    const double* __restrict__ thvS = a.thv;
    const double* __restrict__ exS = a.ex;
    const double* __restrict__ wS = a.w;
    const double* __restrict__ hdg = a.hdg;
    double rho1 = 0, thv1 = 0, ex1 = 0, Th1 = 0;    // full level j-1
    double ex2 = 0;                                  // full level j-2
    double ri1 = 0, M1 = 0, w1 = 0, ti1 = 0;         // half level j-1 (ti = theta_v interpolant)
    double M2 = 0;                                   // half level j-2
    double gam2 = 0.0, exx2 = 0.0;                   // full level j-2
    double cp_prev = 0.0, dp_prev = 0.0;
    for (int j = 0; j <= N; ++j) {
      double rho = 0, thv = 0, ex = 0, ri, ti;
      if (j < N) {
        rho = LM(rhoS, j);
        thv = LM(thvS, j);
        ex = LM(exS, j);
      }
      if (j == 0) {
        ri = rho;
        ti = thv;
      } else if (j == N) {
        ri = rho1;
        ti = thv1;
      } else {
        const double wu = cc[CC_WU * ld + j], wl = cc[CC_WL * ld + j];
        ri = wu * rho1 + wl * rho;
        ti = wu * thv1 + wl * thv;
      }
      const double Mh = ri * ti;
      const double wh = (j == 0 || j == N) ? 0.0 : LM(wS, j);
      F64(F_M, j) = Mh;
      F64(F_RI, j) = ri;
      double gam1 = 0.0, exx1 = 0.0;
      if (j >= 1) {
        const int k = j - 1;                         // full level k: half levels k and k+1
        const double dt1 = cc[CC_DT1BDZ * ld + k];
        const double rxv = rho1 - dt1 * (ri1 * w1 - ri * wh);
        const double txv = Th1 - dt1 * (M1 * w1 - Mh * wh);
        const double g = LM(hdg, k);
        const double pxv = ex1 + g * (txv - Th1);
        const double gd = g * dtau;
        gam1 = g * cc[CC_DTBDZ * ld + k];
        F64(F_RX, k) = rxv;
        F64(F_TX, k) = txv;
        F64(F_PX, k) = pxv;
        F64(F_GD, k) = gd;
        F64(F_GAM, k) = gam1;
        exx1 = pxv - gd * LM(hdt, k);
        if (k >= 1) {                                // row of half level h = k (interpolants ti1, M2..Mh)
          const int h = k;
          const double wexp = w1 + dtau * (-cc[CC_CX * ld + h] * ti1 * (ex2 - ex1) - kGrav);
          const double aa = cc[CC_CA * ld + h] * ti1;
          const double lo = -aa * gam2 * M2;
          const double diag = 1.0 + aa * (gam2 + gam1) * M1;
          const double up = -aa * gam1 * Mh;
          const double rp = recip64(diag - lo * cp_prev);
          const double cpv = up * rp;
          F64(F_LO, h) = lo;
          F64(F_RP, h) = rp;
          F64(F_CP, h) = cpv;
          F64(F_WX, h) = wexp;
          F64(F_AA, h) = aa;
          const double rhs = wexp + dtau * LM(hdw, h) - aa * (exx2 - exx1);
          const double dpv = (rhs - lo * dp_prev) * rp;
          LM(dps, h) = dpv;
          cp_prev = cpv;
          dp_prev = dpv;
        }
      }
      ex2 = ex1;
      gam2 = gam1;
      exx2 = exx1;
      M2 = M1;
      ri1 = ri;
      M1 = Mh;
      w1 = wh;
      ti1 = ti;
      rho1 = rho;
      thv1 = thv;
      ex1 = ex;
      Th1 = rho * thv;
    }
  } else {
    // ---- corrector: stage right-hand side with the stored rows and factors
    double dp_prev = 0.0, exx_prev = 0.0;
    #pragma unroll 4   // lets the loads of four levels overlap (latency bound)
    for (int k = 0; k < N; ++k) {
      const double exx = F64(F_PX, k) - F64(F_GD, k) * LM(hdt, k);
      if (k >= 1) {
        const int h = k;
        const double rhs = F64(F_WX, h) + dtau * LM(hdw, h) - F64(F_AA, h) * (exx_prev - exx);
        const double dpv = (rhs - F64(F_LO, h) * dp_prev) * F64(F_RP, h);
        LM(dps, h) = dpv;
        dp_prev = dpv;
      }
      exx_prev = exx;
    }
  }
  // ---- upward sweep: back substitution, Rayleigh damping, updates of full level h
  double* __restrict__ rho_io = a.rho;
  double* __restrict__ thv_io = a.thv;
  double* __restrict__ ex_io = a.ex;
  double* __restrict__ w_io = a.w;
  double* __restrict__ wflx_io = a.wflx;
  float* __restrict__ rho32 = a.rho32;
  float* __restrict__ thv32 = a.thv32;
  float* __restrict__ exp32 = a.exp32;
  float* __restrict__ w32 = a.w32;
  bool ok = true;
  if (CORR) {
    double x_next = 0.0, w_next = 0.0;               // half level h+1 (undamped, damped)
    double M_next = F64(F_M, N), ri_next = F64(F_RI, N);
    #pragma unroll 4   // lets the loads of four levels overlap (latency bound)
    for (int h = N - 1; h >= 0; --h) {
      double x = 0.0, w = 0.0;
      if (h >= 1) {
        x = LM(dps, h) - F64(F_CP, h) * x_next;
        w = x * cc[CC_DAMP * ld + h];
      }
      const double Mk = F64(F_M, h), rk = F64(F_RI, h);
      const double q = Mk * w - M_next * w_next;
      const double r = rk * w - ri_next * w_next;
      const double dtb = cc[CC_DTBDZ * ld + h];
      const double Dt = LM(hdt, h);
      const double Th_n = (F64(F_TX, h) - dtau * Dt) - dtb * q;
      const double ex_n = (F64(F_PX, h) - F64(F_GD, h) * Dt) - F64(F_GAM, h) * q;
      const double rho_n = (F64(F_RX, h) - dtau * LM(hdr, h)) - dtb * r;
      const double thv_n = Th_n * recip64(rho_n);
      const double wold = LM(w_io, h);
      LM(wflx_io, h) += rk * (kBeta * w + (1.0 - kBeta) * wold) * a.inv_nsub;
      LM(rho_io, h) = rho_n;
      LM(thv_io, h) = thv_n;
      LM(ex_io, h) = ex_n;
      LM(w_io, h) = w;
      thv32[o + h] = f64_to_f32(thv_n);
      rho32[o + h] = f64_to_f32(rho_n);
      exp32[o + h] = f64_to_f32(ex_n - cc[CC_EXREF * ld + h]);
      w32[o + h] = f64_to_f32(w);
      ok = ok && finite64(thv_n) && finite64(ex_n) && finite64(w);
      x_next = x;
      w_next = w;
      M_next = Mk;
      ri_next = rk;
    }
  } else {
    // The predictor's S* exists only as the FP32 shadows the corrector's stencils read:
    // the back substitution and damping stay FP64, the implicit increments of rho,
    // Theta and pi are formed in FP32 from the FP64 explicit parts (pi relative to
    // its reference profile in FP64 first, since pi - pi_ref is what is stored).
    const float dtau32 = f64_to_f32(dtau);
    double x_next = 0.0;
    float w_next = 0.0f, M_next = f64_to_f32(F64(F_M, N)), ri_next = f64_to_f32(F64(F_RI, N));
    for (int h = N - 1; h >= 0; --h) {
      double x = 0.0, w = 0.0;
      if (h >= 1) {
        x = LM(dps, h) - F64(F_CP, h) * x_next;
        w = x * cc[CC_DAMP * ld + h];
      }
      const float w_f = f64_to_f32(w);
      const float Mk = f64_to_f32(F64(F_M, h)), rk = f64_to_f32(F64(F_RI, h));
      const float q = Mk * w_f - M_next * w_next;
      const float r = rk * w_f - ri_next * w_next;
      const float dtb = f64_to_f32(cc[CC_DTBDZ * ld + h]);
      const float Dt = f64_to_f32(LM(hdt, h));
      const float Th_n = (f64_to_f32(F64(F_TX, h)) - dtau32 * Dt) - dtb * q;
      const float exp_n = (f64_to_f32(F64(F_PX, h) - cc[CC_EXREF * ld + h]) - f64_to_f32(F64(F_GD, h)) * Dt) -
                          f64_to_f32(F64(F_GAM, h)) * q;
      const float rho_n = (f64_to_f32(F64(F_RX, h)) - dtau32 * f64_to_f32(LM(hdr, h))) - dtb * r;
      thv32[o + h] = Th_n / rho_n;
      rho32[o + h] = rho_n;
      exp32[o + h] = exp_n;
      w32[o + h] = w_f;
      ok = ok && isfinite(Th_n / rho_n) && isfinite(exp_n) && finite64(w);
      x_next = x;
      w_next = w_f;
      M_next = Mk;
      ri_next = rk;
    }
  }
  w32[o + N] = 0.0f;
  if (!ok) atomicOr(a.status, 1u);
#undef LM
#undef F64
}

template <int NMAX, bool CORR>
__device__ inline void mx_column_any(const MxGeo& G, const MxColArgs& a, int64_t c) {
  if (a.fac64) mx_column_fac_item<NMAX, CORR>(G, a, c);
  else mx_column_item<NMAX, CORR>(G, a, c);
}

// diffusion of theta_v for one column: FP32 increment, FP64 accumulation, Exner at
// constant density, shadows refreshed
// (exref_c: the per-cell reference of terrain-following levels, [Nc][ld], or NULL)
__device__ inline void mx_diff_theta_item(const MxGeo& G, const float* __restrict__ thflx, double* __restrict__ thv,
                                          double* __restrict__ ex, float* __restrict__ thv32, float* __restrict__ exp32,
                                          float dt, int64_t c, const double* __restrict__ exref_c = nullptr) {
  const int64_t nc = G.nc;
  const int ld = G.ld;
  int64_t E[3];
  float sg[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    sg[s] = G.s_ce32[3 * c + s];
  }
  const float dtA = dt * (float)G.inv_Ac[c];
  for (int k = 0; k < G.N; ++k) {
    const float dth = dtA * (sg[0] * thflx[E[0] + k] + sg[1] * thflx[E[1] + k] + sg[2] * thflx[E[2] + k]);
    const int64_t i = (int64_t)k * nc + c;
    const double th = thv[i];
    const double th_n = th + f32_to_f64(dth);
    const double ex_n = ex[i] + ex[i] * f32_to_f64(kRcvF * dth / f64_to_f32(th));
    thv[i] = th_n;
    ex[i] = ex_n;
    thv32[c * ld + k] = f64_to_f32(th_n);
    exp32[c * ld + k] = f64_to_f32(ex_n - (exref_c ? exref_c[c * ld + k] : G.ex_ref[k]));
  }
}

// ---------------------------------------------------------------- per-state kernels

// warp w, lanes [sub*LPE, (sub+1)*LPE) handle entity w * (32/LPE) + sub
#define ITEM_PROLOGUE(LPE, COUNT)                                                        \
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;             \
  const int64_t item = gw * (32 / (LPE)) + (int64_t)((threadIdx.x & 31) / (LPE));        \
  const int lane = (int)(threadIdx.x & ((LPE) - 1));                                     \
  if (item >= (COUNT)) return;

template <int LPE>
__global__ void __launch_bounds__(512) k_mx_vertex(MxGeo G, const float* vn, const float* w, float* zeta, float* w_v) {
  ITEM_PROLOGUE(LPE, G.nv)
  mx_vertex_item<LPE>(G, vn, w, zeta, w_v, item, lane);
}
template <int LPE>
__global__ void __launch_bounds__(512) k_mx_edge_diag(MxGeo G, const float* vn, float* vt) {
  ITEM_PROLOGUE(LPE, G.ne)
  mx_edge_diag_item<LPE>(G, vn, vt, item, lane);
}
template <int LPE>
__global__ void __launch_bounds__(512) k_mx_cell_ke(MxGeo G, const float* vn, const float* vt, float* Kc) {
  ITEM_PROLOGUE(LPE, G.nc)
  mx_cell_ke_item<LPE>(G, vn, vt, Kc, item, lane);
}
template <int LPE, bool TOPO = false>
__global__ void __launch_bounds__(512, 2) k_mx_edge_tend(MxGeo G, MxEdgeArgs a) {
  ITEM_PROLOGUE(LPE, G.ne)
  mx_edge_tend_item<LPE, TOPO>(G, a, item, lane);
}
template <int LPE>
__global__ void __launch_bounds__(512, 2) k_mx_diff_vertex(MxGeo G, const float* vn, float* ux, float* uy, float* uz,
                                                        float* zeta, float* divc) {
  // vertices first, then cells (divergence): both only read vn
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t item = gw * (32 / LPE) + (int64_t)((threadIdx.x & 31) / LPE);
  const int lane = (int)(threadIdx.x & (LPE - 1));
  if (item < G.nv) mx_diff_vertex_item<LPE>(G, vn, ux, uy, uz, zeta, item, lane);
  else if (item < G.nv + G.nc) mx_diff_div_item<LPE>(G, vn, divc, item - G.nv, lane);
}
template <int LPE>
__global__ void __launch_bounds__(512) k_mx_diff_edge(MxGeo G, float* vn, const float* ux, const float* uy,
                                                      const float* uz, const float* zeta, const float* divc,
                                                      const float* thv, float* thflx, float dt) {
  ITEM_PROLOGUE(LPE, G.ne)
  mx_diff_edge_item<LPE>(G, vn, ux, uy, uz, zeta, divc, thv, thflx, dt, item, lane);
}
// Gather step of the stored-factor column path for one state: a block takes 32
// consecutive cells and walks the levels in chunks of LPE; lane groups of LPE
// threads compute one cell's chunk (coalesced reads of its edge and cell rows), the
// results are transposed through shared memory and written level-major as 32
// consecutive cells per level (whole 128/256-byte lines instead of scattered words).
constexpr int kGatherCells = 32;
template <int LPE>
struct GatherTile {
  double sh[4][LPE][kGatherCells + 1];                 // hdr, hdt, hdg, hdw
  float sa[LPE][kGatherCells + 1];                     // Aw0
};

// one tile of 32 cells starting at c0; every thread of the block takes part
template <int LPE, bool CORR>
__device__ inline void mx_gather_tile_body(const MxGeo& G, const MxColArgs& a, int64_t c0, GatherTile<LPE>& T) {
  constexpr int CB = kGatherCells;
  auto& sh = T.sh;
  auto& sa = T.sa;
  const int N = G.N, ld = G.ld;
  const int64_t nc = G.nc;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int grp = tid / LPE, ngrp = nthr / LPE, lane = tid % LPE;
  for (int k0 = 0; k0 < N; k0 += LPE) {
    if (CORR) {
      for (int i = tid; i < LPE * CB; i += nthr) {
        const int r = i / CB, cl = i % CB, h = k0 + r;
        const int64_t c = c0 + cl;
        sa[r][cl] = (h >= 1 && h < N && c < nc) ? a.Aw0[(int64_t)h * nc + c] : 0.0f;
      }
      __syncthreads();
    }
    for (int cl = grp; cl < CB; cl += ngrp) {
      const int64_t c = c0 + cl;
      if (c >= nc) break;
      const int64_t o = c * ld;
      int64_t E[3];
      float sg[3], kw[3];
      for (int s = 0; s < 3; ++s) {
        E[s] = (int64_t)G.c2e[3 * c + s] * ld;
        sg[s] = G.s_ce32[3 * c + s];
        kw[s] = G.kin_w32[3 * c + s];
      }
      const double invA = G.inv_Ac[c];
      const float invA32 = (float)invA;
      const double dwa[3] = {G.div_wa[3 * c], G.div_wa[3 * c + 1], G.div_wa[3 * c + 2]};
      const int k = k0 + lane;
      if (k < N) {
        sh[0][lane][cl] = (dwa[0] * f32_to_f64(a.phi[E[0] + k]) + dwa[1] * f32_to_f64(a.phi[E[1] + k])) +
                          dwa[2] * f32_to_f64(a.phi[E[2] + k]);
        sh[1][lane][cl] =
            f32_to_f64((sg[0] * a.gth[E[0] + k] + sg[1] * a.gth[E[1] + k] + sg[2] * a.gth[E[2] + k]) * invA32);
        if (!CORR) {
          const float pi = a.exp32n[o + k] + a.exref32[k];
          sh[2][lane][cl] = f32_to_f64(kRcvF * (pi / (a.rho32n[o + k] * a.thv32n[o + k])));
        }
      }
      if (k >= 1 && k < N) {
        const float hadv = kw[0] * a.a_e[E[0] + k] + kw[1] * a.a_e[E[1] + k] + kw[2] * a.a_e[E[2] + k];
        const float ws = a.w_stage[o + k];
        float Aw = -hadv - ws * (a.w_stage[o + k - 1] - a.w_stage[o + k + 1]) * G.inv_dz2_32[k];
        if (CORR) Aw = 0.5f * (sa[lane][cl] + Aw);
        else sa[lane][cl] = Aw;
        sh[3][lane][cl] = f32_to_f64(Aw);
      }
    }
    __syncthreads();
    for (int i = tid; i < LPE * CB; i += nthr) {
      const int r = i / CB, cl = i % CB, k = k0 + r;
      const int64_t c = c0 + cl;
      if (c >= nc) continue;
      const int64_t j = (int64_t)k * nc + c;
      if (k < N) {
        a.hdr[j] = sh[0][r][cl];
        a.hdt[j] = sh[1][r][cl];
        if (!CORR) a.hdg[j] = sh[2][r][cl];
      }
      if (k >= 1 && k < N) {
        a.hdw[j] = sh[3][r][cl];
        if (!CORR) a.Aw0[j] = sa[r][cl];
      }
    }
    __syncthreads();
  }
}

// the diffusion edge step with fourth-order background diffusion (option): 32 lanes per edge
__global__ void __launch_bounds__(256) k_mx_diff_edge_bd(MxGeo G, float* vn, const float* ux, const float* uy,
                                                         const float* uz, const float* zeta, const float* divc,
                                                         const float* thv, float* thflx, float dt, const float* D1,
                                                         const float* zeta1, float bd_scale) {
  const int64_t e = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (e >= G.ne) return;
  mx_diff_edge_item<32>(G, vn, ux, uy, uz, zeta, divc, thv, thflx, dt, e, threadIdx.x & 31, D1, zeta1, bd_scale);
}

template <int LPE, bool CORR>
__global__ void __launch_bounds__(512, 3) k_mx_gather_tile(MxGeo G, MxColArgs a) {
  __shared__ GatherTile<LPE> T;
  mx_gather_tile_body<LPE, CORR>(G, a, (int64_t)blockIdx.x * kGatherCells, T);
}

// ---- corrector of the stored-factor column for one state, in two launches. Its only
// sequential parts are the forward elimination of the right-hand side and the back
// substitution; everything else is parallel over the levels.
//   k_mx_corr_solve   one thread per column: right-hand side from the stored rows, forward
//                     elimination with the stored factors, back substitution, damping; the
//                     damped w overwrites the Thomas scratch (level-major, coalesced).
//   k_mx_corr_update  one element per (cell, level), 32 cells by a chunk of levels per
//                     block: the FP64 updates of S^{n+1} and the vertical mass flux from
//                     level-major operands, the FP32 shadows transposed through shared
//                     memory into the cells' [c][ld] rows.
// Same arithmetic as the corrector branch of mx_column_fac_item (which the persistent
// ensemble keeps in one pass).
__device__ inline void mx_corr_solve_item(const MxGeo& G, const MxColArgs& a, int64_t c) {
  const int N = G.N, ld = G.ld;
  const int64_t nc = G.nc, H = N + 1;
  const double dtau = a.dtau;
  const double* __restrict__ cc = a.cc;
  const double* __restrict__ fac = a.fac64;
  double* __restrict__ dps = a.dps;
  const double* __restrict__ hdt = a.hdt;
  const double* __restrict__ hdw = a.hdw;
#define LM(p, k) (p)[(int64_t)(k) * nc + c]
#define F64(f, k) fac[((int64_t)(f) * H + (k)) * nc + c]
  double dp_prev = 0.0, exx_prev = 0.0;
#pragma unroll 4
  for (int k = 0; k < N; ++k) {
    const double exx = F64(F_PX, k) - F64(F_GD, k) * LM(hdt, k);
    if (k >= 1) {
      const double rhs = F64(F_WX, k) + dtau * LM(hdw, k) - F64(F_AA, k) * (exx_prev - exx);
      const double dpv = (rhs - F64(F_LO, k) * dp_prev) * F64(F_RP, k);
      LM(dps, k) = dpv;
      dp_prev = dpv;
    }
    exx_prev = exx;
  }
  double x_next = 0.0;
#pragma unroll 4
  for (int h = N - 1; h >= 1; --h) {
    const double x = LM(dps, h) - F64(F_CP, h) * x_next;
    LM(dps, h) = x * cc[CC_DAMP * ld + h];
    x_next = x;
  }
#undef LM
#undef F64
}

__global__ void __launch_bounds__(128) k_mx_corr_solve(MxGeo G, MxColArgs a) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < G.nc) mx_corr_solve_item(G, a, c);
}

constexpr int kUpdCells = 32, kUpdLevels = 32;
struct UpdTile {
  float sf[4][kUpdLevels][kUpdCells + 1];              // theta_v, rho, pi - pi_ref, w
};

// one tile of 32 cells starting at c0; every thread of the block takes part (a multiple
// of 32 threads); returns false if a non-finite value appeared
__device__ inline bool mx_corr_update_tile(const MxGeo& G, const MxColArgs& a, int64_t c0, UpdTile& T) {
  auto& sf = T.sf;
  const int N = G.N, ld = G.ld;
  const int64_t nc = G.nc, H = N + 1;
  const double dtau = a.dtau;
  const double* __restrict__ cc = a.cc;
  const double* __restrict__ fac = a.fac64;
  const double* __restrict__ wd = a.dps;               // damped w^{n+1}, half levels 1..N-1
  const double* __restrict__ hdt = a.hdt;
  const double* __restrict__ hdr = a.hdr;
  double* __restrict__ rho_io = a.rho;
  double* __restrict__ thv_io = a.thv;
  double* __restrict__ ex_io = a.ex;
  double* __restrict__ w_io = a.w;
  double* __restrict__ wflx_io = a.wflx;
  const int tid = threadIdx.x, cl = tid % kUpdCells, r0 = tid / kUpdCells, nr = blockDim.x / kUpdCells;
  const int64_t c = c0 + cl;
  bool ok = true;
  for (int k0 = 0; k0 < N; k0 += kUpdLevels) {
    for (int r = r0; r < kUpdLevels; r += nr) {
      const int h = k0 + r;
      if (h >= N || c >= nc) continue;
#define LM(p, k) (p)[(int64_t)(k) * nc + c]
#define F64(f, k) fac[((int64_t)(f) * H + (k)) * nc + c]
      const double w = h >= 1 ? LM(wd, h) : 0.0;
      const double w1 = h + 1 < N ? LM(wd, h + 1) : 0.0;
      const double Mk = F64(F_M, h), rk = F64(F_RI, h);
      const double q = Mk * w - F64(F_M, h + 1) * w1;
      const double rr = rk * w - F64(F_RI, h + 1) * w1;
      const double dtb = cc[CC_DTBDZ * ld + h];
      const double Dt = LM(hdt, h);
      const double Th_n = (F64(F_TX, h) - dtau * Dt) - dtb * q;
      const double ex_n = (F64(F_PX, h) - F64(F_GD, h) * Dt) - F64(F_GAM, h) * q;
      const double rho_n = (F64(F_RX, h) - dtau * LM(hdr, h)) - dtb * rr;
      const double thv_n = Th_n * recip64(rho_n);
      const double wold = LM(w_io, h);
      LM(wflx_io, h) += rk * (kBeta * w + (1.0 - kBeta) * wold) * a.inv_nsub;
      LM(rho_io, h) = rho_n;
      LM(thv_io, h) = thv_n;
      LM(ex_io, h) = ex_n;
      LM(w_io, h) = w;
      sf[0][r][cl] = f64_to_f32(thv_n);
      sf[1][r][cl] = f64_to_f32(rho_n);
      sf[2][r][cl] = f64_to_f32(ex_n - cc[CC_EXREF * ld + h]);
      sf[3][r][cl] = f64_to_f32(w);
      ok = ok && finite64(thv_n) && finite64(ex_n) && finite64(w);
#undef LM
#undef F64
    }
    __syncthreads();
    // shadows: each warp writes whole level runs of its cells' [c][ld] rows
    const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    for (int j = warp; j < kUpdCells; j += nwarp) {
      const int64_t cj = c0 + j;
      const int h = k0 + lane;
      if (cj >= nc || h >= N) continue;
      const int64_t o = cj * ld + h;
      a.thv32[o] = sf[0][lane][j];
      a.rho32[o] = sf[1][lane][j];
      a.exp32[o] = sf[2][lane][j];
      a.w32[o] = sf[3][lane][j];
    }
    __syncthreads();
  }
  if (tid < kUpdCells && c < nc) a.w32[c * ld + N] = 0.0f;
  return ok;
}

__global__ void __launch_bounds__(256) k_mx_corr_update(MxGeo G, MxColArgs a) {
  __shared__ UpdTile T;
  const bool ok = mx_corr_update_tile(G, a, (int64_t)blockIdx.x * kUpdCells, T);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(a.status, 1u);
}

template <int NMAX, bool CORR, bool TOPO = false>
__global__ void __launch_bounds__(128) k_mx_column(MxGeo G, MxColArgs a) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.nc) return;
  if constexpr (TOPO) mx_column_item<NMAX, CORR, true>(G, a, c);     // always recomputes its factors
  else mx_column_any<NMAX, CORR>(G, a, c);
}
__global__ void __launch_bounds__(128) k_mx_diff_theta(MxGeo G, const float* thflx, double* thv, double* ex,
                                                       float* thv32, float* exp32, float dt, const double* exref_c) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < G.nc) mx_diff_theta_item(G, thflx, thv, ex, thv32, exp32, dt, c, exref_c);
}

// ---------------------------------------------------------------- lean column (flat levels)
//
// The column of a mixed-precision state on flat levels in the fewest FP64 operations the
// precision split allows. FP64 stays where the method needs it:
//  * the hydrostatic residual of S^n in the w equation (a difference of two terms of size
//    g), taken once per substep into the stage-independent base of the right-hand side
//        B_h = w_h - dtau (cpd theta_ic,h (pi_{h-1} - pi_h) / dzh_h + g),
//    with theta_ic in FP64;
//  * the forward elimination and the back substitution of the tridiagonal w system;
//  * the density update in flux form: the horizontal divergence of the FP32 mass fluxes
//    summed with FP64 weights (gathered per stage), the vertical flux through each half
//    level one FP32 number, differenced in FP64 (exact) and scaled in FP64, so the column
//    and the global mass are conserved to FP64 rounding and the step-mean flux reproduces
//    the density change;
//  * the FP64 prognostics of S^{n+1} (rho, theta_v, Exner, w) and the step-mean vertical
//    mass flux, each updated by one FP64 add.
// Everything that only scales a small increment is FP32: the matrix rows and their LU
// factors, the explicit (1 - beta) fluxes and the state-equation factor (Rd/cvd) pi/Theta,
// the stage part of the right-hand side dtau A_w - a_h (dpi_{h-1} - dpi_h), and the
// increments of Theta and Exner. The FP32 shadows are written through a per-warp
// shared-memory transpose as whole level runs of each cell's [c][ld] row.
// Per cell-level-substep: 6 (B) + 4 (elimination, substitution) + 1 (shadow) in the
// predictor, 4 + 3 (density) + 1 (flux) + 2 (theta_v, Exner) + 1 (shadow) in the corrector,
// plus 3 for the corrector's FP64 divergence: 26 FP64 instructions.

// per-level constants of the lean column for one dtau: FP64 [LD_COUNT][ld], FP32 [LF_COUNT][ld]
enum { LD_WU = 0, LD_WL, LD_CPDZH, LD_IDZ, LD_DAMP, LD_EXREF, LD_COUNT };
enum { LF_WU = 0, LF_WL, LF_CA, LF_DT1, LF_DTB, LF_COUNT };

__global__ void k_mx_leanconst(int N, int ld, const double* __restrict__ wu, const double* __restrict__ wl,
                               const double* __restrict__ dzh, const double* __restrict__ dz,
                               const double* __restrict__ ray, const double* __restrict__ ex_ref, double dtau,
                               double* __restrict__ cd, float* __restrict__ cf) {
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    const bool interior = i > 0 && i < N;
    cd[LD_WU * ld + i] = interior ? wu[i] : 0.0;
    cd[LD_WL * ld + i] = interior ? wl[i] : 0.0;
    cd[LD_CPDZH * ld + i] = interior ? kCpd / dzh[i] : 0.0;
    cd[LD_IDZ * ld + i] = i < N ? dtau / dz[i] : 0.0;
    cd[LD_DAMP * ld + i] = i <= N ? 1.0 / (1.0 + dtau * ray[i]) : 1.0;
    cd[LD_EXREF * ld + i] = i < N ? ex_ref[i] : 0.0;
    cf[LF_WU * ld + i] = interior ? (float)wu[i] : 0.0f;
    cf[LF_WL * ld + i] = interior ? (float)wl[i] : 0.0f;
    cf[LF_CA * ld + i] = interior ? (float)(dtau * kBeta * kCpd / dzh[i]) : 0.0f;
    cf[LF_DT1 * ld + i] = i < N ? (float)(dtau * (1.0 - kBeta) / dz[i]) : 0.0f;
    cf[LF_DTB * ld + i] = i < N ? (float)(dtau * kBeta / dz[i]) : 0.0f;
  }
}

struct MxLeanArgs {
  // FP64 prognostics S^n (level-major [k][Nc]; updated in place by the corrector)
  double *rho, *thv, *ex, *w, *wflx;
  // FP32 edge inputs of the stage ([Ne][ld]) and the w shadow of the stage state ([Nc][ld])
  const float *phi, *gth, *a_e, *w_stage;
  float* Aw0;                              // level-major [h][Nc]: the predictor's A_w
  // gathered per stage, level-major [k][Nc]: dtau D_rho (FP64 in the corrector; FP32 in the
  // predictor, stored in the first half of the same buffer), dtau D_Theta, dtau A_w
  double* dr64;
  float *dr32, *dt32, *aw32;
  double* B;                               // stage-independent right-hand-side base [h][Nc]
  double* dp;                              // forward-elimination values [h][Nc]
  float* cp;                               // LU factor up_h / pivot_h [h][Nc]
  // FP32 shadows written by this stage, [Nc][ld]
  float *rho32, *thv32, *exp32, *w32;
  const double* cd;                        // per-level constants (FP64)
  const float* cf;                         // per-level constants (FP32)
  const double* dwa_t;                     // [Nc][3] dtau s l / A_c (FP64)
  const float4* cw32;                      // [Nc] FP32 dtau s l / A_c of the three edges, dtau / A_c
  unsigned* status;
  double dtau, inv_nsub;
  int hdamp;                               // half levels h < hdamp are Rayleigh-damped
  // corrector with divergence damping (fused into its gather): the undamped vn^{n+1}, the
  // cell Laplacian of its divergence, the stage shadows for the fluxes, c4 Abar^2, the
  // damped vn^{n+1} (stored by each edge's lower-id cell, which also accumulates the
  // step-mean mass flux)
  const float *dd_vn, *dd_L, *dd_rho, *dd_thv;
  float* dd_out;
  double* mflx;
  float dd_scale;
  int dd_upwind;
  // terrain-following levels (TOPO instances): the column's per-cell tables, level-major
  // [k][Nc] (upper interpolation weight, 1/dz, 1/dzh, reference Exner), the stage's
  // contravariant correction wcc at half levels ([Nc][ld]); for the gather w - wcc and 1/dzh
  // ([Nc][ld]) and the layer thickness at edges ([Ne][ld])
  const double *t_wu_lm, *t_idz_lm, *t_idzh_lm, *t_exref_lm;
  const float *t_wcc, *t_wcon, *t_inv_dzh, *t_dz_e;
};

// per-warp shadow transpose: CH levels of 32 columns (16 in the per-state kernel, 8 in the
// persistent ensemble, whose blocks hold four warps' tiles)
template <int CH>
struct LeanTile {
  float t[4][CH][33];                      // rho, theta_v, pi - pi_ref, w of 32 columns
};

// gather of the lean column's stage inputs for 32 consecutive cells: lanes over levels
// (LPE per cell), transposed through shared memory into level-major rows
template <int LPE>
struct LeanGatherTile {
  double d[LPE][kGatherCells + 1];
  float f[4][LPE][kGatherCells + 1];       // dtau D_Theta, dtau A_w, A_w (predictor), dtau D_rho (predictor)
};

// TOPO (terrain-following levels): the damped fluxes through the edges' layer thickness, the
// vertical advection of w with w - wcc and the cell's own 1/dzh; the divergences stay per unit
// thickness here and the column scales them by the cell's 1/dz
template <int LPE, bool CORR, bool DDF = false, bool TOPO = false>
__device__ inline void mx_lean_gather_body(const MxGeo& G, const MxLeanArgs& a, int64_t c0, LeanGatherTile<LPE>& T) {
  constexpr int CB = kGatherCells;
  const int N = G.N, ld = G.ld;
  const int64_t nc = G.nc;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int grp = tid / LPE, ngrp = nthr / LPE, lane = tid % LPE;
  const float dtau32 = (float)a.dtau;
  for (int k0 = 0; k0 < N; k0 += LPE) {
    if (CORR) {
      for (int i = tid; i < LPE * CB; i += nthr) {
        const int r = i / CB, cl = i % CB, h = k0 + r;
        const int64_t c = c0 + cl;
        T.f[2][r][cl] = (h >= 1 && h < N && c < nc) ? a.Aw0[(int64_t)h * nc + c] : 0.0f;
      }
      __syncthreads();
    }
    for (int cl = grp; cl < CB; cl += ngrp) {
      const int64_t c = c0 + cl;
      if (c >= nc) break;
      const int64_t o = c * ld;
      int64_t E[3];
      float sg[3], kw[3];
      double dwt[3];
      const float4 cw = a.cw32[c];
      const float dw32[3] = {cw.x, cw.y, cw.z};
      int64_t Ca[3], Cb[3];                  // DDF: the edges' two cells (row offsets)
      float sc[3], le[3];
      bool own[3];
      for (int s = 0; s < 3; ++s) {
        const int e = G.c2e[3 * c + s];
        E[s] = (int64_t)e * ld;
        sg[s] = G.s_ce32[3 * c + s];
        kw[s] = G.kin_w32[3 * c + s];
        if (CORR) dwt[s] = a.dwa_t[3 * c + s];
        if (DDF) {
          const int ca = G.e2c[2 * e], cb = G.e2c[2 * e + 1];
          Ca[s] = (int64_t)ca * ld;
          Cb[s] = (int64_t)cb * ld;
          sc[s] = a.dd_scale * G.inv_de32[e];
          le[s] = G.l_e32[e];
          own[s] = ca == c;
        }
      }
      const float ta = cw.w;
      const int k = k0 + lane;
      if (k < N) {
        float F[3], Gt[3];
        if (DDF) {
          // damped vn^{n+1} and its fluxes, as the damping's edge update forms them
          for (int s = 0; s < 3; ++s) {
            const float vd = a.dd_vn[E[s] + k] - sc[s] * (a.dd_L[Cb[s] + k] - a.dd_L[Ca[s] + k]);
            F[s] = 0.5f * (a.dd_rho[Ca[s] + k] + a.dd_rho[Cb[s] + k]) * vd;
            if constexpr (TOPO) F[s] *= a.t_dz_e[E[s] + k];
            const float t1 = a.dd_thv[Ca[s] + k], t2 = a.dd_thv[Cb[s] + k];
            Gt[s] = (le[s] * F[s]) * (a.dd_upwind ? (vd >= 0.0f ? t1 : t2) : 0.5f * (t1 + t2));
            if (own[s]) {
              a.dd_out[E[s] + k] = vd;
              a.mflx[E[s] + k] += (double)F[s] * a.inv_nsub;
            }
          }
        } else {
          for (int s = 0; s < 3; ++s) {
            F[s] = a.phi[E[s] + k];
            Gt[s] = a.gth[E[s] + k];
          }
        }
        // the hardware conversion here: the gather leaves the FP64 pipe half idle, and the
        // integer-pipe form costs more issue slots (measured 6.0 against 5.6 ms per step)
        if (CORR) T.d[lane][cl] = (dwt[0] * (double)F[0] + dwt[1] * (double)F[1]) + dwt[2] * (double)F[2];
        else T.f[3][lane][cl] = (dw32[0] * F[0] + dw32[1] * F[1]) + dw32[2] * F[2];
        T.f[0][lane][cl] = (sg[0] * Gt[0] + sg[1] * Gt[1] + sg[2] * Gt[2]) * ta;
      }
      if (k >= 1 && k < N) {
        const float hadv = kw[0] * a.a_e[E[0] + k] + kw[1] * a.a_e[E[1] + k] + kw[2] * a.a_e[E[2] + k];
        float Aw;
        if constexpr (TOPO)
          Aw = -hadv - a.t_wcon[o + k] * (a.w_stage[o + k - 1] - a.w_stage[o + k + 1]) * (0.5f * a.t_inv_dzh[o + k]);
        else
          Aw = -hadv - a.w_stage[o + k] * (a.w_stage[o + k - 1] - a.w_stage[o + k + 1]) * G.inv_dz2_32[k];
        if (CORR) Aw = 0.5f * (T.f[2][lane][cl] + Aw);
        else T.f[2][lane][cl] = Aw;
        T.f[1][lane][cl] = dtau32 * Aw;
      }
    }
    __syncthreads();
    for (int i = tid; i < LPE * CB; i += nthr) {
      const int r = i / CB, cl = i % CB, k = k0 + r;
      const int64_t c = c0 + cl;
      if (c >= nc || k >= N) continue;
      const int64_t j = (int64_t)k * nc + c;
      if (CORR) a.dr64[j] = T.d[r][cl];
      else a.dr32[j] = T.f[3][r][cl];
      a.dt32[j] = T.f[0][r][cl];
      if (k >= 1) {
        a.aw32[j] = T.f[1][r][cl];
        if (!CORR) a.Aw0[j] = T.f[2][r][cl];
      }
    }
    __syncthreads();
  }
}

template <int LPE, bool CORR, bool DDF = false, bool TOPO = false>
__global__ void __launch_bounds__(512, 3) k_mx_lean_gather(MxGeo G, MxLeanArgs a) {
  __shared__ LeanGatherTile<LPE> T;
  mx_lean_gather_body<LPE, CORR, DDF, TOPO>(G, a, (int64_t)blockIdx.x * kGatherCells, T);
}

// the corrector's gather with the damping fused in (32 lanes per cell, 256-thread blocks: the
// fastest of six tiles measured at R2B6/90, within 13 % of one another)
void launch_lean_gather_dd(const MxGeo& G, const MxLeanArgs& a, bool topo, cudaStream_t st) {
  const unsigned nb = (unsigned)((G.nc + kGatherCells - 1) / kGatherCells);
  if (topo) k_mx_lean_gather<32, true, true, true><<<nb, 256, 0, st>>>(G, a);
  else k_mx_lean_gather<32, true, true><<<nb, 256, 0, st>>>(G, a);
}

// write the finished chunk [k0, k0 + CH) of the warp's 32 columns (first cell c0): CH lanes
// per column row, 32 / CH rows per store instruction
template <int CH>
__device__ inline void lean_flush(const MxGeo& G, const MxLeanArgs& a, const LeanTile<CH>& T, int64_t c0, int k0,
                                  int lane) {
  __syncwarp();
  constexpr int RPI = 32 / CH;             // rows per instruction
  const int r = lane & (CH - 1), sub = lane / CH;
  const int k = k0 + r;
  float* const outs[4] = {a.rho32, a.thv32, a.exp32, a.w32};
  if (k < G.N) {
    for (int jj = 0; jj < 32; jj += RPI) {
      const int j = jj + sub;
      const int64_t c = c0 + j;
      if (c >= G.nc) continue;
      const int64_t o = c * G.ld + k;
#pragma unroll
      for (int f = 0; f < 4; ++f) outs[f][o] = T.t[f][r][j];
    }
  }
  __syncwarp();
}

// one column per thread (lane); every lane of the warp runs the loops (lanes past the last
// cell compute on zeros and store nothing) so that the chunk flushes stay warp-synchronous
// TOPO (terrain-following levels): each cell's interpolation weights, 1/dz and 1/dzh and
// reference Exner (level-major tables) in place of the per-level constants, the contravariant
// (1 - beta) w - wcc in the explicit vertical fluxes (zero at the lid and the ground), the
// gathered divergences scaled by the cell's 1/dz, and the stage's terrain-following w at the
// ground
template <bool CORR, int U, int CH, bool TOPO = false>
__device__ inline void mx_lean_column_item(const MxGeo& G, const MxLeanArgs& a, int64_t c, int64_t c0, int lane,
                                           LeanTile<CH>& T) {
  const int N = G.N, ld = G.ld;
  const int64_t nc = G.nc;
  const bool act = c < nc;
  const int64_t cc = act ? c : 0;
  const double* __restrict__ cd = a.cd;
  const float* __restrict__ cf = a.cf;
  const double dtau = a.dtau;
#define LMV(p, k) (p)[(int64_t)(k) * nc + cc]
  // ---- downward sweep: at step j half level j becomes known, completing full level
  // k = j - 1 and, for k >= 1, the row of half level h = k
  double thv1 = 0.0, ex1 = 0.0, ex2 = 0.0;          // full levels j-1 and j-2 (FP64)
  float rho1f = 0.f, thv1f = 0.f;
  double ti1 = 0.0;                                  // theta_ic at half level j-1 (FP64)
  float ti1f = 0.f, M1 = 0.f, M2 = 0.f, xv1 = 0.f;   // half level j-1 (and j-2 for M)
  double w1 = 0.0;
  float gam2 = 0.f, dpe2 = 0.f;                      // full level j-2
  float cp_prev = 0.f;
  double dp_prev = 0.0;
#pragma unroll U
  for (int j = 0; j <= N; ++j) {
    double rho = 0.0, thv = 0.0, ex = 0.0;
    if (j < N) {
      rho = LMV(a.rho, j);
      thv = LMV(a.thv, j);
      ex = LMV(a.ex, j);
    }
    const float rhof = f64_to_f32(rho), thvf = f64_to_f32(thv);
    // theta_v at half level j: FP64 only where the predictor forms the hydrostatic base
    double ti = 0.0;
    float rif, tif;
    if (j == 0) {
      ti = thv;
      rif = rhof;
      tif = thvf;
    } else if (j == N) {
      ti = thv1;
      rif = rho1f;
      tif = thv1f;
    } else if constexpr (TOPO) {
      const double wu = LMV(a.t_wu_lm, j);
      const float wuf = f64_to_f32(wu);
      rif = wuf * rho1f + (1.0f - wuf) * rhof;
      if (!CORR) {
        ti = wu * thv1 + (1.0 - wu) * thv;
        tif = f64_to_f32(ti);
      } else {
        tif = wuf * thv1f + (1.0f - wuf) * thvf;
      }
    } else {
      rif = cf[LF_WU * ld + j] * rho1f + cf[LF_WL * ld + j] * rhof;
      if (!CORR) {
        ti = cd[LD_WU * ld + j] * thv1 + cd[LD_WL * ld + j] * thv;
        tif = f64_to_f32(ti);
      } else {
        tif = cf[LF_WU * ld + j] * thv1f + cf[LF_WL * ld + j] * thvf;
      }
    }
    const float Mh = rif * tif;
    const double wh = (j == 0 || j == N) ? 0.0 : LMV(a.w, j);
    const float whf = f64_to_f32(wh);
    // the explicit vertical velocity through half level j: w on flat levels (the factor
    // 1 - beta is in the level constant), (1 - beta) w - wcc on terrain-following ones
    float xvj = whf;
    if constexpr (TOPO) xvj = (j == 0 || j == N) ? 0.0f : (float)(1.0 - kBeta) * whf - a.t_wcc[cc * ld + j];
    float gam1 = 0.f, dpe1 = 0.f;
    if (j >= 1) {
      const int k = j - 1;
      float dtk = LMV(a.dt32, k), dt1, dtb;
      if constexpr (TOPO) {
        const double idz = LMV(a.t_idz_lm, k);
        dtk *= f64_to_f32(idz);
        dt1 = f64_to_f32(dtau * idz);
        dtb = f64_to_f32(dtau * kBeta * idz);
      } else {
        dt1 = cf[LF_DT1 * ld + k];
        dtb = cf[LF_DTB * ld + k];
      }
      const float dthe = -dtk - dt1 * (M1 * xv1 - Mh * xvj);
      const float g = kRcvF * __fdividef(f64_to_f32(ex1), rho1f * thv1f);
      gam1 = g * dtb;
      dpe1 = g * dthe;
      if (k >= 1) {
        const int h = k;
        double cpdzh;                                    // cpd / dzh of half level h
        float ca;
        if constexpr (TOPO) {
          const double idzh = LMV(a.t_idzh_lm, h);
          cpdzh = kCpd * idzh;
          ca = f64_to_f32(dtau * kBeta * kCpd * idzh);
        } else {
          cpdzh = cd[LD_CPDZH * ld + h];
          ca = cf[LF_CA * ld + h];
        }
        const float aa = ca * ti1f;
        const float lo = -aa * gam2 * M2;
        const float di = 1.0f + aa * (gam2 + gam1) * M1;
        const float up = -aa * gam1 * Mh;
        double B;
        if (!CORR) {
          B = w1 - dtau * fma(cpdzh * ti1, ex2 - ex1, kGrav);
          if (act) LMV(a.B, h) = B;
        } else {
          B = LMV(a.B, h);
        }
        const float inc = LMV(a.aw32, h) - aa * (dpe2 - dpe1);
        const float piv = __fdividef(1.0f, di - lo * cp_prev);
        const float cpv = up * piv;
        const double dpv = (B + f32_to_f64(inc) - f32_to_f64(lo) * dp_prev) * f32_to_f64(piv);
        if (act) {
          LMV(a.dp, h) = dpv;
          LMV(a.cp, h) = cpv;
        }
        cp_prev = cpv;
        dp_prev = dpv;
      }
    }
    gam2 = gam1;
    dpe2 = dpe1;
    M2 = M1;
    M1 = Mh;
    w1 = wh;
    xv1 = xvj;
    ti1 = ti;
    ti1f = tif;
    ex2 = ex1;
    ex1 = ex;
    thv1 = thv;
    rho1f = rhof;
    thv1f = thvf;
  }
  // ---- upward sweep: back substitution, damping and the update of full level k (between
  // half levels k and k+1); the level above (k-1) is loaded one step ahead for the
  // half-level interpolants
  bool ok = true;
  double x_next = 0.0, wn_next = 0.0;                // half level k+1: undamped, damped
  float wnf_next = 0.f;
  // half level k+1 quantities carried upward
  float ri_next = 0.f, M_next = 0.f, xv_next = 0.f;  // at k+1 (explicit vertical velocity of S^n)
  float fflux_next = 0.f;                            // corrector: vertical mass flux at k+1
  // full level k (current) and k-1 (next), FP64 and FP32
  double rho_k = act ? LMV(a.rho, N - 1) : 0.0, thv_k = act ? LMV(a.thv, N - 1) : 0.0;
  double ex_k = act ? LMV(a.ex, N - 1) : 0.0;
  {
    // half level N: interpolants of the lowest full level, w = 0
    ri_next = f64_to_f32(rho_k);
    M_next = ri_next * f64_to_f32(thv_k);
  }
  const int64_t o = cc * ld;
#pragma unroll U
  for (int k = N - 1; k >= 0; --k) {
    // half level k: the level above
    double rho_u = 0.0, thv_u = 0.0, ex_u = 0.0;
    if (k >= 1) {
      rho_u = LMV(a.rho, k - 1);
      thv_u = LMV(a.thv, k - 1);
      ex_u = LMV(a.ex, k - 1);
    }
    // the FP32 roundings of level k are formed again rather than carried from the level
    // above: carried, the two extra live values spill at this kernel's 48 registers
    const float rho_kf = f64_to_f32(rho_k), thv_kf = f64_to_f32(thv_k);
    float ri_k, M_k;
    if (k == 0) {
      ri_k = rho_kf;
      M_k = rho_kf * thv_kf;
    } else if constexpr (TOPO) {
      const float wuf = f64_to_f32(LMV(a.t_wu_lm, k));
      ri_k = wuf * f64_to_f32(rho_u) + (1.0f - wuf) * rho_kf;
      M_k = ri_k * (wuf * f64_to_f32(thv_u) + (1.0f - wuf) * thv_kf);
    } else {
      ri_k = cf[LF_WU * ld + k] * f64_to_f32(rho_u) + cf[LF_WL * ld + k] * rho_kf;
      M_k = ri_k * (cf[LF_WU * ld + k] * f64_to_f32(thv_u) + cf[LF_WL * ld + k] * thv_kf);
    }
    const float wf_k = k >= 1 ? f64_to_f32(LMV(a.w, k)) : 0.0f;
    float xv_k = wf_k;
    if constexpr (TOPO) xv_k = k >= 1 ? (float)(1.0 - kBeta) * wf_k - a.t_wcc[o + k] : 0.0f;
    // back substitution at half level k
    double x = 0.0, wn = 0.0;
    if (k >= 1) {
      x = LMV(a.dp, k) - f32_to_f64(LMV(a.cp, k)) * x_next;
      wn = k < a.hdamp ? x * cd[LD_DAMP * ld + k] : x;
    }
    const float wnf = f64_to_f32(wn);
    // full level k
    float dtb, dt1, dtk = LMV(a.dt32, k);
    double idz = 0.0, exref;
    if constexpr (TOPO) {
      idz = LMV(a.t_idz_lm, k);
      dtk *= f64_to_f32(idz);
      dt1 = f64_to_f32(dtau * idz);
      dtb = f64_to_f32(dtau * kBeta * idz);
      exref = LMV(a.t_exref_lm, k);
    } else {
      dtb = cf[LF_DTB * ld + k];
      dt1 = cf[LF_DT1 * ld + k];
      exref = cd[LD_EXREF * ld + k];
    }
    const float dthe = -dtk - dt1 * (M_k * xv_k - M_next * xv_next);
    const float g = kRcvF * __fdividef(f64_to_f32(ex_k), rho_kf * thv_kf);
    const float q = M_k * wnf - M_next * wnf_next;
    const float dTh = dthe - dtb * q;                // Theta increment
    const float dex = g * dthe - g * dtb * q;        // Exner increment (linearised state equation)
    float s_rho, s_thv, s_exp;
    if (!CORR) {
      float drk = LMV(a.dr32, k);
      if constexpr (TOPO) drk *= f64_to_f32(idz);
      const float drho = -drk - dt1 * (ri_k * xv_k - ri_next * xv_next) - dtb * (ri_k * wnf - ri_next * wnf_next);
      s_rho = rho_kf + drho;
      s_thv = thv_kf + __fdividef(dTh - drho * thv_kf, s_rho);
      s_exp = f64_to_f32(ex_k - exref) + dex;
      ok = ok && isfinite(s_thv) && isfinite(s_exp) && isfinite(wnf);
    } else {
      // vertical mass flux through half level k of the step: rho_ic ((1 - beta) w^n + beta w^{n+1}),
      // less rho_ic wcc on terrain-following levels
      double t;
      float fk;
      if constexpr (TOPO) {
        fk = ri_k * (xv_k + (float)kBeta * wnf);
        t = fma(dtau * idz, f32_to_f64(fk) - f32_to_f64(fflux_next), LMV(a.dr64, k) * idz);
      } else {
        fk = ri_k * ((float)(1.0 - kBeta) * wf_k + (float)kBeta * wnf);
        t = fma(cd[LD_IDZ * ld + k], f32_to_f64(fk) - f32_to_f64(fflux_next), LMV(a.dr64, k));
      }
      const double rho_n = rho_k - t;
      const float rho_nf = f64_to_f32(rho_n);
      const double thv_n = thv_k + f32_to_f64(__fdividef(dTh + f64_to_f32(t) * thv_kf, rho_nf));
      const double ex_n = ex_k + f32_to_f64(dex);
      if (act) {
        LMV(a.wflx, k) = fma(f32_to_f64(fk), a.inv_nsub, LMV(a.wflx, k));
        LMV(a.rho, k) = rho_n;
        LMV(a.thv, k) = thv_n;
        LMV(a.ex, k) = ex_n;
        LMV(a.w, k) = wn;
      }
      s_rho = rho_nf;
      s_thv = f64_to_f32(thv_n);
      s_exp = f64_to_f32(ex_n - exref);
      ok = ok && finite64(thv_n) && finite64(ex_n) && finite64(wn);
      fflux_next = fk;
    }
    const int k0 = k & ~(CH - 1);
    T.t[0][k - k0][lane] = s_rho;
    T.t[1][k - k0][lane] = s_thv;
    T.t[2][k - k0][lane] = s_exp;
    T.t[3][k - k0][lane] = wnf;
    if (k == k0) lean_flush(G, a, T, c0, k0, lane);
    x_next = x;
    wn_next = wn;
    wnf_next = wnf;
    ri_next = ri_k;
    M_next = M_k;
    xv_next = xv_k;
    rho_k = rho_u;
    thv_k = thv_u;
    ex_k = ex_u;
  }
  (void)wn_next;
  if (act) {
    if constexpr (TOPO) {                            // the ground: the stage's terrain-following w
      const float wg = a.t_wcc[o + N];
      a.w32[o + N] = wg;
      if (CORR) LMV(a.w, N) = f32_to_f64(wg);
    } else {
      a.w32[o + N] = 0.0f;
      if (CORR) LMV(a.w, N) = 0.0;                   // the ground (w^n there is 0 already)
    }
  }
  if (!ok && act) atomicOr(a.status, 1u);
#undef LMV
}

template <bool CORR, int U, int CH, int THREADS, int MINB, bool TOPO = false>
__global__ void __launch_bounds__(THREADS, MINB) k_mx_lean_column(MxGeo G, MxLeanArgs a) {
  __shared__ LeanTile<CH> T[THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c0 = (int64_t)blockIdx.x * THREADS + warp * 32;
  if (c0 >= G.nc) return;                            // whole warp past the end
  mx_lean_column_item<CORR, U, CH, TOPO>(G, a, c0 + lane, c0, lane, T[warp]);
}

// launch shapes of the lean column, one thread per column in blocks of four warps: the tile's
// "lanes" is the unroll factor of the two sweeps and its "block" the resident blocks per SM
// the registers are held to (6: 80 registers, 8: 64, 9: 56, 10: 48, 12: 40). Only the register
// cap varies among the candidates: it leaves the arithmetic as it is, while another unroll factor
// changes which multiply-adds the compiler fuses and with them the FP32 roundings (measured:
// unroll 1 or 4 moves vn by 1e-7 relative after one step), and a tuner choosing by timing
// must not change results. The kernel waits on memory latency and gains from occupancy (12.2 ms
// per R2B6/90 step at 10 blocks against 16.9 ms with 64-thread blocks at 94 registers); the
// default, 9 blocks (36 warps per SM, 56 registers, no spills), measured 11.21 against 11.68 ms
// at 10 blocks (48 registers, spilling in the corrector) and 161.3 against 162.4 ms at R2B8/90.
const TileChoice kLeanShapes[] = {{2, 9}, {2, 10}, {2, 8}, {2, 12}, {2, 6}};
const TileChoice kLeanDefault = {2, 9};

bool lean_shape_ok(const TileChoice& t) {
  for (const TileChoice& c : kLeanShapes)
    if (c.lanes == t.lanes && c.block == t.block) return true;
  return false;
}

template <bool CORR, bool TOPO = false>
void launch_lean_column_as(const MxGeo& G, const MxLeanArgs& a, const TileChoice& t, cudaStream_t st) {
  const unsigned nb = blocks_for(G.nc, 128);
  if (t.block == 8) k_mx_lean_column<CORR, 2, 8, 128, 8, TOPO><<<nb, 128, 0, st>>>(G, a);
  else if (t.block == 10) k_mx_lean_column<CORR, 2, 8, 128, 10, TOPO><<<nb, 128, 0, st>>>(G, a);
  else if (t.block == 12) k_mx_lean_column<CORR, 2, 8, 128, 12, TOPO><<<nb, 128, 0, st>>>(G, a);
  else if (t.block == 6) k_mx_lean_column<CORR, 2, 8, 128, 6, TOPO><<<nb, 128, 0, st>>>(G, a);
  else k_mx_lean_column<CORR, 2, 8, 128, 9, TOPO><<<nb, 128, 0, st>>>(G, a);
}

template <bool CORR>
void launch_lean_column(const MxGeo& G, const MxLeanArgs& a, const TileChoice& t, bool topo, cudaStream_t st) {
  if (topo) launch_lean_column_as<CORR, true>(G, a, t, st);
  else launch_lean_column_as<CORR, false>(G, a, t, st);
}

MxGeo make_mx_geo(const icon_grid* grid, const StateDev& s) {
  const GridDev& g = grid->g;
  const Vertical& v = grid->vert;
  MxGeo G;
  G.nc = g.nc; G.ne = g.ne; G.nv = g.nv; G.N = v.N; G.ld = v.ld;
  G.c2e = g.c2e; G.e2c = g.e2c; G.e2v = g.e2v; G.v2e = g.v2e; G.v2c = g.v2c; G.vdeg = g.vdeg;
  G.e2vt = g.e2vt; G.e2q = g.e2q;
  G.div_w32 = g.div_w32; G.rot_w32 = g.rot_w32; G.vt_w32 = g.vt_w32; G.kin_w32 = g.kin_w32;
  G.lsq_w32 = g.lsq_w32; G.inv_de32 = g.inv_de32; G.inv_le32 = g.inv_le32; G.f_e32 = g.f_e32;
  G.l_e32 = g.l_e32; G.n_e32 = g.n_e32; G.t_e32 = g.t_e32; G.L34inv32 = g.L34inv32; G.s_ce32 = g.s_ce32;
  G.inv_Ac = g.inv_Ac;
  G.div_wa = g.div_wa;
  G.dz = v.d_dz; G.dzh = v.d_dzh; G.wu = v.d_wu; G.wl = v.d_wl; G.dz2 = v.d_dz2; G.ray = v.d_ray;
  G.ex_ref = s.ex_ref;
  G.inv_dz32 = v.d_inv_dz32; G.wu32 = v.d_wu32; G.wl32 = v.d_wl32; G.inv_dz2_32 = v.d_inv_dz2_32;
  return G;
}

// stage arguments of one state
MxEdgeArgs edge_args(StateDev& s, bool corr, double dtau, int nsub) {
  MxEdgeArgs ea;
  ea.vn = corr ? s.vn32_s : s.vn32;
  ea.w = corr ? s.w32_s : s.w32;
  ea.rho = corr ? s.rho32_s : s.rho32;
  ea.thv = corr ? s.thv32_s : s.thv32;
  ea.exp = corr ? s.exp32_s : s.exp32;
  ea.vt = s.vt32; ea.Kc = s.Kc32; ea.zeta = s.zeta32; ea.w_v = s.wv32;
  ea.vn_base = s.vn32;
  ea.vn_out = corr ? s.vn32 : s.vn32_s;
  ea.Avn0 = s.Avn0_32;
  ea.phi = s.F32; ea.gth = s.G32; ea.a_e = s.ae32; ea.mflx = s.mflx;
  ea.dtau = (float)dtau; ea.inv_nsub = 1.0 / nsub; ea.corrector = corr;
  ea.skip_flux = 0;
  ea.upwind_theta = 0;
  const TopoDev& T = s.topo;
  ea.t_wu_e = T.wu_e32; ea.t_inv_dz_e = T.inv_dz_e32; ea.t_dz_e = T.dz_e32; ea.t_csn = T.csn32; ea.t_bf = T.bf32;
  ea.t_wcon = T.wcon32; ea.t_hdpdz = T.hdpdz32;
  return ea;
}

MxColArgs col_args(StateDev& s, bool corr, double dtau, int nsub) {
  MxColArgs ca;
  ca.rho = s.rho; ca.thv = s.thv; ca.ex = s.ex; ca.w = s.w; ca.wflx = s.wflx;
  ca.phi = s.F32; ca.gth = s.G32; ca.a_e = s.ae32;
  ca.w_stage = corr ? s.w32_s : s.w32;
  ca.Aw0 = s.Aw0_32;
  ca.rho32 = corr ? s.rho32 : s.rho32_s;
  ca.thv32 = corr ? s.thv32 : s.thv32_s;
  ca.exp32 = corr ? s.exp32 : s.exp32_s;
  ca.w32 = corr ? s.w32 : s.w32_s;
  ca.cc = s.colconst;
  ca.fac64 = s.fac64;
  ca.hdr = s.hdr;
  ca.hdt = s.hdt;
  ca.hdw = s.hdw;
  ca.hdg = s.hdg;
  ca.rho32n = s.rho32;
  ca.thv32n = s.thv32;
  ca.exp32n = s.exp32;
  ca.exref32 = s.exref32;
  ca.dps = s.dps;
  ca.status = s.status;
  ca.dtau = dtau; ca.inv_nsub = 1.0 / nsub;
  const TopoDev& T = s.topo;
  ca.t_wu_lm = T.wu_lm; ca.t_idz_lm = T.idz_lm; ca.t_idzh_lm = T.idzh_lm; ca.t_exref_lm = T.exref_lm;
  ca.t_wcc = T.wcc32; ca.t_wcon = T.wcon32;
  return ca;
}

MxLeanArgs lean_args(StateDev& s, bool corr, double dtau, int nsub) {
  MxLeanArgs la;
  la.rho = s.rho; la.thv = s.thv; la.ex = s.ex; la.w = s.w; la.wflx = s.wflx;
  la.phi = s.F32; la.gth = s.G32; la.a_e = s.ae32;
  la.w_stage = corr ? s.w32_s : s.w32;
  la.Aw0 = s.Aw0_32;
  la.dr64 = s.ln_dr64;
  la.dr32 = reinterpret_cast<float*>(s.ln_dr64);
  la.dt32 = s.ln_dt32;
  la.aw32 = s.ln_aw32;
  la.B = s.ln_B;
  la.dp = s.ln_dp;
  la.cp = s.ln_cp;
  la.rho32 = corr ? s.rho32 : s.rho32_s;
  la.thv32 = corr ? s.thv32 : s.thv32_s;
  la.exp32 = corr ? s.exp32 : s.exp32_s;
  la.w32 = corr ? s.w32 : s.w32_s;
  la.cd = s.ln_cd;
  la.cf = s.ln_cf;
  la.dwa_t = s.ln_dwa;
  la.cw32 = reinterpret_cast<const float4*>(s.ln_cw32);
  la.status = s.status;
  la.dtau = dtau;
  la.inv_nsub = 1.0 / nsub;
  la.hdamp = s.ln_hdamp;
  la.dd_vn = la.dd_L = la.dd_rho = la.dd_thv = nullptr;
  la.dd_out = nullptr;
  la.mflx = s.mflx;
  la.dd_scale = 0.0f;
  la.dd_upwind = 0;
  const TopoDev& T = s.topo;
  la.t_wu_lm = T.wu_lm; la.t_idz_lm = T.idz_lm; la.t_idzh_lm = T.idzh_lm; la.t_exref_lm = T.exref_lm;
  la.t_wcc = T.wcc32; la.t_wcon = T.wcon32; la.t_inv_dzh = T.inv_dzh_c32; la.t_dz_e = T.dz_e32;
  return la;
}

// the gather's per-cell weights for one dtau: FP64 dtau s l / A_c of the three edges, and
// their FP32 roundings with the FP32 dtau / A_c (formed as the product of the two FP32
// roundings), so that the gather's inner loop converts nothing
__global__ void k_mx_dwa_t(int64_t nc, const double* __restrict__ div_wa, const double* __restrict__ inv_Ac,
                           double dtau, double* __restrict__ out, float* __restrict__ out32) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  float4 f;
  float* fp = &f.x;
  for (int s = 0; s < 3; ++s) {
    const double v = dtau * div_wa[3 * c + s];
    out[3 * c + s] = v;
    fp[s] = (float)v;
  }
  f.w = (float)dtau * (float)inv_Ac[c];
  reinterpret_cast<float4*>(out32)[c] = f;
}

// ---------------------------------------------------------------- launch helpers with tile choices
unsigned item_blocks(int64_t n, int lpe, int block) {
  const int64_t per_block = (int64_t)(block / 32) * (32 / lpe);
  return (unsigned)((n + per_block - 1) / per_block);
}

// the lane count of a tile as a compile-time constant (8, 16 or 32 lanes per entity)
template <typename F>
void with_lanes(int lanes, F f) {
  if (lanes == 8) f(std::integral_constant<int, 8>{});
  else if (lanes == 16) f(std::integral_constant<int, 16>{});
  else f(std::integral_constant<int, 32>{});
}

void launch_kind(int kind, const TileChoice& t, const MxGeo& G, StateDev& s, const MxEdgeArgs& ea,
                 const MxColArgs& ca, float dt, cudaStream_t st) {
  const int B = t.block;
  switch (kind) {
    case K_MX_VERTEX:
      with_lanes(t.lanes, [&](auto L) {
        constexpr int LPE = decltype(L)::value;
        k_mx_vertex<LPE><<<item_blocks(G.nv, LPE, B), B, 0, st>>>(G, ea.vn, ea.w, s.zeta32, s.wv32);
      });
      break;
    case K_MX_EDGE:
      with_lanes(t.lanes, [&](auto L) {
        constexpr int LPE = decltype(L)::value;
        k_mx_edge_diag<LPE><<<item_blocks(G.ne, LPE, B), B, 0, st>>>(G, ea.vn, s.vt32);
      });
      break;
    case K_MX_CELL_KE:
      with_lanes(t.lanes, [&](auto L) {
        constexpr int LPE = decltype(L)::value;
        k_mx_cell_ke<LPE><<<item_blocks(G.nc, LPE, B), B, 0, st>>>(G, ea.vn, s.vt32, s.Kc32);
      });
      break;
    case K_MX_EDGE_TEND:
      with_lanes(t.lanes, [&](auto L) {
        constexpr int LPE = decltype(L)::value;
        if (s.topo.on) k_mx_edge_tend<LPE, true><<<item_blocks(G.ne, LPE, B), B, 0, st>>>(G, ea);
        else k_mx_edge_tend<LPE><<<item_blocks(G.ne, LPE, B), B, 0, st>>>(G, ea);
      });
      break;
    case K_MX_DIFF_VERTEX:
      with_lanes(t.lanes, [&](auto L) {
        constexpr int LPE = decltype(L)::value;
        k_mx_diff_vertex<LPE><<<item_blocks(G.nv + G.nc, LPE, B), B, 0, st>>>(G, s.vn32, s.uvx32, s.uvy32, s.uvz32,
                                                                              s.zeta32, s.Kc32);
      });
      break;
    case K_MX_COLUMN_PREP: {   // the predictor's gather (the corrector's only differs in the Aw0 average)
      const unsigned nb = (unsigned)((G.nc + 31) / 32);
      with_lanes(t.lanes, [&](auto L) {
        constexpr int LPE = decltype(L)::value;
        if (s.ln_B) {
          const MxLeanArgs la = lean_args(s, false, (double)ea.dtau, 1);
          if (s.topo.on) k_mx_lean_gather<LPE, false, false, true><<<nb, B, 0, st>>>(G, la);
          else k_mx_lean_gather<LPE, false><<<nb, B, 0, st>>>(G, la);
        } else {
          k_mx_gather_tile<LPE, false><<<nb, B, 0, st>>>(G, ca);
        }
      });
      break;
    }
    case K_MX_LEAN: {          // the predictor's lean column (writes only the stage's scratch and S*)
      const MxLeanArgs la = lean_args(s, false, (double)ea.dtau, 1);
      launch_lean_column<false>(G, la, t, s.topo.on, st);
      break;
    }
    case K_MX_DIFF_EDGE:
      with_lanes(t.lanes, [&](auto L) {
        constexpr int LPE = decltype(L)::value;
        k_mx_diff_edge<LPE><<<item_blocks(G.ne, LPE, B), B, 0, st>>>(G, s.vn32, s.uvx32, s.uvy32, s.uvz32, s.zeta32,
                                                                     s.Kc32, s.thv32, s.vt32, dt);
      });
      break;
    default: break;
  }
}

template <bool CORR>
void launch_mx_column(const MxGeo& G, const MxColArgs& a, bool topo, cudaStream_t st) {
  const unsigned nb = blocks_for(G.nc, 128);
  if (topo) {
    if (G.N <= 32) k_mx_column<32, CORR, true><<<nb, 128, 0, st>>>(G, a);
    else if (G.N <= 64) k_mx_column<64, CORR, true><<<nb, 128, 0, st>>>(G, a);
    else if (G.N <= 96) k_mx_column<96, CORR, true><<<nb, 128, 0, st>>>(G, a);
    else if (G.N <= 128) k_mx_column<128, CORR, true><<<nb, 128, 0, st>>>(G, a);
    else k_mx_column<256, CORR, true><<<nb, 128, 0, st>>>(G, a);
    return;
  }
  if (CORR && a.fac64) {
    k_mx_corr_solve<<<nb, 128, 0, st>>>(G, a);
    k_mx_corr_update<<<(unsigned)((G.nc + kUpdCells - 1) / kUpdCells), 256, 0, st>>>(G, a);
    return;
  }
  if (G.N <= 32) k_mx_column<32, CORR><<<nb, 128, 0, st>>>(G, a);
  else if (G.N <= 64) k_mx_column<64, CORR><<<nb, 128, 0, st>>>(G, a);
  else if (G.N <= 96) k_mx_column<96, CORR><<<nb, 128, 0, st>>>(G, a);
  else if (G.N <= 128) k_mx_column<128, CORR><<<nb, 128, 0, st>>>(G, a);
  else k_mx_column<256, CORR><<<nb, 128, 0, st>>>(G, a);
}

// ---------------------------------------------------------------- autotuner
// Candidate tiles over (entity, level): 32 lanes per entity (one entity per warp), 16
// (two per warp) or 8 (four per warp), blocks of 64, 128, 256 or 512 threads: twelve per
// stencil kind. The lean column (one thread per column) chooses among its precompiled
// launch shapes (kLeanShapes). Each kind is timed on the state's own data (three launches
// per candidate after one untimed, CUDA events) and the fastest kept, in the order of the
// step, so that every trial reads inputs its predecessors formed. Choices are cached per
// (kind, grid size, levels, GPU) in the process and, if the environment variable
// ICON_TUNE_CACHE names a file, in that file.
const int kTunedKinds[] = {K_MX_VERTEX, K_MX_EDGE, K_MX_CELL_KE, K_MX_EDGE_TEND, K_MX_COLUMN_PREP, K_MX_LEAN,
                           K_MX_DIFF_VERTEX};
const int kTileLanes[] = {32, 16, 8};
const int kTileBlocks[] = {128, 256, 512, 64};
std::mutex g_tune_mu;
std::map<std::string, TileChoice> g_tune_cache;
bool g_tune_file_loaded = false;

std::string tune_key(int kind, const MxGeo& G) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, dev);
  char buf[160];
  snprintf(buf, sizeof(buf), "k%d_nc%lld_N%d_sm%d%d_n%d", kind, (long long)G.nc, G.N, p.major, p.minor,
           p.multiProcessorCount);
  return buf;
}

void load_tune_file() {
  if (g_tune_file_loaded) return;
  g_tune_file_loaded = true;
  const char* path = getenv("ICON_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[160];
  int lanes, block;
  while (fscanf(f, "%159s %d %d", key, &lanes, &block) == 3) g_tune_cache[key] = TileChoice{lanes, block};
  fclose(f);
}

void save_tune_entry(const std::string& key, const TileChoice& t) {
  const char* path = getenv("ICON_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d\n", key.c_str(), t.lanes, t.block);
  fclose(f);
}

}  // namespace

bool lean_column_shape_ok(int unroll, int blocks_per_sm) { return lean_shape_ok(TileChoice{unroll, blocks_per_sm}); }

void autotune_mixed(icon_state* st, double dt, int nsub, cudaStream_t stream) {
  StateDev& s = st->s;
  const MxGeo G = make_mx_geo(st->grid, s);
  const double dtau = dt / nsub;
  // the predictor's arguments: every tuned kernel then writes only scratch or S* buffers
  const MxEdgeArgs ea = edge_args(s, false, dtau, nsub);
  const MxColArgs ca = col_args(s, false, dtau, nsub);
  const bool lean = s.ln_B != nullptr;
  if (lean) {
    // the lean gather's weights and the column's per-level constants for this dtau, so that
    // the gather and column trials compute on valid inputs
    k_mx_leanconst<<<1, 128, 0, stream>>>(G.N, G.ld, G.wu, G.wl, G.dzh, G.dz, G.ray, s.ex_ref, dtau, s.ln_cd, s.ln_cf);
    k_mx_dwa_t<<<blocks_for(G.nc, 256), 256, 0, stream>>>(G.nc, G.div_wa, G.inv_Ac, dtau, s.ln_dwa, s.ln_cw32);
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_tune_file();
  for (int kind : kTunedKinds) {
    if (st->tile[kind].lanes != 0 && st->tile_forced[kind]) continue;
    if (kind == K_MX_COLUMN_PREP && !s.fac64 && !lean) continue;
    if (kind == K_MX_LEAN && !lean) continue;
    const std::string key = tune_key(kind, G);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      st->tile[kind] = it->second;
      continue;
    }
    std::vector<TileChoice> cands;
    if (kind == K_MX_LEAN) {
      for (const TileChoice& c : kLeanShapes) cands.push_back(c);
    } else {
      for (int lanes : kTileLanes)
        for (int block : kTileBlocks) cands.push_back(TileChoice{lanes, block});
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    TileChoice bestc = cands[0];
    for (const TileChoice& t : cands) {
      launch_kind(kind, t, G, s, ea, ca, (float)dt, stream);     // warm
      cudaEventRecord(e0, stream);
      for (int r = 0; r < 3; ++r) launch_kind(kind, t, G, s, ea, ca, (float)dt, stream);
      cudaEventRecord(e1, stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bestc = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st->tile[kind] = bestc;
    g_tune_cache[key] = bestc;
    save_tune_entry(key, bestc);
  }
  // a trial that met a non-finite value would have flagged the state; the step that
  // follows checks it again
  cudaMemsetAsync(s.status, 0, sizeof(unsigned), stream);
  st->tuned = true;
}

void enqueue_step_mixed(icon_state* st, double dt, int nsub, cudaStream_t stream) {
  const icon_grid* grid = st->grid;
  StateDev& s = st->s;
  const MxGeo G = make_mx_geo(grid, s);
  const int64_t nc = G.nc;
  const double dtau = dt / nsub;
  cudaMemsetAsync(s.mflx, 0, sizeof(double) * G.ne * G.ld, stream);
  cudaMemsetAsync(s.wflx, 0, sizeof(double) * nc * (G.N + 1), stream);
  k_mx_colconst<<<1, 128, 0, stream>>>(G.N, G.ld, G.wu, G.wl, G.dzh, G.dz, G.ray, s.ex_ref, dtau, s.colconst);
  const bool lean = s.ln_B != nullptr;
  if (lean) {
    k_mx_leanconst<<<1, 128, 0, stream>>>(G.N, G.ld, G.wu, G.wl, G.dzh, G.dz, G.ray, s.ex_ref, dtau, s.ln_cd, s.ln_cf);
    k_mx_dwa_t<<<blocks_for(nc, 256), 256, 0, stream>>>(nc, G.div_wa, G.inv_Ac, dtau, s.ln_dwa, s.ln_cw32);
  }
  auto tile = [&](int kind) { return st->tile[kind].lanes ? st->tile[kind] : TileChoice{32, 256}; };
  // The next stage's edge diagnostics (vt) and cell kinetic energy read only that stage's vn,
  // final once this stage's edge tendency (predictor) or damped gather (corrector) has run,
  // and write vt32 and Kc32, which neither this stage's gather nor its column reads. While a
  // step on flat levels is recorded into its graph they go on a second branch beside the
  // column, whose last wave of blocks leaves part of the SMs idle; the branch is joined before
  // the next stage's edge tendency. Eager (profiled) steps keep one stream. Measured: R2B6/90
  // 29.5 -> 28.7 ms per step, R2B8/90 439.7 -> 438.5 ms; on coarser grids the joins cost about
  // what the branch saves (64 states of R2B4/60 and R2B5/60 stepped one after another: 270 ->
  // 285 ms), over terrain and for the FP64 step the branch measured slower or equal: it is
  // recorded for flat mixed states of at least kBranchMinCells cells (R2B6) only.
  constexpr int64_t kBranchMinCells = 327680;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(stream, &cs);
  const bool overlap = lean && !s.topo.on && nc >= kBranchMinCells && st->side_stream &&
                       cs == cudaStreamCaptureStatusActive;
  bool diag_ahead = false;                 // this stage's vt32 and Kc32 are on the branch
  auto fork_diag = [&](bool next_corr) {
    const MxEdgeArgs en = edge_args(s, next_corr, dtau, nsub);
    cudaEventRecord(st->fork_ev, stream);
    cudaStreamWaitEvent(st->side_stream, st->fork_ev, 0);
    launch_kind(K_MX_EDGE, tile(K_MX_EDGE), G, s, en, col_args(s, next_corr, dtau, nsub), (float)dt, st->side_stream);
    launch_kind(K_MX_CELL_KE, tile(K_MX_CELL_KE), G, s, en, col_args(s, next_corr, dtau, nsub), (float)dt,
                st->side_stream);
    cudaEventRecord(st->join_ev, st->side_stream);
    diag_ahead = true;
  };
  for (int it = 0; it < nsub; ++it) {
    for (int stage = 0; stage < 2; ++stage) {
      const bool corr = stage == 1;
      const MxEdgeArgs ea = edge_args(s, corr, dtau, nsub);
      const MxColArgs ca = col_args(s, corr, dtau, nsub);
      const bool damp = corr && st->divdamp4 > 0.0;
      // lean column with damping: the corrector's undamped vn^{n+1} goes to Avn0_32 (dead once
      // the edge tendency has read it, element by element), the damping's edge update is
      // formed inside the gather, which writes the damped vn^{n+1} and the step-mean flux
      const bool fused = lean && damp;
      MxEdgeArgs ead = ea;
      ead.skip_flux = damp ? 1 : 0;
      ead.upwind_theta = st->upwind_theta ? 1 : 0;
      if (fused) ead.vn_out = s.Avn0_32;
      for (int kind : {K_MX_VERTEX, K_MX_EDGE, K_MX_CELL_KE, K_MX_EDGE_TEND}) {
        if (diag_ahead && (kind == K_MX_EDGE || kind == K_MX_CELL_KE)) continue;
        if (diag_ahead && kind == K_MX_EDGE_TEND) {
          cudaStreamWaitEvent(stream, st->join_ev, 0);
          diag_ahead = false;
        }
        if (kind == K_MX_EDGE_TEND && s.topo.on) topo_stage32(st, ea.vn, s.vt32, ea.w, ea.exp, stream);
        prof_begin(stream, kind);
        launch_kind(kind, tile(kind), G, s, ead, ca, (float)dt, stream);
        prof_end(stream);
      }
      if (damp) {
        // scratch until the next stage's diagnostics: Kc32 holds the divergence, vt32 (an
        // edge array, larger than a cell array) its Laplacian
        const double abar = st->abar;
        MxDDArgs da;
        da.L = s.vt32; da.rho = ea.rho; da.thv = ea.thv;
        da.dz_e = s.topo.on ? s.topo.dz_e32 : nullptr;
        da.vn = s.vn32; da.phi = s.F32; da.gth = s.G32; da.mflx = s.mflx;
        da.scale = (float)(st->divdamp4 * abar * abar); da.inv_nsub = 1.0 / nsub;
        da.upwind_theta = st->upwind_theta ? 1 : 0;
        const unsigned nbc8 = (unsigned)((nc + 7) / 8), nbe8 = (unsigned)((G.ne + 7) / 8);
        prof_begin(stream, K_DIVDAMP);
        k_mx_dd_div<<<nbc8, 256, 0, stream>>>(G, fused ? s.Avn0_32 : s.vn32, s.Kc32);
        k_mx_dd_lap<<<nbc8, 256, 0, stream>>>(G, s.Kc32, s.vt32);
        if (!fused) k_mx_dd_edge<<<nbe8, 256, 0, stream>>>(G, da);
        prof_end(stream);
      }
      if (lean) {
        MxLeanArgs la = lean_args(s, corr, dtau, nsub);
        if (fused) {
          la.dd_vn = s.Avn0_32; la.dd_L = s.vt32; la.dd_rho = ea.rho; la.dd_thv = ea.thv;
          la.dd_out = s.vn32; la.mflx = s.mflx;
          la.dd_scale = (float)(st->divdamp4 * st->abar * st->abar);
          la.dd_upwind = st->upwind_theta ? 1 : 0;
        }
        const TileChoice t = tile(K_MX_COLUMN_PREP);
        const unsigned nb = (unsigned)((nc + 31) / 32);
        prof_begin(stream, K_MX_LEAN_GATHER);
        if (corr && fused) {
          launch_lean_gather_dd(G, la, s.topo.on, stream);
        } else {
          with_lanes(t.lanes, [&](auto L) {
            constexpr int LPE = decltype(L)::value;
            if (s.topo.on) {
              if (corr) k_mx_lean_gather<LPE, true, false, true><<<nb, t.block, 0, stream>>>(G, la);
              else k_mx_lean_gather<LPE, false, false, true><<<nb, t.block, 0, stream>>>(G, la);
            } else {
              if (corr) k_mx_lean_gather<LPE, true><<<nb, t.block, 0, stream>>>(G, la);
              else k_mx_lean_gather<LPE, false><<<nb, t.block, 0, stream>>>(G, la);
            }
          });
        }
        prof_end(stream);
        if (overlap && (!corr || it + 1 < nsub)) fork_diag(!corr);
        prof_begin(stream, K_MX_LEAN);
        // the autotuner times the predictor's column (the corrector updates S^n in place and
        // cannot be run again on the state); the corrector, whose extra live values spill at
        // 48 registers, keeps the default shape (56 registers, no spills) unless one is forced
        const TileChoice tc = st->tile[K_MX_LEAN].lanes ? st->tile[K_MX_LEAN] : kLeanDefault;
        const TileChoice tcc = st->tile_forced[K_MX_LEAN] ? tc : kLeanDefault;
        if (corr) launch_lean_column<true>(G, la, tcc, s.topo.on, stream);
        else launch_lean_column<false>(G, la, tc, s.topo.on, stream);
        prof_end(stream);
        continue;
      }
      if (s.fac64) {
        const TileChoice t = tile(K_MX_COLUMN_PREP);
        const unsigned nb = (unsigned)((nc + 31) / 32);
        prof_begin(stream, K_MX_COLUMN_PREP);
        with_lanes(t.lanes, [&](auto L) {
          constexpr int LPE = decltype(L)::value;
          if (corr) k_mx_gather_tile<LPE, true><<<nb, t.block, 0, stream>>>(G, ca);
          else k_mx_gather_tile<LPE, false><<<nb, t.block, 0, stream>>>(G, ca);
        });
        prof_end(stream);
      }
      prof_begin(stream, K_MX_COLUMN);
      if (corr) launch_mx_column<true>(G, ca, s.topo.on, stream);
      else launch_mx_column<false>(G, ca, s.topo.on, stream);
      prof_end(stream);
    }
  }
  const MxEdgeArgs ea = edge_args(s, false, dtau, nsub);
  const MxColArgs ca = col_args(s, false, dtau, nsub);
  prof_begin(stream, K_MX_DIFF_VERTEX);
  launch_kind(K_MX_DIFF_VERTEX, tile(K_MX_DIFF_VERTEX), G, s, ea, ca, (float)dt, stream);
  prof_end(stream);
  if (st->diff4 > 0.0) {
    // dead after the substeps: ae32 (edges) holds L(vn), w32_s its curl, exp32_s its divergence
    const double abar = st->abar;
    prof_begin(stream, K_DIFF4);
    k_mx_bd_lap<<<(unsigned)((G.ne + 7) / 8), 256, 0, stream>>>(G, s.zeta32, s.Kc32, s.ae32);
    k_mx_bd_curldiv<<<(unsigned)((G.nv + nc + 7) / 8), 256, 0, stream>>>(G, s.ae32, s.w32_s, s.exp32_s);
    prof_end(stream);
    prof_begin(stream, K_MX_DIFF_EDGE);
    const unsigned nbe8 = (unsigned)((G.ne + 7) / 8);
    k_mx_diff_edge_bd<<<nbe8, 256, 0, stream>>>(G, s.vn32, s.uvx32, s.uvy32, s.uvz32, s.zeta32, s.Kc32, s.thv32,
                                                s.vt32, (float)dt, s.exp32_s, s.w32_s, (float)(st->diff4 * abar * abar));
    prof_end(stream);
  } else {
    prof_begin(stream, K_MX_DIFF_EDGE);
    launch_kind(K_MX_DIFF_EDGE, tile(K_MX_DIFF_EDGE), G, s, ea, ca, (float)dt, stream);
    prof_end(stream);
  }
  prof_begin(stream, K_MX_DIFF_THETA);
  k_mx_diff_theta<<<blocks_for(nc, 128), 128, 0, stream>>>(G, s.vt32, s.thv, s.ex, s.thv32, s.exp32, (float)dt,
                                                           s.topo.on ? s.topo.exref_c : nullptr);
  prof_end(stream);
}

// ---------------------------------------------------------------- self-test of the integer-pipe conversions
// and of the Newton-Raphson reciprocal
namespace {
__device__ inline uint64_t st_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// n random binary32 normals and zeros, and n random binary64 values in the binary32
// normal range (including exact halfway cases), against the hardware conversions
__global__ void k_selftest_conv(int64_t n, unsigned* fails) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t r = st_mix(0x9E3779B97F4A7C15ull * (uint64_t)(i + 1));
  unsigned u = (unsigned)r;
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0xffu) u &= ~0x40000000u;                           // keep it finite
  if (e == 0u) u &= 0x80000000u;                               // normals and signed zeros only
  const float f = __uint_as_float(u);
  const double a = f32_to_f64(f), b = (double)f;
  if (__double_as_longlong(a) != __double_as_longlong(b)) atomicAdd(fails, 1u);
  // binary64 in the binary32 normal range; every 4th value sits exactly halfway
  const uint64_t r2 = st_mix(r);
  uint64_t bits = r2 & 0x800fffffffffffffull;
  const unsigned ee = 897u + (unsigned)((r2 >> 52) % 254u);   // up to the largest binary32 exponent
  bits |= (uint64_t)ee << 52;
  if ((i & 3) == 0) bits = (bits & ~0x1fffffffull) | 0x10000000ull;
  const double d = __longlong_as_double((long long)bits);
  const float x = f64_to_f32(d), y = (float)d;
  if (__float_as_uint(x) != __float_as_uint(y)) atomicAdd(fails, 1u);
  if (i == 0) {
    if (__double_as_longlong(f32_to_f64(-0.0f)) != __double_as_longlong(-0.0)) atomicAdd(fails, 1u);
    if (__float_as_uint(f64_to_f32(0.0)) != 0u) atomicAdd(fails, 1u);
  }
  // outside the binary32 normal range, the documented mapping: binary64 below it to a signed
  // zero, above it (infinities and NaNs included) to a signed infinity, binary32 subnormals
  // to a signed zero
  const uint64_t r5 = st_mix(r2 + 1);
  const uint64_t sg = r5 & 0x8000000000000000ull, man = r5 & 0x000fffffffffffffull;
  const uint64_t elow = (r5 >> 52) % 897u, ehigh = 1151u + (r5 >> 40) % 897u;
  const unsigned s32 = (unsigned)(sg >> 32);
  if (__float_as_uint(f64_to_f32(__longlong_as_double((long long)(sg | (elow << 52) | man)))) != s32)
    atomicAdd(fails, 1u);
  if (__float_as_uint(f64_to_f32(__longlong_as_double((long long)(sg | (ehigh << 52) | man)))) != (s32 | 0x7f800000u))
    atomicAdd(fails, 1u);
  const unsigned us = s32 | ((unsigned)(r5 >> 8) & 0x007fffffu);
  if (__double_as_longlong(f32_to_f64(__uint_as_float(us))) != (long long)((uint64_t)s32 << 32)) atomicAdd(fails, 1u);
  // Newton-Raphson reciprocal: within one ulp of the IEEE quotient 1/x, and a * recip64(b)
  // within two ulps of a / b, for x, b of either sign with exponents in [-120, 120]
  const uint64_t r3 = st_mix(r2 ^ 0xD1B54A32D192ED03ull);
  const uint64_t r4 = st_mix(r3);
  const uint64_t ex3 = 903u + (r3 >> 56) % 241u, ex4 = 903u + (r4 >> 56) % 241u;
  const double xv = __longlong_as_double((long long)((r3 & 0x800fffffffffffffull) | (ex3 << 52)));
  const double av = __longlong_as_double((long long)((r4 & 0x800fffffffffffffull) | (ex4 << 52)));
  const double q1 = 1.0 / xv, y1 = recip64(xv);
  const long long dq = __double_as_longlong(q1) - __double_as_longlong(y1);
  if (dq > 1 || dq < -1) atomicAdd(fails, 1u);
  const double q2 = av / xv, y2 = av * recip64(xv);
  const long long dq2 = __double_as_longlong(q2) - __double_as_longlong(y2);
  if (dq2 > 2 || dq2 < -2) atomicAdd(fails, 1u);
}
}  // namespace

int selftest_conversions(int64_t n, unsigned* host_fails) {
  unsigned* d = nullptr;
  ICON_CUDA(cudaMalloc(&d, sizeof(unsigned)));
  cudaMemset(d, 0, sizeof(unsigned));
  k_selftest_conv<<<blocks_for(n, 256), 256>>>(n, d);
  cudaError_t e = cudaMemcpy(host_fails, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "icon_selftest");
  return ICON_OK;
}

// ---------------------------------------------------------------- persistent ensemble kernel
//
// All members of an ensemble (grids of any size, one precision, one level count)
// advance through one step in ONE cooperative launch: every phase of the step
// (vertex, edge diagnostics, cell kinetic energy, edge tendency, column solve for
// predictor and corrector, then the diffusion phases) is a static work list over
// (member, entity) or (member, column) shared by all blocks, separated by a grid
// barrier. The column-input gather is a work list over (member, 32-cell tile) taken
// by whole blocks. Blocks of 128 threads held to 64 registers and a 21 KB gather tile
// keep 8 blocks (32 warps) on every SM: the stencil phases are latency bound and gain
// more from occupancy than they lose to the few spilled kernel-level registers. The
// barrier spins a bounded number of times; if it runs out it sets the timeout bit of
// the status word, every block leaves at its next barrier and the kernel returns
// normally.
namespace {

struct MemberDev {
  MxGeo G;
  MxEdgeArgs ea[2];
  MxColArgs ca[2];
  double* mflx;
  double* wflx;
  double* colconst;
  const double* ex_ref;
  float *vn32, *uvx32, *uvy32, *uvz32, *zeta32, *Kc32, *thv32, *exp32, *wv32, *vt32;
  double *thv, *ex;
  double dtau, dt;
  int64_t off_v, off_e, off_c;  // this member's first item in each work list
  int64_t off_t;                // first 32-cell tile of the column-input gather
  MxDDArgs dd;                  // fourth-order divergence damping of the corrector's vn
  int damp;                     // 1 if the member damps (dd.scale > 0)
  MxLeanArgs la[2];             // lean column of the predictor and the corrector
};

struct EnsArgs {
  const MemberDev* m;
  int nm;
  int nsub;
  int64_t tot_v, tot_e, tot_c, tot_t;
  unsigned* bar;                // [0] arrivals, [1] generation
  unsigned* status;             // ensemble status word (bit 1: barrier timeout)
  long long spin_limit;
  int skip_first_barrier;       // test hook: block 0 does not arrive at the first barrier
  int any_damp;                 // some member damps: the corrector runs the damping phases
  unsigned long long* prof;     // if set: (phase kind, global ns) after every barrier, by block 0
  int prof_max;                 // entries (pairs) prof holds
};

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline int find_member(const int64_t* off, int nm, int64_t item) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// warp-level work list: warp w takes items [K w, K w + K), then the next chunk K * nwarps
// further on; the member is looked up once per chunk and advanced at member boundaries
template <int K, typename F>
__device__ inline void warp_items(const int64_t* off, int nm, int64_t tot, int64_t gwarp, int64_t nwarps, F f) {
  for (int64_t i0 = gwarp * K; i0 < tot; i0 += nwarps * K) {
    int m = find_member(off, nm, i0);
    int64_t next = m + 1 < nm ? off[m + 1] : tot;
    for (int j = 0; j < K; ++j) {
      const int64_t i = i0 + j;
      if (i >= tot) break;
      while (i >= next) {
        ++m;
        next = m + 1 < nm ? off[m + 1] : tot;
      }
      f(m, i - off[m]);
    }
  }
}

// the same work list taken two items at a time: when both items of a pair belong to one
// member, the two half-warps take one each with 16 lanes over the levels (f16(m, first item
// of the pair)); a pair that straddles a member boundary is taken by the whole warp, one
// item after the other (f32(m, item))
template <int K, typename F16, typename F32>
__device__ inline void warp_pairs(const int64_t* off, int nm, int64_t tot, int64_t gwarp, int64_t nwarps, F16 f16,
                                  F32 f32) {
  static_assert(K % 2 == 0, "pairs");
  for (int64_t i0 = gwarp * K; i0 < tot; i0 += nwarps * K) {
    int m = find_member(off, nm, i0);
    int64_t next = m + 1 < nm ? off[m + 1] : tot;
    for (int j = 0; j < K; j += 2) {
      const int64_t i = i0 + j;
      if (i >= tot) break;
      while (i >= next) {
        ++m;
        next = m + 1 < nm ? off[m + 1] : tot;
      }
      if (i + 1 < next) {
        f16(m, i - off[m]);
      } else {
        f32(m, i - off[m]);
        if (i + 1 < tot) {
          while (i + 1 >= next) {
            ++m;
            next = m + 1 < nm ? off[m + 1] : tot;
          }
          f32(m, i + 1 - off[m]);
        }
      }
    }
  }
}

// bounded grid barrier; returns false (for every thread of the block) once any block gave up
__device__ bool grid_barrier(const EnsArgs& A, bool skip) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = A.bar + 1;
    volatile unsigned* vstat = A.status;
    int ok = ((*vstat) & 2u) == 0;
    if (ok && !skip) {
      const unsigned gen = *vgen;
      __threadfence();
      const unsigned arrived = atomicAdd(A.bar, 1u);
      if (arrived == gridDim.x - 1) {
        A.bar[0] = 0;
        __threadfence();
        atomicAdd(A.bar + 1, 1u);
      } else {
        long long spins = 0;
        while (*vgen == gen) {
          if ((*vstat) & 2u) { ok = 0; break; }
          if (++spins > A.spin_limit) {
            atomicOr(A.status, 2u);
            ok = 0;
            break;
          }
          __nanosleep(100);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr int kChunk = 4;   // consecutive work items per warp

// Each warp copies its current member's geometry and phase arguments into shared memory
// when the member changes. Read from the global member table, every field would be
// reloaded after each store of a phase (a global store may alias the table); read from
// shared memory they cannot alias, as the kernel parameters of the per-state kernels
// cannot. (Keeping a phase out of line, with registers of its own, measured slower: the
// call saves and restores the caller's registers.)
union MemberArgs {
  MxEdgeArgs ea;
  MxLeanArgs la;
};
static_assert(sizeof(MxGeo) % 8 == 0 && sizeof(MxEdgeArgs) % 8 == 0 && sizeof(MxLeanArgs) % 8 == 0,
              "member structs are copied in 8-byte words");
__shared__ MxGeo s_ens_geo[4];
__shared__ MemberArgs s_ens_arg[4];

struct SlotCache {
  const MemberDev* mt;
  int geo_m = -1, arg_m = -1;
  __device__ explicit SlotCache(const MemberDev* t) : mt(t) {}
  __device__ static void copy(void* dst, const void* src, int bytes) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int i = lane; i < bytes / 8; i += 32)
      static_cast<unsigned long long*>(dst)[i] = static_cast<const unsigned long long*>(src)[i];
    __syncwarp();
  }
  __device__ const MxGeo& geo(int m) {
    MxGeo& g = s_ens_geo[threadIdx.x >> 5];
    if (m != geo_m) {
      copy(&g, &mt[m].G, sizeof(MxGeo));
      geo_m = m;
    }
    return g;
  }
  __device__ const MxEdgeArgs& edge(int m, int stage) {
    MxEdgeArgs& e = s_ens_arg[threadIdx.x >> 5].ea;
    if (m != arg_m) {
      copy(&e, &mt[m].ea[stage], sizeof(MxEdgeArgs));
      arg_m = m;
    }
    return e;
  }
  __device__ const MxLeanArgs& lean(int m, int stage) {
    MxLeanArgs& l = s_ens_arg[threadIdx.x >> 5].la;
    if (m != arg_m) {
      copy(&l, &mt[m].la[stage], sizeof(MxLeanArgs));
      arg_m = m;
    }
    return l;
  }
};

// shared tiles of the persistent kernel: the lean form needs only the lean gather tile and
// the column's shadow transposes (8-level chunks; 4-level chunks, which would leave the
// stencil phases more L1, measured 13 % slower in the column and no faster elsewhere); the
// stored-factor forms need the gather and corrector-update tiles
constexpr int kEnsLeanCH = 8;
template <bool LEAN>
union EnsTiles {
  GatherTile<16> g;
  UpdTile u;
  LeanGatherTile<16> lg;
  LeanTile<8> lt[4];
};
template <>
union EnsTiles<true> {
  LeanGatherTile<16> lg;
  LeanTile<kEnsLeanCH> lt[4];
};

template <int NMAX, bool ALLFAC, bool LEAN, int MINB = 8>
__global__ void __launch_bounds__(128, MINB) k_ensemble_step(EnsArgs A) {
  __shared__ int64_t s_off_v[64], s_off_e[64], s_off_c[64], s_off_t[64];
  __shared__ EnsTiles<LEAN> tiles;
  for (int i = threadIdx.x; i < A.nm; i += blockDim.x) {
    s_off_v[i] = A.m[i].off_v;
    s_off_e[i] = A.m[i].off_e;
    s_off_c[i] = A.m[i].off_c;
    s_off_t[i] = A.m[i].off_t;
  }
  __syncthreads();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nwarps = nthreads >> 5;
  const int64_t gwarp = gtid >> 5;
  const int lane = threadIdx.x & 31;
  bool first = true;
  // phase timer (icon_ensemble_step_profile): block 0 stamps the global timer at the start
  // and as it leaves each barrier, with the kind of the phase that barrier closes
  const bool stamps = A.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0;
  int nstamp = 0;
  auto stamp = [&](int kind) {
    if (stamps && nstamp < A.prof_max) {
      A.prof[2 * nstamp] = (unsigned long long)kind;
      A.prof[2 * nstamp + 1] = global_ns();
      ++nstamp;
    }
  };
  auto sync = [&](int kind) {
    const bool skip = first && A.skip_first_barrier && blockIdx.x == 0;
    first = false;
    const bool ok = grid_barrier(A, skip);
    stamp(kind);
    return ok;
  };
  stamp(ICON_ENS_PHASE_COUNT);                       // the start

  SlotCache sc(A.m);
  auto geo = [&](int m) -> const MxGeo& { return sc.geo(m); };
  auto edge_args_of = [&](int m, int stage) -> const MxEdgeArgs& { return sc.edge(m, stage); };
  auto lean_args_of = [&](int m, int stage) -> const MxLeanArgs& { return sc.lean(m, stage); };
  int& arg_m = sc.arg_m;

  // phase 0: zero the accumulators
  for (int m = 0; m < A.nm; ++m) {
    const MemberDev& M = A.m[m];
    const int64_t ne = M.G.ne * M.G.ld, nh = M.G.nc * (M.G.N + 1);
    for (int64_t i = gtid; i < ne; i += nthreads) M.mflx[i] = 0.0;
    for (int64_t i = gtid; i < nh; i += nthreads) M.wflx[i] = 0.0;
  }
  if (!sync(ICON_ENS_PH_ZERO)) return;
  for (int it = 0; it < A.nsub; ++it) {
    for (int stage = 0; stage < 2; ++stage) {
      // the stencil phases take two entities per warp (16 lanes over the levels each), as
      // the per-state kernels' tuned tiles do
      warp_pairs<kChunk>(
          s_off_v, A.nm, A.tot_v, gwarp, nwarps,
          [&](int m, int64_t j) {
            const MemberDev& M = A.m[m];
            mx_vertex_item<16>(geo(m), M.ea[stage].vn, M.ea[stage].w, M.zeta32, M.wv32, j + (lane >> 4), lane & 15);
          },
          [&](int m, int64_t j) {
            const MemberDev& M = A.m[m];
            mx_vertex_item<32>(geo(m), M.ea[stage].vn, M.ea[stage].w, M.zeta32, M.wv32, j, lane);
          });
      if (!sync(ICON_ENS_PH_VERTEX)) return;
      warp_pairs<kChunk>(
          s_off_e, A.nm, A.tot_e, gwarp, nwarps,
          [&](int m, int64_t j) {
            const MemberDev& M = A.m[m];
            mx_edge_diag_item<16>(geo(m), M.ea[stage].vn, M.vt32, j + (lane >> 4), lane & 15);
          },
          [&](int m, int64_t j) {
            const MemberDev& M = A.m[m];
            mx_edge_diag_item<32>(geo(m), M.ea[stage].vn, M.vt32, j, lane);
          });
      if (!sync(ICON_ENS_PH_EDGE_DIAG)) return;
      warp_pairs<kChunk>(
          s_off_c, A.nm, A.tot_c, gwarp, nwarps,
          [&](int m, int64_t j) {
            const MemberDev& M = A.m[m];
            mx_cell_ke_item<16>(geo(m), M.ea[stage].vn, M.vt32, M.Kc32, j + (lane >> 4), lane & 15);
          },
          [&](int m, int64_t j) {
            const MemberDev& M = A.m[m];
            mx_cell_ke_item<32>(geo(m), M.ea[stage].vn, M.vt32, M.Kc32, j, lane);
          });
      if (!sync(ICON_ENS_PH_CELL_KE)) return;
      arg_m = -1;
      warp_pairs<kChunk>(
          s_off_e, A.nm, A.tot_e, gwarp, nwarps,
          [&](int m, int64_t j) {
            mx_edge_tend_item<16, false, false>(geo(m), edge_args_of(m, stage), j + (lane >> 4), lane & 15);
          },
          [&](int m, int64_t j) { mx_edge_tend_item<32, false, false>(geo(m), edge_args_of(m, stage), j, lane); });
      if (!sync(ICON_ENS_PH_EDGE_TEND)) return;
      if (stage == 1 && A.any_damp) {
        // divergence damping of vn^{n+1}: cell divergence (into Kc32), its Laplacian (into
        // vt32), then the edge update with the fluxes the edge tendency left out
        warp_items<kChunk>(s_off_c, A.nm, A.tot_c, gwarp, nwarps, [&](int m, int64_t j) {
          const MemberDev& M = A.m[m];
          if (M.damp) mx_dd_div_item(geo(m), M.dd.vn, M.Kc32, j, lane);
        });
        if (!sync(ICON_ENS_PH_DD_DIV)) return;
        warp_items<kChunk>(s_off_c, A.nm, A.tot_c, gwarp, nwarps, [&](int m, int64_t j) {
          const MemberDev& M = A.m[m];
          if (M.damp) mx_dd_lap_item(geo(m), M.Kc32, M.vt32, j, lane);
        });
        if (!sync(ICON_ENS_PH_DD_LAP)) return;
        if (!LEAN) {     // the lean column's gather forms the damped fluxes itself
          warp_items<kChunk>(s_off_e, A.nm, A.tot_e, gwarp, nwarps, [&](int m, int64_t j) {
            const MemberDev& M = A.m[m];
            if (M.damp) mx_dd_edge_item(M.G, M.dd, j, lane);
          });
          if (!sync(ICON_ENS_PH_DD_EDGE)) return;
        }
      }
      // column-input gather: one 32-cell tile per block at a time (members without
      // stored factors have no tiles)
      arg_m = -1;
      for (int64_t t = blockIdx.x; t < A.tot_t; t += gridDim.x) {
        const int m = find_member(s_off_t, A.nm, t);
        const MemberDev& M = A.m[m];
        const int64_t c0 = (t - M.off_t) * kGatherCells;
        if constexpr (LEAN) {
          const MxGeo& G = geo(m);
          const MxLeanArgs& la = lean_args_of(m, stage);
          if (stage == 0) mx_lean_gather_body<16, false>(G, la, c0, tiles.lg);
          else if (M.damp) mx_lean_gather_body<16, true, true>(G, la, c0, tiles.lg);
          else mx_lean_gather_body<16, true>(G, la, c0, tiles.lg);
        } else {
          if (stage == 0) mx_gather_tile_body<16, false>(M.G, M.ca[0], c0, tiles.g);
          else mx_gather_tile_body<16, true>(M.G, M.ca[1], c0, tiles.g);
        }
      }
      if (!sync(ICON_ENS_PH_GATHER)) return;
      if constexpr (LEAN) {
        // lean column: one warp per 32-column tile, both sweeps and the updates in one pass
        arg_m = -1;
        for (int64_t t = gwarp; t < A.tot_t; t += nwarps) {
          const int m = find_member(s_off_t, A.nm, t);
          const MemberDev& M = A.m[m];
          const int64_t c0 = (t - M.off_t) * kGatherCells;
          LeanTile<kEnsLeanCH>& lt = tiles.lt[threadIdx.x >> 5];
          const MxGeo& G = geo(m);
          const MxLeanArgs& la = lean_args_of(m, stage);
          if (stage == 0) mx_lean_column_item<false, 2, kEnsLeanCH>(G, la, c0 + lane, c0, lane, lt);
          else mx_lean_column_item<true, 2, kEnsLeanCH>(G, la, c0 + lane, c0, lane, lt);
        }
        if (!sync(ICON_ENS_PH_COLUMN)) return;
      } else {
        for (int64_t i = gtid; i < A.tot_c; i += nthreads) {
          const int m = find_member(s_off_c, A.nm, i);
          const MemberDev& M = A.m[m];
          if (ALLFAC) {
            if (stage == 0) mx_column_fac_item<NMAX, false>(M.G, M.ca[0], i - M.off_c);
            else mx_corr_solve_item(M.G, M.ca[1], i - M.off_c);
          } else {
            if (stage == 0) mx_column_any<NMAX, false>(M.G, M.ca[0], i - M.off_c);
            else mx_column_any<NMAX, true>(M.G, M.ca[1], i - M.off_c);
          }
        }
        if (ALLFAC && stage == 1) {
          // corrector updates: element-parallel 32-cell tiles (the member's tile list)
          if (!sync(ICON_ENS_PH_COLUMN)) return;
          static_assert(kUpdCells == kGatherCells, "the corrector update reuses the gather tile list");
          for (int64_t t = blockIdx.x; t < A.tot_t; t += gridDim.x) {
            const int m = find_member(s_off_t, A.nm, t);
            const MemberDev& M = A.m[m];
            if (!mx_corr_update_tile(M.G, M.ca[1], (t - M.off_t) * kUpdCells, tiles.u)) atomicOr(M.ca[1].status, 1u);
            __syncthreads();
          }
        }
        if (!sync(ALLFAC && stage == 1 ? ICON_ENS_PH_CORR_UPDATE : ICON_ENS_PH_COLUMN)) return;
      }
    }
  }
  // diffusion
  for (int64_t i = gwarp; i < A.tot_v + A.tot_c; i += nwarps) {
    if (i < A.tot_v) {
      const int m = find_member(s_off_v, A.nm, i);
      const MemberDev& M = A.m[m];
      mx_diff_vertex_item<32>(M.G, M.vn32, M.uvx32, M.uvy32, M.uvz32, M.zeta32, i - M.off_v, lane);
    } else {
      const int64_t j = i - A.tot_v;
      const int m = find_member(s_off_c, A.nm, j);
      const MemberDev& M = A.m[m];
      mx_diff_div_item<32>(M.G, M.vn32, M.Kc32, j - M.off_c, lane);
    }
  }
  if (!sync(ICON_ENS_PH_DIFF_VERTEX)) return;
  warp_items<kChunk>(s_off_e, A.nm, A.tot_e, gwarp, nwarps, [&](int m, int64_t j) {
    const MemberDev& M = A.m[m];
    mx_diff_edge_item<32>(M.G, M.vn32, M.uvx32, M.uvy32, M.uvz32, M.zeta32, M.Kc32, M.thv32, M.vt32, (float)M.dt,
                          j, lane);
  });
  if (!sync(ICON_ENS_PH_DIFF_EDGE)) return;
  for (int64_t i = gtid; i < A.tot_c; i += nthreads) {
    const int m = find_member(s_off_c, A.nm, i);
    const MemberDev& M = A.m[m];
    mx_diff_theta_item(M.G, M.vt32, M.thv, M.ex, M.thv32, M.exp32, (float)M.dt, i - M.off_c);
  }
  stamp(ICON_ENS_PH_DIFF_THETA);                     // block 0's own end of the last phase
}

__global__ void k_ens_colconst(const MemberDev* m, int nm) {
  const int i = blockIdx.x;
  if (i >= nm) return;
  const MemberDev& M = m[i];
  const MxGeo& G = M.G;
  const int ld = G.ld, N = G.N;
  const double dtau = M.dtau;
  double* cc = M.colconst;
  for (int h = threadIdx.x; h < ld; h += blockDim.x) {
    const bool interior = h > 0 && h < N;
    cc[CC_WU * ld + h] = h <= N ? G.wu[h] : 0.0;
    cc[CC_WL * ld + h] = h <= N ? G.wl[h] : 0.0;
    cc[CC_CA * ld + h] = interior ? dtau * kBeta * kCpd / G.dzh[h] : 0.0;
    cc[CC_CX * ld + h] = interior ? (1.0 - kBeta) * kCpd / G.dzh[h] : 0.0;
    cc[CC_DAMP * ld + h] = h <= N ? 1.0 / (1.0 + dtau * G.ray[h]) : 1.0;
    cc[CC_DTBDZ * ld + h] = h < N ? dtau * kBeta / G.dz[h] : 0.0;
    cc[CC_DT1BDZ * ld + h] = h < N ? dtau * (1.0 - kBeta) / G.dz[h] : 0.0;
    cc[CC_EXREF * ld + h] = h < N ? M.ex_ref[h] : 0.0;
  }
}

}  // namespace

int ensemble_prepare(EnsembleDev& E, icon_state* const* members, int n, const double* dts, int nsub) {
  if (n > 64) {
    set_error("icon_ensemble_step: at most 64 members in one persistent launch");
    return ICON_EINVAL;
  }
  std::vector<MemberDev> host(n);
  int64_t ov = 0, oe = 0, oc = 0, ot = 0;
  int N = -1;
  bool all_fac = true;
  bool any_damp = false;
  // the lean column when every member has its buffers (flat mixed states); otherwise the
  // stored-factor column, whose buffers lean-form members get here when they fit (else
  // that member's column recomputes its factors)
  bool all_lean = true;
  for (int i = 0; i < n; ++i) all_lean = all_lean && members[i]->s.ln_B != nullptr;
  if (!all_lean)
    for (int i = 0; i < n; ++i)
      if (!members[i]->s.fac64 && members[i]->s.ln_B) alloc_mixed_factors(members[i]);
  E.lean_consts.clear();
  for (int i = 0; i < n; ++i) {
    icon_state* st = members[i];
    StateDev& s = st->s;
    if (s.precision != ICON_MIXED) {
      set_error("icon_ensemble_step: the persistent ensemble runs mixed-precision members");
      return ICON_EINVAL;
    }
    MemberDev& M = host[i];
    M.G = make_mx_geo(st->grid, s);
    if (N >= 0 && M.G.N != N) {
      set_error("icon_ensemble_step: members must share one level count");
      return ICON_EINVAL;
    }
    N = M.G.N;
    const double dtau = dts[i] / nsub;
    M.dtau = dtau;
    M.dt = dts[i];
    for (int stage = 0; stage < 2; ++stage) {
      M.ea[stage] = edge_args(s, stage == 1, dtau, nsub);
      M.ca[stage] = col_args(s, stage == 1, dtau, nsub);
    }
    M.damp = st->divdamp4 > 0.0 ? 1 : 0;
    M.ea[1].skip_flux = M.damp;
    M.dd.L = s.vt32; M.dd.rho = M.ea[1].rho; M.dd.thv = M.ea[1].thv; M.dd.dz_e = nullptr;
    M.dd.vn = s.vn32; M.dd.phi = s.F32; M.dd.gth = s.G32; M.dd.mflx = s.mflx;
    M.dd.scale = (float)(st->divdamp4 * st->abar * st->abar); M.dd.inv_nsub = 1.0 / nsub;
    M.dd.upwind_theta = 0;
    any_damp = any_damp || M.damp;
    M.mflx = s.mflx; M.wflx = s.wflx; M.colconst = s.colconst; M.ex_ref = s.ex_ref;
    M.vn32 = s.vn32; M.uvx32 = s.uvx32; M.uvy32 = s.uvy32; M.uvz32 = s.uvz32; M.zeta32 = s.zeta32;
    M.Kc32 = s.Kc32; M.thv32 = s.thv32; M.exp32 = s.exp32; M.thv = s.thv; M.ex = s.ex;
    M.wv32 = s.wv32; M.vt32 = s.vt32;
    M.off_v = ov; M.off_e = oe; M.off_c = oc; M.off_t = ot;
    ov += M.G.nv; oe += M.G.ne; oc += M.G.nc;
    if (s.fac64 || all_lean) ot += (M.G.nc + kGatherCells - 1) / kGatherCells;
    else all_fac = false;
    if (all_lean) {
      for (int stage = 0; stage < 2; ++stage) M.la[stage] = lean_args(s, stage == 1, dtau, nsub);
      if (M.damp) {
        // as the per-state lean step: undamped vn^{n+1} in Avn0_32, damping fused into the gather
        M.ea[1].vn_out = s.Avn0_32;
        M.dd.vn = s.Avn0_32;
        MxLeanArgs& la = M.la[1];
        la.dd_vn = s.Avn0_32; la.dd_L = s.vt32; la.dd_rho = M.ea[1].rho; la.dd_thv = M.ea[1].thv;
        la.dd_out = s.vn32; la.mflx = s.mflx; la.dd_scale = M.dd.scale; la.dd_upwind = 0;
      }
      E.lean_consts.push_back({M.G.N, M.G.ld, M.G.nc, M.G.wu, M.G.wl, M.G.dzh, M.G.dz, M.G.ray, s.ex_ref, dtau,
                               s.ln_cd, s.ln_cf, M.G.div_wa, M.G.inv_Ac, s.ln_dwa, s.ln_cw32});
    }
  }
  if (all_lean) all_fac = false;
  E.N = N;
  E.tot_v = ov; E.tot_e = oe; E.tot_c = oc; E.tot_t = ot;
  E.all_fac = all_fac;
  E.all_lean = all_lean;
  E.any_damp = any_damp;
  E.nm = n;
  E.nsub = nsub;
  if (!E.members) {
    E.members = E.arena.get(sizeof(MemberDev) * 64);
    static_assert(sizeof(MemberDev) * 64 < (1 << 20), "member table");
    E.bar = E.arena.get_n<unsigned>(64);
    if (!E.members || !E.bar) {
      set_error("icon_ensemble_step: out of device memory");
      return ICON_ENOMEM;
    }
  }
  cudaStream_t st = current_stream();
  ICON_CUDA(cudaMemcpyAsync(E.members, host.data(), sizeof(MemberDev) * n, cudaMemcpyHostToDevice, st));
  ICON_CUDA(cudaMemsetAsync(E.bar, 0, 64 * sizeof(unsigned), st));
  ICON_CUDA(cudaStreamSynchronize(st));
  return ICON_OK;
}

int ensemble_launch(EnsembleDev& E, cudaStream_t st, unsigned long long* prof, int prof_max) {
  EnsArgs A;
  A.prof = prof;
  A.prof_max = prof_max;
  A.m = static_cast<const MemberDev*>(E.members);
  A.nm = E.nm;
  A.nsub = E.nsub;
  A.tot_v = E.tot_v; A.tot_e = E.tot_e; A.tot_c = E.tot_c; A.tot_t = E.tot_t;
  A.bar = E.bar;
  A.status = E.bar + 8;
  A.spin_limit = E.spin_limit;
  A.skip_first_barrier = E.test_skip_barrier;
  A.any_damp = E.any_damp ? 1 : 0;
  void (*kern)(EnsArgs);
  // The lean form keeps 8 CTAs per SM (64 registers, a few hundred bytes of spills): on a
  // 64-member R2B4/R2B5 ensemble it measured faster than 7, 6, 5 and 4 CTAs per SM (72 to
  // 120 registers, fewer or no spills) in every phase but the edge tendency, which gains
  // nothing from the extra registers; the grid barriers wait on the slowest CTA and more
  // resident warps hide that.
  if (E.all_lean)      // the lean column has no level arrays
    kern = k_ensemble_step<32, false, true, 8>;
  else if (E.N <= 32) kern = E.all_fac ? k_ensemble_step<32, true, false> : k_ensemble_step<32, false, false>;
  else if (E.N <= 64) kern = E.all_fac ? k_ensemble_step<64, true, false> : k_ensemble_step<64, false, false>;
  else if (E.N <= 96) kern = E.all_fac ? k_ensemble_step<96, true, false> : k_ensemble_step<96, false, false>;
  else {
    set_error("icon_ensemble_step: the persistent ensemble supports up to 96 levels");
    return ICON_EINVAL;
  }
  if (E.grid_blocks == 0) {
    int dev = 0, nsm = 0, per = 0, smem_sm = 0;
    ICON_CUDA(cudaGetDevice(&dev));
    ICON_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    ICON_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    // ask for no more shared memory than 8 resident blocks take (with the 1 KB the
    // system reserves per block): the rest of the SM's unified memory stays L1 cache for
    // the stencil phases
    cudaFuncAttributes fa;
    ICON_CUDA(cudaFuncGetAttributes(&fa, kern));
    const double need = 8.0 * ((double)fa.sharedSizeBytes + 1024.0);
    const int pct = smem_sm > 0 ? (int)std::ceil(100.0 * need / smem_sm) : 100;
    ICON_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct < 100 ? pct : 100));
    ICON_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 128, 0));
    if (per < 1) {
      set_error("icon_ensemble_step: the persistent kernel does not fit on an SM");
      return ICON_ECUDA;
    }
    E.grid_blocks = nsm * per;
  }
  k_ens_colconst<<<E.nm, 64, 0, st>>>(A.m, E.nm);
  for (const EnsembleDev::LeanConst& L : E.lean_consts) {
    k_mx_leanconst<<<1, 128, 0, st>>>(L.N, L.ld, L.wu, L.wl, L.dzh, L.dz, L.ray, L.ex_ref, L.dtau, L.cd, L.cf);
    k_mx_dwa_t<<<blocks_for(L.nc, 256), 256, 0, st>>>(L.nc, L.div_wa, L.inv_Ac, L.dtau, L.dwa, L.cw32);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(E.grid_blocks);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof_begin(st, K_ENSEMBLE);
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, A);
  prof_end(st);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the ensemble kernel");
  return ICON_OK;
}

}  // namespace icon
