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
//    ([entity][ld]) so that a warp gathers whole neighbour rows.
//  * rho, theta_v, Exner and w are FP64 prognostics stored level-major ([k][Nc]):
//    only the thread-per-column solve reads and writes them, and in this layout
//    its loads and stores are coalesced across the 32 columns of a warp. FP32
//    shadows ([Nc][ld]: rho, theta_v, Exner - Exner_ref(z), w) feed the stencils.
//  * FP64 is used where the method needs it: the hydrostatic-cancellation terms
//    (the explicit w predictor and a_k (pi_{k-1} - pi_k) in the right-hand side),
//    the tridiagonal system and its solution, the rho / Theta / Exner updates, the
//    horizontal mass-flux divergence (FP32 edge flux integrals l_e rho_e vn summed
//    in FP64, so that the two cells of an edge use the same value and the global
//    mass is conserved to rounding) and the accumulated mass fluxes. Coefficients
//    that only multiply small increments (the linearised state equation factor
//    (Rd/cvd) pi/Theta) are FP32.
//  * The predictor writes the provisional state S* only as FP32 shadows: S* is
//    consumed by FP32 stencils, while the corrector's column uses coefficients
//    frozen at S^n.
#include "icon_internal.h"

namespace icon {
namespace {

constexpr int kWarps = 8;
constexpr float kRcvF = (float)(kRd / kCvd);

struct MxGeo {
  int64_t nc, ne, nv;
  int N, ld;
  const int *c2e, *e2c, *e2v, *v2e, *v2c, *vdeg, *e2vt, *e2q;
  const float *div_w32, *rot_w32, *vt_w32, *kin_w32, *lsq_w32, *inv_de32, *inv_le32, *f_e32, *l_e32;
  const float *n_e32, *t_e32, *L34inv32, *s_ce32;
  const double* inv_Ac;                    // 1 / A_c (FP64)
  const double *dz, *dzh, *wu, *wl, *dz2, *ray, *ex_ref;
  const float *inv_dz32, *wu32, *wl32, *inv_dz2_32;
};

__device__ inline int64_t warp_entity() { return (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); }

__device__ inline float half32(const float* __restrict__ f, const float* __restrict__ wu,
                               const float* __restrict__ wl, int h, int N) {
  if (h == 0) return f[0];
  if (h == N) return f[N - 1];
  return wu[h] * f[h - 1] + wl[h] * f[h];
}

// zeta (full levels), w_v (half levels)
__global__ void __launch_bounds__(256) k_mx_vertex(MxGeo G, const float* __restrict__ vn, const float* __restrict__ w,
                                                   float* __restrict__ zeta, float* __restrict__ w_v) {
  const int64_t v = warp_entity();
  if (v >= G.nv) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[6], C[6];
  float rw[6];
  for (int j = 0; j < 6; ++j) {
    E[j] = (int64_t)G.v2e[6 * v + j] * ld;
    C[j] = (int64_t)G.v2c[6 * v + j] * ld;
    rw[j] = G.rot_w32[6 * v + j];
  }
  const int deg = G.vdeg[v];
  const float inv_deg = 1.0f / (float)deg;
  for (int k = lane; k < G.N; k += 32) {
    float acc = 0.f;
    for (int j = 0; j < 6; ++j) acc += rw[j] * vn[E[j] + k];
    zeta[v * ld + k] = acc;
  }
  for (int h = lane; h <= G.N; h += 32) {
    float acc = 0.f;
    for (int j = 0; j < 5; ++j) acc += w[C[j] + h];
    if (deg == 6) acc += w[C[5] + h];
    w_v[v * ld + h] = acc * inv_deg;
  }
}

// vt and K_e
__global__ void __launch_bounds__(256) k_mx_edge_diag(MxGeo G, const float* __restrict__ vn, float* __restrict__ vt,
                                                      float* __restrict__ Ke) {
  const int64_t e = warp_entity();
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t S[5];
  float W[5];
  for (int j = 0; j < 5; ++j) {
    S[j] = (int64_t)G.e2vt[5 * e + j] * ld;
    W[j] = G.vt_w32[5 * e + j];
  }
  for (int k = lane; k < G.N; k += 32) {
    float acc = 0.f;
    for (int j = 0; j < 5; ++j) acc += W[j] * vn[S[j] + k];
    const float v0 = vn[e * ld + k];
    vt[e * ld + k] = acc;
    Ke[e * ld + k] = 0.5f * (v0 * v0 + acc * acc);
  }
}

__global__ void __launch_bounds__(256) k_mx_cell_ke(MxGeo G, const float* __restrict__ Ke, float* __restrict__ Kc) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[3];
  float kw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    kw[s] = G.kin_w32[3 * c + s];
  }
  for (int k = lane; k < G.N; k += 32) Kc[c * ld + k] = kw[0] * Ke[E[0] + k] + kw[1] * Ke[E[1] + k] + kw[2] * Ke[E[2] + k];
}

struct MxEdgeArgs {
  const float *vn, *w, *rho, *thv, *exp;   // stage state (FP32 shadows; exp = Exner - Exner_ref)
  const float *vt, *Kc, *zeta, *w_v;
  const float* vn_base;
  float* vn_out;
  float* Avn0;
  float *phi, *gth, *a_e;                  // l_e rho_e vn, l_e rho_e vn theta_e, w-advection edge term
  double* mflx;
  float dtau;
  double inv_nsub;
  int corrector;
};

__global__ void __launch_bounds__(256) k_mx_edge_tend(MxGeo G, MxEdgeArgs a) {
  const int64_t e = warp_entity();
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld, N = G.N;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld;
  const int64_t v1 = (int64_t)G.e2v[2 * e] * ld, v2 = (int64_t)G.e2v[2 * e + 1] * ld;
  const float ide = G.inv_de32[e], ile = G.inv_le32[e], fe = G.f_e32[e], le = G.l_e32[e];
  const float* vn = a.vn + e * ld;
  const float* vt = a.vt + e * ld;
  const int64_t o = e * ld;
  for (int k = lane; k < N; k += 32) {
    const float vie0 = half32(vn, G.wu32, G.wl32, k, N);
    const float vie1 = half32(vn, G.wu32, G.wl32, k + 1, N);
    const float wbar = 0.25f * ((a.w[c1 + k] + a.w[c2 + k]) + (a.w[c1 + k + 1] + a.w[c2 + k + 1]));
    const float zeta_e = 0.5f * (a.zeta[v1 + k] + a.zeta[v2 + k]);
    const float A = -(a.Kc[c2 + k] - a.Kc[c1 + k]) * ide + (zeta_e + fe) * vt[k] - wbar * (vie0 - vie1) * G.inv_dz32[k];
    const float th_e = 0.5f * (a.thv[c1 + k] + a.thv[c2 + k]);
    const float pg = (float)kCpd * th_e * ((a.exp[c2 + k] - a.exp[c1 + k]) * ide);
    float vnew;
    if (a.corrector) {
      vnew = a.vn_base[o + k] + a.dtau * (0.5f * (a.Avn0[o + k] + A) - pg);
    } else {
      vnew = a.vn_base[o + k] + a.dtau * (A - pg);
      a.Avn0[o + k] = A;
    }
    a.vn_out[o + k] = vnew;
    const float F = 0.5f * (a.rho[c1 + k] + a.rho[c2 + k]) * vnew;
    const float phi = le * F;
    a.phi[o + k] = phi;
    a.gth[o + k] = phi * th_e;
    if (a.corrector) a.mflx[o + k] += (double)F * a.inv_nsub;
  }
  for (int h = lane; h <= N; h += 32) {
    const float vie = half32(vn, G.wu32, G.wl32, h, N);
    const float tie = half32(vt, G.wu32, G.wl32, h, N);
    a.a_e[o + h] = vie * (a.w[c2 + h] - a.w[c1 + h]) * ide + tie * (a.w_v[v2 + h] - a.w_v[v1 + h]) * ile;
  }
}

struct MxColArgs {
  // FP64 prognostics S^n, level-major [k][Nc]
  double *rho, *thv, *ex, *w;
  double* wflx;                            // level-major [h][Nc]
  // FP32 inputs
  const float *phi, *gth, *a_e;            // [Ne][ld]
  const float* w_stage;                    // [Nc][ld] w shadow of the stage state
  float* Aw0;                              // level-major [h][Nc]
  // FP32 shadows written by this stage, [Nc][ld]
  float *rho32, *thv32, *exp32, *w32;
  unsigned* status;
  double dtau, inv_nsub;
};

// one thread per column; CORR selects predictor (shadows of S* only) or corrector
// (FP64 S^{n+1} in place, shadows of S^{n+1}, accumulated vertical mass flux)
template <int NMAX, bool CORR>
__global__ void __launch_bounds__(128) k_mx_column(MxGeo G, MxColArgs a) {
  __shared__ double s_wu[NMAX + 1], s_wl[NMAX + 1], s_cA[NMAX + 1], s_cX[NMAX + 1], s_damp[NMAX + 1];
  __shared__ double s_dtbdz[NMAX], s_dt1bdz[NMAX], s_exref[NMAX];
  __shared__ float s_idz2[NMAX + 1];
  const int N = G.N;
  const double dtau = a.dtau;
  for (int i = threadIdx.x; i <= N; i += blockDim.x) {
    s_wu[i] = G.wu[i];
    s_wl[i] = G.wl[i];
    const double dzh = G.dzh[i];
    s_cA[i] = (i > 0 && i < N) ? dtau * kBeta * kCpd / dzh : 0.0;
    s_cX[i] = (i > 0 && i < N) ? (1.0 - kBeta) * kCpd / dzh : 0.0;
    s_damp[i] = 1.0 / (1.0 + dtau * G.ray[i]);
    s_idz2[i] = G.inv_dz2_32[i];
    if (i < N) {
      s_dtbdz[i] = dtau * kBeta / G.dz[i];
      s_dt1bdz[i] = dtau * (1.0 - kBeta) / G.dz[i];
      s_exref[i] = G.ex_ref[i];
    }
  }
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = G.nc;
  if (c >= nc) return;
  const int ld = G.ld;
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

  double rho_ic[NMAX + 1], M[NMAX + 1], Thx[NMAX], exx[NMAX], rhox[NMAX], cp[NMAX], dp[NMAX];
  float gam[NMAX];
  // half-level interpolants of S^n and explicit predictors at full levels
  double rho_m = LM(a.rho, 0), thv_m = LM(a.thv, 0);
  rho_ic[0] = rho_m;
  M[0] = rho_m * thv_m;
  for (int k = 0; k < N; ++k) {
    const double rho = (k == 0) ? rho_m : LM(a.rho, k);
    const double thv = (k == 0) ? thv_m : LM(a.thv, k);
    if (k > 0) {
      const double ri = s_wu[k] * rho_m + s_wl[k] * rho;
      rho_ic[k] = ri;
      M[k] = ri * (s_wu[k] * thv_m + s_wl[k] * thv);
    }
    rho_m = rho;
    thv_m = thv;
  }
  rho_ic[N] = rho_m;
  M[N] = rho_m * thv_m;
  for (int k = 0; k < N; ++k) {
    // horizontal divergences: rho with an FP64 sum of the FP32 edge flux integrals
    const float p0 = sg[0] * a.phi[E[0] + k], p1 = sg[1] * a.phi[E[1] + k], p2 = sg[2] * a.phi[E[2] + k];
    const double Dr = (((double)p0 + (double)p1) + (double)p2) * invA;
    const float Dt = (sg[0] * a.gth[E[0] + k] + sg[1] * a.gth[E[1] + k] + sg[2] * a.gth[E[2] + k]) * invA32;
    const double rho = LM(a.rho, k), thv = LM(a.thv, k), ex = LM(a.ex, k);
    const double w0 = LM(a.w, k), w1 = LM(a.w, k + 1);
    const double Th = rho * thv;
    rhox[k] = rho - dtau * Dr - s_dt1bdz[k] * (rho_ic[k] * w0 - rho_ic[k + 1] * w1);
    const double thx = Th - (double)(dtau32 * Dt) - s_dt1bdz[k] * (M[k] * w0 - M[k + 1] * w1);
    Thx[k] = thx;
    const float g = kRcvF * ((float)ex / (float)Th);
    exx[k] = ex + (double)g * (thx - Th);
    gam[k] = g * (float)s_dtbdz[k];
  }
  // tridiagonal system at interior half levels, Thomas forward sweep
  double thv_m1 = LM(a.thv, 0), ex_m1 = LM(a.ex, 0);
  for (int h = 1; h < N; ++h) {
    const float hadv = kw[0] * a.a_e[E[0] + h] + kw[1] * a.a_e[E[1] + h] + kw[2] * a.a_e[E[2] + h];
    const float ws = a.w_stage[o + h];
    float Aw = -hadv - ws * (a.w_stage[o + h - 1] - a.w_stage[o + h + 1]) * s_idz2[h];
    if (CORR) Aw = 0.5f * (LM(a.Aw0, h) + Aw);
    else LM(a.Aw0, h) = Aw;
    const double thv_h = LM(a.thv, h), ex_h = LM(a.ex, h);
    const double th_ic = s_wu[h] * thv_m1 + s_wl[h] * thv_h;
    const double wx = LM(a.w, h) + dtau * ((double)Aw - s_cX[h] * th_ic * (ex_m1 - ex_h) - kGrav);
    const double aa = s_cA[h] * th_ic;
    const double gm = (double)gam[h - 1], gk = (double)gam[h];
    const double lower = -aa * gm * M[h - 1];
    const double diag = 1.0 + aa * (gm + gk) * M[h];
    const double upper = -aa * gk * M[h + 1];
    const double rhs = wx - aa * (exx[h - 1] - exx[h]);
    const int i = h - 1;
    if (i == 0) {
      const double r = 1.0 / diag;
      cp[0] = upper * r;
      dp[0] = rhs * r;
    } else {
      const double r = 1.0 / (diag - lower * cp[i - 1]);
      cp[i] = upper * r;
      dp[i] = (rhs - lower * dp[i - 1]) * r;
    }
    thv_m1 = thv_h;
    ex_m1 = ex_h;
  }
  for (int i = N - 3; i >= 0; --i) dp[i] = dp[i] - cp[i] * dp[i + 1];
  // updates
  double wn_prev = 0.0;
  bool bad = false;
  for (int k = 0; k < N; ++k) {
    const int h1 = k + 1;
    const double wn1 = (h1 < N) ? dp[h1 - 1] * s_damp[h1] : 0.0;
    const double q = M[k] * wn_prev - M[k + 1] * wn1;
    const double r = rho_ic[k] * wn_prev - rho_ic[k + 1] * wn1;
    const double Th_n = Thx[k] - s_dtbdz[k] * q;
    const double ex_n = exx[k] - (double)gam[k] * q;
    const double rho_n = rhox[k] - s_dtbdz[k] * r;
    const float exp_n = (float)(ex_n - s_exref[k]);
    if (CORR) {
      const double thv_n = Th_n / rho_n;
      const double wold = LM(a.w, k);
      LM(a.wflx, k) += rho_ic[k] * (kBeta * wn_prev + (1.0 - kBeta) * wold) * a.inv_nsub;
      LM(a.rho, k) = rho_n;
      LM(a.thv, k) = thv_n;
      LM(a.ex, k) = ex_n;
      LM(a.w, k) = wn_prev;
      a.thv32[o + k] = (float)thv_n;
      bad |= !isfinite(thv_n) || !isfinite(ex_n) || !isfinite(wn_prev);
    } else {
      const float rho32 = (float)rho_n;
      a.thv32[o + k] = (float)Th_n / rho32;
      bad |= !isfinite(rho_n) || !isfinite(ex_n) || !isfinite(wn_prev);
    }
    a.rho32[o + k] = (float)rho_n;
    a.exp32[o + k] = exp_n;
    a.w32[o + k] = (float)wn_prev;
    wn_prev = wn1;
  }
  a.w32[o + N] = 0.0f;
  if (CORR) {
    LM(a.wflx, N) += rho_ic[N] * ((1.0 - kBeta) * LM(a.w, N)) * a.inv_nsub;
    LM(a.w, N) = 0.0;
  }
  if (bad) atomicOr(a.status, 1u);
#undef LM
}

// ---------------------------------------------------------------- diffusion (once per step)
__global__ void __launch_bounds__(256) k_mx_diff_vertex(MxGeo G, const float* __restrict__ vn, float* __restrict__ ux,
                                                        float* __restrict__ uy, float* __restrict__ uz,
                                                        float* __restrict__ zeta) {
  const int64_t v = warp_entity();
  if (v >= G.nv) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[6];
  for (int j = 0; j < 6; ++j) E[j] = (int64_t)G.v2e[6 * v + j] * ld;
  const float* lw = G.lsq_w32 + 18 * v;
  const float* rw = G.rot_w32 + 6 * v;
  float L[18], R[6];
  for (int j = 0; j < 18; ++j) L[j] = lw[j];
  for (int j = 0; j < 6; ++j) R[j] = rw[j];
  for (int k = lane; k < G.N; k += 32) {
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

__global__ void __launch_bounds__(256) k_mx_diff_div(MxGeo G, const float* __restrict__ vn, float* __restrict__ divc) {
  const int64_t c = warp_entity();
  if (c >= G.nc) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t E[3];
  float dw[3];
  for (int s = 0; s < 3; ++s) {
    E[s] = (int64_t)G.c2e[3 * c + s] * ld;
    dw[s] = G.div_w32[3 * c + s];
  }
  for (int k = lane; k < G.N; k += 32) divc[c * ld + k] = dw[0] * vn[E[0] + k] + dw[1] * vn[E[1] + k] + dw[2] * vn[E[2] + k];
}

__global__ void __launch_bounds__(256) k_mx_diff_edge(MxGeo G, float* __restrict__ vn, const float* __restrict__ ux,
                                                      const float* __restrict__ uy, const float* __restrict__ uz,
                                                      const float* __restrict__ zeta, const float* __restrict__ divc,
                                                      const float* __restrict__ thv, float* __restrict__ thflx,
                                                      float dt) {
  const int64_t e = warp_entity();
  if (e >= G.ne) return;
  const int lane = threadIdx.x & 31, ld = G.ld;
  int64_t Q[4];
  for (int j = 0; j < 4; ++j) Q[j] = (int64_t)G.e2q[4 * e + j] * ld;
  const int64_t c1 = (int64_t)G.e2c[2 * e] * ld, c2 = (int64_t)G.e2c[2 * e + 1] * ld;
  const int64_t v1 = (int64_t)G.e2v[2 * e] * ld, v2 = (int64_t)G.e2v[2 * e + 1] * ld;
  const float nx = G.n_e32[3 * e], ny = G.n_e32[3 * e + 1], nz = G.n_e32[3 * e + 2];
  const float tx = G.t_e32[3 * e], ty = G.t_e32[3 * e + 1], tz = G.t_e32[3 * e + 2];
  const float ide = G.inv_de32[e], ile = G.inv_le32[e], i34 = G.L34inv32[e], le = G.l_e32[e];
  const float cs2ld = (float)(kCsSmag * kCsSmag) * le / ide;
  for (int k = lane; k < G.N; k += 32) {
    const float ax = ux[Q[3] + k] - ux[Q[2] + k], ay = uy[Q[3] + k] - uy[Q[2] + k], az = uz[Q[3] + k] - uz[Q[2] + k];
    const float bx = ux[Q[1] + k] - ux[Q[0] + k], by = uy[Q[1] + k] - uy[Q[0] + k], bz = uz[Q[1] + k] - uz[Q[0] + k];
    const float DT = (ax * nx + ay * ny + az * nz) * i34 - (bx * tx + by * ty + bz * tz) * ile;
    const float DS = (ax * tx + ay * ty + az * tz) * i34 + (bx * nx + by * ny + bz * nz) * ile;
    const float Kh = cs2ld * sqrtf(DT * DT + DS * DS);
    const float lap = (divc[c2 + k] - divc[c1 + k]) * ide - (zeta[v2 + k] - zeta[v1 + k]) * ile;
    vn[e * ld + k] += dt * Kh * lap;
    thflx[e * ld + k] = le * Kh * (thv[c2 + k] - thv[c1 + k]) * ide;
  }
}

// one thread per column: theta_v += dt/A sum s l K_h dtheta/d (FP32 increment, FP64
// accumulation), Exner at constant density, shadows refreshed
__global__ void __launch_bounds__(128) k_mx_diff_theta(MxGeo G, const float* __restrict__ thflx, double* __restrict__ thv,
                                                       double* __restrict__ ex, float* __restrict__ thv32,
                                                       float* __restrict__ exp32, float dt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = G.nc;
  if (c >= nc) return;
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
    const double th_n = th + (double)dth;
    const double ex_n = ex[i] + ex[i] * (double)(kRcvF * dth / (float)th);
    thv[i] = th_n;
    ex[i] = ex_n;
    thv32[c * ld + k] = (float)th_n;
    exp32[c * ld + k] = (float)(ex_n - G.ex_ref[k]);
  }
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
  G.dz = v.d_dz; G.dzh = v.d_dzh; G.wu = v.d_wu; G.wl = v.d_wl; G.dz2 = v.d_dz2; G.ray = v.d_ray;
  G.ex_ref = s.ex_ref;
  G.inv_dz32 = v.d_inv_dz32; G.wu32 = v.d_wu32; G.wl32 = v.d_wl32; G.inv_dz2_32 = v.d_inv_dz2_32;
  return G;
}

template <bool CORR>
void launch_mx_column(const MxGeo& G, const MxColArgs& a, cudaStream_t st) {
  const unsigned nb = blocks_for(G.nc, 128);
  if (G.N <= 32) k_mx_column<32, CORR><<<nb, 128, 0, st>>>(G, a);
  else if (G.N <= 64) k_mx_column<64, CORR><<<nb, 128, 0, st>>>(G, a);
  else if (G.N <= 96) k_mx_column<96, CORR><<<nb, 128, 0, st>>>(G, a);
  else if (G.N <= 128) k_mx_column<128, CORR><<<nb, 128, 0, st>>>(G, a);
  else k_mx_column<256, CORR><<<nb, 128, 0, st>>>(G, a);
}

}  // namespace

void enqueue_step_mixed(icon_state* st, double dt, int nsub, cudaStream_t stream) {
  const icon_grid* grid = st->grid;
  StateDev& s = st->s;
  const MxGeo G = make_mx_geo(grid, s);
  const int64_t nc = G.nc;
  const double dtau = dt / nsub;
  const unsigned nbv = blocks_for(G.nv, kWarps), nbe = blocks_for(G.ne, kWarps), nbc = blocks_for(G.nc, kWarps);
  cudaMemsetAsync(s.mflx, 0, sizeof(double) * G.ne * G.ld, stream);
  cudaMemsetAsync(s.wflx, 0, sizeof(double) * nc * (G.N + 1), stream);
  for (int it = 0; it < nsub; ++it) {
    for (int stage = 0; stage < 2; ++stage) {
      const bool corr = stage == 1;
      const float* vn = corr ? s.vn32_s : s.vn32;
      const float* w = corr ? s.w32_s : s.w32;
      prof_begin(stream, K_MX_VERTEX);
      k_mx_vertex<<<nbv, 256, 0, stream>>>(G, vn, w, s.zeta32, s.wv32);
      prof_end(stream);
      prof_begin(stream, K_MX_EDGE);
      k_mx_edge_diag<<<nbe, 256, 0, stream>>>(G, vn, s.vt32, s.Ke32);
      prof_end(stream);
      prof_begin(stream, K_MX_CELL_KE);
      k_mx_cell_ke<<<nbc, 256, 0, stream>>>(G, s.Ke32, s.Kc32);
      prof_end(stream);
      MxEdgeArgs ea;
      ea.vn = vn; ea.w = w;
      ea.rho = corr ? s.rho32_s : s.rho32;
      ea.thv = corr ? s.thv32_s : s.thv32;
      ea.exp = corr ? s.exp32_s : s.exp32;
      ea.vt = s.vt32; ea.Kc = s.Kc32; ea.zeta = s.zeta32; ea.w_v = s.wv32;
      ea.vn_base = s.vn32;
      ea.vn_out = corr ? s.vn32 : s.vn32_s;
      ea.Avn0 = s.Avn0_32;
      ea.phi = s.F32; ea.gth = s.G32; ea.a_e = s.ae32; ea.mflx = s.mflx;
      ea.dtau = (float)dtau; ea.inv_nsub = 1.0 / nsub; ea.corrector = corr;
      prof_begin(stream, K_MX_EDGE_TEND);
      k_mx_edge_tend<<<nbe, 256, 0, stream>>>(G, ea);
      prof_end(stream);
      MxColArgs ca;
      ca.rho = s.rho; ca.thv = s.thv; ca.ex = s.ex; ca.w = s.w; ca.wflx = s.wflx;
      ca.phi = s.F32; ca.gth = s.G32; ca.a_e = s.ae32;
      ca.w_stage = w;
      ca.Aw0 = s.Aw0_32;
      ca.rho32 = corr ? s.rho32 : s.rho32_s;
      ca.thv32 = corr ? s.thv32 : s.thv32_s;
      ca.exp32 = corr ? s.exp32 : s.exp32_s;
      ca.w32 = corr ? s.w32 : s.w32_s;
      ca.status = s.status;
      ca.dtau = dtau; ca.inv_nsub = 1.0 / nsub;
      prof_begin(stream, K_MX_COLUMN);
      if (corr) launch_mx_column<true>(G, ca, stream);
      else launch_mx_column<false>(G, ca, stream);
      prof_end(stream);
    }
  }
  prof_begin(stream, K_MX_DIFF_VERTEX);
  k_mx_diff_vertex<<<nbv, 256, 0, stream>>>(G, s.vn32, s.uvx32, s.uvy32, s.uvz32, s.zeta32);
  k_mx_diff_div<<<nbc, 256, 0, stream>>>(G, s.vn32, s.Kc32);
  prof_end(stream);
  prof_begin(stream, K_MX_DIFF_EDGE);
  k_mx_diff_edge<<<nbe, 256, 0, stream>>>(G, s.vn32, s.uvx32, s.uvy32, s.uvz32, s.zeta32, s.Kc32, s.thv32, s.Ke32,
                                           (float)dt);
  prof_end(stream);
  prof_begin(stream, K_MX_DIFF_THETA);
  k_mx_diff_theta<<<blocks_for(nc, 128), 128, 0, stream>>>(G, s.Ke32, s.thv, s.ex, s.thv32, s.exp32, (float)dt);
  prof_end(stream);
}

}  // namespace icon
