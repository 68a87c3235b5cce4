// Terrain-following height coordinate over topography (FP64 form).
//
// The paper's atmosphere computes on a terrain-following hybrid height coordinate
// (Sec. "Current State of the Art") and prints none of its formulas. The levels
// here are of SLEVE type with one decay scale s_d = 4000 m: half level h of a
// column standing on surface height hs lies at
//   z_h = zeta_h + hs b_h,   b_h = sinh((z_top - zeta_h)/s_d) / sinh(z_top/s_d),
// zeta_h the flat levels, so the lowest level is the ground and the lid is flat;
// full levels lie midway (zf = zeta_f + hs bf, bf the mean of the two b). An edge
// is a column at the mean of its two cells' hs, a vertex one at the mean of its
// cells'. The topography is a Gaussian mountain hs = h0 exp(-(r/a)^2), r the
// great-circle distance to 90E 30N.
//
// Everything metric is separable (an entity scalar times a level profile): the
// slope of a coordinate surface at an edge is b_h (hs_c2 - hs_c1)/d_e normal to it
// and b_h (hs_v2 - hs_v1)/l_e along it. What the FP64-bound step kernels would
// otherwise divide for at every cell- or edge-level (1/dz, 1/dzh, the half-level
// interpolation weights, the reference Exner exp(-g zf/(cpd 250 K))) is tabulated
// once here in [entity][ld] rows: the kernels have spare memory bandwidth but no
// spare FP64 issue slots.
//
// Per stage, k_topo_cell forms at every cell (one warp, lanes over levels)
//   X_c,k = bf_k sum_e (kappa_ce sn_e vn_e,k + kappa_ce st_e vt_e,k)   (full levels)
//   wcc_c,h = the half-level interpolant of X with the cell's weights (contravariant
//            correction, in ICON's order); at the ground sum_e kappa_ce (sn_e vn + st_e vt)
//            with the lowest full level's wind,
//   w - wcc at interior half levels (0 at the lid and the ground),
//   pi' = pi - pi_ref and half of d pi'/dz at full levels (the half-level interpolants
//            differenced over dz, one-sided at the top and bottom full levels),
// which the edge tendency (vertical advection of vn, metric pressure gradient) and
// the column solve (contravariant vertical fluxes, advection of w) consume, so that
// those FP64-bound kernels load these terms instead of forming them per edge.
#include <cmath>
#include "icon_internal.h"

namespace icon {
namespace {

constexpr int kWarps = 8;

// The tables are formed with explicitly rounded products (__dmul_rn is never fused into
// a multiply-add), the same arithmetic as a plain evaluation of the formulas.
#define MUL __dmul_rn

// surface height of every cell: the Gaussian mountain
__global__ void k_topo_hs(int64_t nc, const double* __restrict__ x_c, double h0, double radius, double cx, double cy,
                          double cz, double* __restrict__ hs) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double x = x_c[3 * c], y = x_c[3 * c + 1], z = x_c[3 * c + 2];
  const double px = MUL(y, cz) - MUL(z, cy), py = MUL(z, cx) - MUL(x, cz), pz = MUL(x, cy) - MUL(y, cx);
  const double r = kR * atan2(sqrt((MUL(px, px) + MUL(py, py)) + MUL(pz, pz)), (MUL(x, cx) + MUL(y, cy)) + MUL(z, cz));
  const double q = r / radius;
  hs[c] = h0 * exp(-(q * q));
}

struct LevelArgs {
  int N, ld;
  const double *dz, *dzh, *z_f, *b, *bf;      // flat profiles and the decay, [ld]
};

// one thread per (cell, level slot): the cell tables
__global__ void k_topo_cells(LevelArgs L, int64_t nc, const double* __restrict__ hs, double* __restrict__ inv_dz,
                             double* __restrict__ inv_dzh, double* __restrict__ wu, double* __restrict__ exref,
                             double* __restrict__ dzc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nc * L.ld) return;
  const int64_t c = t / L.ld;
  const int k = (int)(t % L.ld);
  const double h = hs[c];
  double idz = 0.0, idzh = 0.0, w = 0.0, er = 0.0, d = 0.0;
  if (k < L.N) {
    d = L.dz[k] + MUL(h, L.b[k] - L.b[k + 1]);
    idz = 1.0 / d;
    const double zf = L.z_f[k] + MUL(h, L.bf[k]);
    er = exp(-kGrav * zf / (kCpd * kTopoTref));
  }
  if (k >= 1 && k < L.N) {
    idzh = 1.0 / (L.dzh[k] + MUL(h, L.bf[k - 1] - L.bf[k]));
    const double dm = L.dz[k - 1] + MUL(h, L.b[k - 1] - L.b[k]);
    w = d / (dm + d);
  }
  inv_dz[t] = idz;
  inv_dzh[t] = idzh;
  wu[t] = w;
  exref[t] = er;
  dzc[t] = d;
}

// mean surface height of the cells around vertex v (the O5 vertex mean)
__device__ inline double vertex_hs(int64_t v, const int* __restrict__ v2c, const int* __restrict__ vdeg,
                                   const double* __restrict__ hs) {
  double acc = 0.0;
  for (int j = 0; j < 5; ++j) acc += hs[v2c[6 * v + j]];
  const int deg = vdeg[v];
  acc += deg == 6 ? hs[v2c[6 * v + 5]] : 0.0;
  return acc / (double)deg;
}

// one thread per (edge, level slot): the edge tables and, at slot 0, the two slopes
__global__ void k_topo_edges(LevelArgs L, int64_t ne, const int* __restrict__ e2c, const int* __restrict__ e2v,
                             const int* __restrict__ v2c, const int* __restrict__ vdeg,
                             const double* __restrict__ d_e, const double* __restrict__ l_e,
                             const double* __restrict__ hs, double* __restrict__ wu, double* __restrict__ qinv_dz,
                             double* __restrict__ dze, double* __restrict__ sn, double* __restrict__ st) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne * L.ld) return;
  const int64_t e = t / L.ld;
  const int k = (int)(t % L.ld);
  const double h1 = hs[e2c[2 * e]], h2 = hs[e2c[2 * e + 1]];
  const double h = 0.5 * (h1 + h2);
  double qidz = 0.0, w = 0.0, d = 0.0;
  if (k < L.N) {
    d = L.dz[k] + MUL(h, L.b[k] - L.b[k + 1]);
    qidz = 0.25 / d;
  }
  if (k >= 1 && k < L.N) {
    const double dm = L.dz[k - 1] + MUL(h, L.b[k - 1] - L.b[k]);
    w = d / (dm + d);
  }
  wu[t] = w;
  qinv_dz[t] = qidz;
  dze[t] = d;
  if (k == 0) {
    sn[e] = (h2 - h1) / d_e[e];
    const double hv1 = vertex_hs(e2v[2 * e], v2c, vdeg, hs), hv2 = vertex_hs(e2v[2 * e + 1], v2c, vdeg, hs);
    st[e] = (hv2 - hv1) / l_e[e];
  }
}

struct StageArgs {
  int64_t nc;
  int N, ld;
  const int* c2e;
  const double* kin_w;
  const double *vn, *vt, *w, *ex;             // stage state and its tangential velocity
  const double *bf, *sn, *st;
  const double *wu_c, *inv_dz_c, *inv_dzh_c, *exref_c;
  double *wcc, *wcon, *ep, *hdpdz;
};

// one warp per cell, lanes over levels: the stage's contravariant correction and
// contravariant velocity at half levels, the Exner perturbation and half its vertical
// derivative at full levels. FP64-pipe bound like the step's stencils: the kappa and
// slope factors of the three edges are combined once per cell (6 fused multiply-adds
// per full level), and the half-level interpolant takes the level above from the
// neighbouring lane. Windows of 31 levels: lane l holds full level k = base + l and the
// half level above it; lane 30's full level is carried to the next window.
__global__ void __launch_bounds__(256, 4) k_topo_cell(StageArgs a) {
  const int64_t c = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (c >= a.nc) return;
  const int lane = threadIdx.x & 31, ld = a.ld, N = a.N;
  const int64_t o = c * ld;
  int64_t E[3];
  double An[3], At[3];
  for (int s = 0; s < 3; ++s) {
    const int e = a.c2e[3 * c + s];
    E[s] = (int64_t)e * ld;
    const double kw = a.kin_w[3 * c + s];
    An[s] = kw * a.sn[e];
    At[s] = kw * a.st[e];
  }
  double carry = 0.0;                       // X of the full level above the window
  for (int base = 0; base <= N; base += 31) {
    const int k = base + lane;
    const bool own = lane < 31 && k <= N;   // half level k (and full level k if k < N)
    double Y = 0.0;
    if (lane < 31 && k < N) {
      for (int s = 0; s < 3; ++s) {
        Y = fma(An[s], a.vn[E[s] + k], Y);
        Y = fma(At[s], a.vt[E[s] + k], Y);
      }
    }
    const double X = (lane < 31 && k < N) ? Y * a.bf[k] : 0.0;
    double Xm = __shfl_up_sync(0xffffffffu, X, 1);
    if (lane == 0) Xm = carry;
    carry = __shfl_sync(0xffffffffu, X, 30);
    if (own) {
      if (k > 0 && k < N) {
        const double wcc = fma(a.wu_c[o + k], Xm - X, X);
        a.wcc[o + k] = wcc;
        a.wcon[o + k] = a.w[o + k] - wcc;
      } else {
        if (k == 0) a.wcc[o] = 0.0;
        a.wcon[o + k] = 0.0;
      }
      if (k == N - 1) a.wcc[o + N] = Y;     // ground: surface slopes, lowest full level's wind
    }
  }
  for (int k = lane; k < N; k += 32) {
    const double* ex = a.ex + o;
    const double* er = a.exref_c + o;
    const double p0 = ex[k] - er[k];
    double d;
    if (k == 0) {
      d = (p0 - (ex[1] - er[1])) * a.inv_dzh_c[o + 1];
    } else if (k == N - 1) {
      d = ((ex[N - 2] - er[N - 2]) - p0) * a.inv_dzh_c[o + N - 1];
    } else {
      const double pm = ex[k - 1] - er[k - 1], pp = ex[k + 1] - er[k + 1];
      const double fa = fma(a.wu_c[o + k], pm - p0, p0);
      const double fb = fma(a.wu_c[o + k + 1], p0 - pp, pp);
      d = (fa - fb) * a.inv_dz_c[o + k];
    }
    a.ep[o + k] = p0;
    a.hdpdz[o + k] = 0.5 * d;
  }
}

// FP32 copy of an FP64 table
__global__ void k_topo_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n, double scale) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)(scale * a[i]);
}

// FP32 1/dz at edges from the FP64 thickness
__global__ void k_topo_inv32(const double* __restrict__ dz, float* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = dz[i] != 0.0 ? (float)(1.0 / dz[i]) : 0.0f;
}

// [c][ld] -> level-major [k][nc], rows 0..rows-1
__global__ void k_topo_lm(const double* __restrict__ src, double* __restrict__ dst, int64_t nc, int rows, int ld) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nc * rows) return;
  const int64_t k = t / nc, c = t % nc;
  dst[t] = src[c * ld + k];
}

struct StageArgs32 {
  int64_t nc;
  int N, ld;
  const int* c2e;
  const float* kin_w;
  const double *sn, *st;
  const float *vn, *vt, *w, *exp;             // FP32 stage shadows (exp against the per-cell reference)
  const float *bf, *wu_c, *inv_dz_c, *inv_dzh_c;
  float *wcc, *wcon, *hdpdz;
};

// the mixed-precision form of k_topo_cell: the same terms in FP32 (the precision of the
// stencils that consume them), the Exner perturbation being the state's FP32 shadow
__global__ void __launch_bounds__(256) k_topo_cell32(StageArgs32 a) {
  const int64_t c = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (c >= a.nc) return;
  const int lane = threadIdx.x & 31, ld = a.ld, N = a.N;
  const int64_t o = c * ld;
  int64_t E[3];
  float An[3], At[3];
  for (int s = 0; s < 3; ++s) {
    const int e = a.c2e[3 * c + s];
    E[s] = (int64_t)e * ld;
    const float kw = a.kin_w[3 * c + s];
    An[s] = kw * (float)a.sn[e];
    At[s] = kw * (float)a.st[e];
  }
  float carry = 0.0f;
  for (int base = 0; base <= N; base += 31) {
    const int k = base + lane;
    const bool own = lane < 31 && k <= N;
    float Y = 0.0f;
    if (lane < 31 && k < N) {
      for (int s = 0; s < 3; ++s) {
        Y = fmaf(An[s], a.vn[E[s] + k], Y);
        Y = fmaf(At[s], a.vt[E[s] + k], Y);
      }
    }
    const float X = (lane < 31 && k < N) ? Y * a.bf[k] : 0.0f;
    float Xm = __shfl_up_sync(0xffffffffu, X, 1);
    if (lane == 0) Xm = carry;
    carry = __shfl_sync(0xffffffffu, X, 30);
    if (own) {
      if (k > 0 && k < N) {
        const float wcc = fmaf(a.wu_c[o + k], Xm - X, X);
        a.wcc[o + k] = wcc;
        a.wcon[o + k] = a.w[o + k] - wcc;
      } else {
        if (k == 0) a.wcc[o] = 0.0f;
        a.wcon[o + k] = 0.0f;
      }
      if (k == N - 1) a.wcc[o + N] = Y;
    }
  }
  for (int k = lane; k < N; k += 32) {
    const float* ep = a.exp + o;
    const float p0 = ep[k];
    float d;
    if (k == 0) {
      d = (p0 - ep[1]) * a.inv_dzh_c[o + 1];
    } else if (k == N - 1) {
      d = (ep[N - 2] - p0) * a.inv_dzh_c[o + N - 1];
    } else {
      const float fa = fmaf(a.wu_c[o + k], ep[k - 1] - p0, p0);
      const float fb = fmaf(a.wu_c[o + k + 1], p0 - ep[k + 1], ep[k + 1]);
      d = (fa - fb) * a.inv_dz_c[o + k];
    }
    a.hdpdz[o + k] = 0.5f * d;
  }
}

}  // namespace

int topo_build(icon_state* st, double h0, double radius, cudaStream_t stream) {
  const icon_grid* grid = st->grid;
  const GridDev& g = grid->g;
  const Vertical& v = grid->vert;
  TopoDev& T = st->s.topo;
  DeviceArena& A = st->arena;
  const size_t C = (size_t)(g.nc * v.ld), E = (size_t)(g.ne * v.ld);
  T.h0 = h0;
  T.radius = radius;
  T.hs = A.get_n<double>(g.nc);
  T.b = A.get_n<double>(v.ld);
  T.bf = A.get_n<double>(v.ld);
  T.sn = A.get_n<double>(g.ne);
  T.st = A.get_n<double>(g.ne);
  double** cells[] = {&T.inv_dz_c, &T.inv_dzh_c, &T.wu_c, &T.exref_c, &T.dz_c, &T.wcc, &T.wcon, &T.ep, &T.hdpdz};
  for (double** p : cells) *p = A.get_n<double>(C);
  double** edges[] = {&T.wu_e, &T.qinv_dz_e, &T.dz_e};
  for (double** p : edges) *p = A.get_n<double>(E);
  if (A.failed) {
    set_error("out of device memory for the terrain-following metric tables");
    return ICON_ENOMEM;
  }
  // decay profile on the host (per level, once)
  std::vector<double> b(v.ld, 0.0), bf(v.ld, 0.0);
  const double den = std::sinh(v.z_top / kTopoDecay);
  for (int h = 0; h <= v.N; ++h) b[h] = std::sinh((v.z_top - v.z_h[h]) / kTopoDecay) / den;
  for (int k = 0; k < v.N; ++k) bf[k] = 0.5 * (b[k] + b[k + 1]);
  ICON_CUDA(cudaMemcpyAsync(T.b, b.data(), sizeof(double) * v.ld, cudaMemcpyHostToDevice, stream));
  ICON_CUDA(cudaMemcpyAsync(T.bf, bf.data(), sizeof(double) * v.ld, cudaMemcpyHostToDevice, stream));
  const double pi = 3.141592653589793, lon = 90.0 * pi / 180.0, lat = 30.0 * pi / 180.0;
  k_topo_hs<<<blocks_for(g.nc, 256), 256, 0, stream>>>(g.nc, g.x_c, h0, radius, std::cos(lat) * std::cos(lon),
                                                       std::cos(lat) * std::sin(lon), std::sin(lat), T.hs);
  LevelArgs L;
  L.N = v.N; L.ld = v.ld; L.dz = v.d_dz; L.dzh = v.d_dzh; L.z_f = v.d_z_f; L.b = T.b; L.bf = T.bf;
  k_topo_cells<<<blocks_for(g.nc * v.ld, 256), 256, 0, stream>>>(L, g.nc, T.hs, T.inv_dz_c, T.inv_dzh_c, T.wu_c,
                                                                 T.exref_c, T.dz_c);
  k_topo_edges<<<blocks_for(g.ne * v.ld, 256), 256, 0, stream>>>(L, g.ne, g.e2c, g.e2v, g.v2c, g.vdeg, g.d_e, g.l_e,
                                                                 T.hs, T.wu_e, T.qinv_dz_e, T.dz_e, T.sn, T.st);
  ICON_CUDA(cudaGetLastError());
  for (double* p : {T.wcc, T.wcon, T.ep, T.hdpdz}) ICON_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * C, stream));
  if (st->s.precision == ICON_MIXED) {
    float** e32[] = {&T.wu_e32, &T.inv_dz_e32, &T.dz_e32};
    for (float** p : e32) *p = A.get_n<float>(E);
    float** c32[] = {&T.wu_c32, &T.inv_dz_c32, &T.inv_dzh_c32, &T.wcc32, &T.wcon32, &T.hdpdz32};
    for (float** p : c32) *p = A.get_n<float>(C);
    T.csn32 = A.get_n<float>(g.ne);
    T.bf32 = A.get_n<float>(v.ld);
    const size_t LMN = (size_t)g.nc * (v.N + 1);
    double** lm[] = {&T.wu_lm, &T.idz_lm, &T.idzh_lm, &T.exref_lm};
    for (double** p : lm) *p = A.get_n<double>(LMN);
    if (A.failed) {
      set_error("out of device memory for the terrain-following metric tables");
      return ICON_ENOMEM;
    }
    const unsigned bE = blocks_for((int64_t)E, 256), bC = blocks_for((int64_t)C, 256);
    k_topo_f32<<<bE, 256, 0, stream>>>(T.wu_e, T.wu_e32, (int64_t)E, 1.0);
    k_topo_inv32<<<bE, 256, 0, stream>>>(T.dz_e, T.inv_dz_e32, (int64_t)E);
    k_topo_f32<<<bE, 256, 0, stream>>>(T.dz_e, T.dz_e32, (int64_t)E, 1.0);
    k_topo_f32<<<bC, 256, 0, stream>>>(T.wu_c, T.wu_c32, (int64_t)C, 1.0);
    k_topo_f32<<<bC, 256, 0, stream>>>(T.inv_dz_c, T.inv_dz_c32, (int64_t)C, 1.0);
    k_topo_f32<<<bC, 256, 0, stream>>>(T.inv_dzh_c, T.inv_dzh_c32, (int64_t)C, 1.0);
    k_topo_f32<<<blocks_for(g.ne, 256), 256, 0, stream>>>(T.sn, T.csn32, g.ne, kCpd);
    k_topo_f32<<<1, 256, 0, stream>>>(T.bf, T.bf32, v.ld, 1.0);
    const unsigned bL = blocks_for((int64_t)LMN, 256);
    k_topo_lm<<<bL, 256, 0, stream>>>(T.wu_c, T.wu_lm, g.nc, v.N + 1, v.ld);
    k_topo_lm<<<bL, 256, 0, stream>>>(T.inv_dz_c, T.idz_lm, g.nc, v.N + 1, v.ld);
    k_topo_lm<<<bL, 256, 0, stream>>>(T.inv_dzh_c, T.idzh_lm, g.nc, v.N + 1, v.ld);
    k_topo_lm<<<bL, 256, 0, stream>>>(T.exref_c, T.exref_lm, g.nc, v.N + 1, v.ld);
    ICON_CUDA(cudaGetLastError());
    for (float* p : {T.wcc32, T.wcon32, T.hdpdz32}) ICON_CUDA(cudaMemsetAsync(p, 0, sizeof(float) * C, stream));
  }
  T.on = true;
  return ICON_OK;
}

void topo_stage(icon_state* st, const double* vn, const double* vt, const double* w, const double* ex,
                cudaStream_t stream) {
  const icon_grid* grid = st->grid;
  const GridDev& g = grid->g;
  const Vertical& v = grid->vert;
  const TopoDev& T = st->s.topo;
  StageArgs a;
  a.nc = g.nc; a.N = v.N; a.ld = v.ld;
  a.c2e = g.c2e; a.kin_w = g.kin_w;
  a.vn = vn; a.vt = vt; a.w = w; a.ex = ex;
  a.bf = T.bf; a.sn = T.sn; a.st = T.st;
  a.wu_c = T.wu_c; a.inv_dz_c = T.inv_dz_c; a.inv_dzh_c = T.inv_dzh_c; a.exref_c = T.exref_c;
  a.wcc = T.wcc; a.wcon = T.wcon; a.ep = T.ep; a.hdpdz = T.hdpdz;
  prof_begin(stream, K_TERRAIN);
  k_topo_cell<<<blocks_for(g.nc, kWarps), 256, 0, stream>>>(a);
  prof_end(stream);
}

void topo_stage32(icon_state* st, const float* vn, const float* vt, const float* w, const float* exp,
                  cudaStream_t stream) {
  const icon_grid* grid = st->grid;
  const GridDev& g = grid->g;
  const Vertical& v = grid->vert;
  const TopoDev& T = st->s.topo;
  StageArgs32 a;
  a.nc = g.nc; a.N = v.N; a.ld = v.ld;
  a.c2e = g.c2e; a.kin_w = g.kin_w32;
  a.sn = T.sn; a.st = T.st;
  a.vn = vn; a.vt = vt; a.w = w; a.exp = exp;
  a.bf = T.bf32; a.wu_c = T.wu_c32; a.inv_dz_c = T.inv_dz_c32; a.inv_dzh_c = T.inv_dzh_c32;
  a.wcc = T.wcc32; a.wcon = T.wcon32; a.hdpdz = T.hdpdz32;
  prof_begin(stream, K_TERRAIN);
  k_topo_cell32<<<blocks_for(g.nc, kWarps), 256, 0, stream>>>(a);
  prof_end(stream);
}

}  // namespace icon
