// Vertical grid and analytic initial states on the GPU.
//
// Vertical coordinate: flat bottom, rigid lid z_top; half level i = 0..N (top to
// bottom) at z_top (exp(s (N-i)/N) - 1)/(exp(s) - 1) -- a stretched height grid
// standing in for the paper's terrain-following hybrid height coordinate over
// flat ground (Sec. "Current State of the Art"; 90 levels in Table 2).
//
// Initial states (the paper starts from reanalysis data, which is replaced here
// by analytic states with the same sizes):
//   rest   isothermal 250 K, no wind;
//   SBR    u = u0 cos(phi), u0 = 20 m/s, 250 K, in gradient balance:
//          ln p = ln p0 - g z/(Rd T0) - (R Omega u0 + u0^2/2) sin^2(phi)/(Rd T0);
//   jet    ln p = ln p0 - z/H0 - B S(z) Phi(phi), H0 = Rd T_j/g, T_j = 288 K,
//          S = exp(-((z - 10 km)/10 km)^2), Phi = 4/15 - 4(cos^3/3 - cos^5/5)
//          (Phi centred and the 10 km half-width keep the state statically stable:
//          N^2 >= 1.4e-4 1/s^2 everywhere),
//          T = g/(Rd (1/H0 + B S' Phi)), u the gradient-wind root continuous with
//          geostrophy, B such that u = 35 m/s at 45 deg at z = 10 km, plus a
//          Gaussian zonal bump amp exp(-(r/(R/10))^2) (1 m/s at 20E 40N, or a
//          seeded amplitude in U(0.5, 2) m/s and a position uniform on the sphere
//          for an ensemble member).
// theta_v comes from the analytic T and p; Exner is analytic at the lowest level
// and integrated upward in discrete hydrostatic balance
// pi_{k-1} = pi_k - g dzh_k / (cpd theta_ic,k); rho from the state equation.
// Seeded noise theta_v += a (2U - 1), U the SplitMix64 draw number (cell*N + k),
// with Exner held fixed and rho recomputed.
#include <cmath>
#include "icon_internal.h"

namespace icon {

// SplitMix64 (Steele, Lea, Flood 2014): output number idx of the generator started at seed
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline double uniform01(uint64_t seed, uint64_t idx) {
  return (double)(splitmix64(seed, idx) >> 11) * (1.0 / 9007199254740992.0);
}

void make_vertical(Vertical& v, int nlev, double top_m, double stretch_s, double damp_m) {
  const int N = nlev;
  if (top_m <= 0) top_m = N >= 60 ? 75000.0 : 30000.0;
  if (stretch_s <= 0) stretch_s = N >= 60 ? 5.5 : 2.0;
  if (damp_m <= 0) damp_m = N >= 60 ? 45000.0 : 20000.0;
  v.N = N;
  v.ld = ((N + 1 + 31) / 32) * 32;
  v.z_top = top_m; v.s = stretch_s; v.z_d = damp_m;
  v.z_h.assign(v.ld, 0.0); v.z_f.assign(v.ld, 0.0); v.dz.assign(v.ld, 0.0); v.dzh.assign(v.ld, 0.0);
  v.wu.assign(v.ld, 0.0); v.wl.assign(v.ld, 0.0); v.rayleigh.assign(v.ld, 0.0); v.dz2.assign(v.ld, 0.0);
  const double den = std::exp(stretch_s) - 1.0;
  for (int i = 0; i <= N; ++i) v.z_h[i] = top_m * (std::exp(stretch_s * (N - i) / N) - 1.0) / den;
  v.z_h[N] = 0.0;
  v.z_h[0] = top_m;
  for (int k = 0; k < N; ++k) {
    v.dz[k] = v.z_h[k] - v.z_h[k + 1];
    v.z_f[k] = 0.5 * (v.z_h[k] + v.z_h[k + 1]);
  }
  for (int h = 1; h < N; ++h) {
    v.dzh[h] = v.z_f[h - 1] - v.z_f[h];
    v.wu[h] = v.dz[h] / (v.dz[h - 1] + v.dz[h]);
    v.wl[h] = 1.0 - v.wu[h];
    v.dz2[h] = v.z_h[h - 1] - v.z_h[h + 1];
  }
  const double pi = 3.141592653589793;
  for (int h = 0; h <= N; ++h) {
    double z = v.z_h[h];
    if (z > damp_m) {
      double sn = std::sin(0.5 * pi * (z - damp_m) / (top_m - damp_m));
      v.rayleigh[h] = 0.05 * (sn * sn);
    }
  }
}

namespace {

struct CaseDev {
  int case_id, N, ld;
  double noise, B, H0;
  uint64_t seed;
  int has_bump;
  double bamp, bx, by, bz;   // bump amplitude and unit centre
};

__device__ inline void basis(double x, double y, double z, double& cphi, double& sphi, double& elx, double& ely) {
  cphi = sqrt(x * x + y * y);
  sphi = z;
  double safe = cphi > 0.0 ? cphi : 1.0;
  elx = -y / safe;
  ely = x / safe;
}

// ln p, T, zonal wind of the analytic state at unit position (x, y, z) and height zz
__device__ void analytic(const CaseDev& cd, double x, double y, double zu, double zz, double& lnp, double& T,
                         double& u) {
  double cphi, sphi, elx, ely;
  basis(x, y, zu, cphi, sphi, elx, ely);
  if (cd.case_id == ICON_CASE_REST) {
    lnp = (log(kP0) - kGrav * zz / (kRd * 250.0)) + 0.0 * x;
    T = 250.0;
    u = 0.0;
  } else if (cd.case_id == ICON_CASE_SBR) {
    const double u0 = 20.0, T0 = 250.0;
    lnp = (log(kP0) - kGrav * zz / (kRd * T0)) - ((kR * kOmega * u0 + 0.5 * u0 * u0) * (sphi * sphi)) / (kRd * T0);
    T = T0;
    u = u0 * cphi;
  } else {
    const double zj = 10000.0, hj = 10000.0;
    double q = (zz - zj) / hj;
    double S = exp(-(q * q));
    double dS = -2.0 * (zz - zj) / (hj * hj) * S;
    double c3 = cphi * cphi * cphi, c5 = c3 * cphi * cphi;
    double Phi = -4.0 * (c3 / 3.0 - c5 / 5.0) + 4.0 / 15.0;
    lnp = (log(kP0) - zz / cd.H0) - cd.B * S * Phi;
    T = kGrav / (kRd * (1.0 / cd.H0 + cd.B * dS * Phi));
    double c = (kRd * T / kR) * cd.B * S * (4.0 * (cphi * cphi) * (sphi * sphi));
    double a = cphi > 1e-12 ? 1.0 / (kR * cphi) : 0.0;
    double b = 2.0 * kOmega;
    u = 2.0 * c / (b + sqrt(b * b + 4.0 * a * c));
  }
}

// one thread per column: theta_v, discrete hydrostatic Exner, noise, rho
// cells c0 .. c0+n-1; outputs at rows (c - c0) of the [n][ld] arrays
// On terrain-following levels (hs != NULL) a cell's full levels lie at z_f + hs bf and its
// centre spacings and interpolation weights are its own (wu_c, [Nc][ld]).
__global__ void k_init_cells(CaseDev cd, int64_t c0, int64_t n, const double* __restrict__ x_c,
                             const double* __restrict__ z_f, const double* __restrict__ dzh,
                             const double* __restrict__ wu, const double* __restrict__ wl,
                             const double* __restrict__ hs, const double* __restrict__ bf,
                             const double* __restrict__ wu_c, double* __restrict__ rho,
                             double* __restrict__ thv, double* __restrict__ ex, double* __restrict__ w) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t c = c0 + t;
  const int N = cd.N, ld = cd.ld;
  double x = x_c[3 * c], y = x_c[3 * c + 1], z = x_c[3 * c + 2];
  double* th = thv + t * ld;
  double* pe = ex + t * ld;
  double* rr = rho + t * ld;
  const double kap = kRd / kCpd;
  double exan_bottom = 0.0;
  const double hsc = hs ? hs[c] : 0.0;
  for (int k = 0; k < N; ++k) {
    double lnp, T, u;
    analytic(cd, x, y, z, hs ? z_f[k] + hsc * bf[k] : z_f[k], lnp, T, u);
    double exan = exp(kap * (lnp - log(kP0)));
    th[k] = T / exan;
    if (k == N - 1) exan_bottom = exan;
  }
  pe[N - 1] = exan_bottom;
  for (int k = N - 1; k > 0; --k) {
    double thic, dzk;
    if (hs) {
      const double wuc = wu_c[c * ld + k];
      thic = wuc * th[k - 1] + (1.0 - wuc) * th[k];
      dzk = dzh[k] + hsc * (bf[k - 1] - bf[k]);
    } else {
      thic = wu[k] * th[k - 1] + wl[k] * th[k];
      dzk = dzh[k];
    }
    pe[k - 1] = pe[k] - kGrav * dzk / (kCpd * thic);
  }
  if (cd.noise > 0.0) {
    for (int k = 0; k < N; ++k) {
      double U = uniform01(cd.seed, (uint64_t)c * (uint64_t)N + (uint64_t)k);
      th[k] = th[k] + cd.noise * (2.0 * U - 1.0);
    }
  }
  for (int k = 0; k < N; ++k) rr[k] = kP0 * pow(pe[k], kCvd / kRd) / (kRd * th[k]);
  for (int k = N; k < ld; ++k) { th[k] = 0.0; pe[k] = 0.0; rr[k] = 0.0; }
  for (int h = 0; h < ld; ++h) w[t * ld + h] = 0.0;
}

// one thread per (edge, level): vn = u . n with u = u_lambda e_lambda
// edges e0 .. e0+n-1; output rows (e - e0)
// on terrain-following levels an edge's full levels lie at z_f + hs_e bf, hs_e the mean of
// its two cells' surface heights
__global__ void k_init_edges(CaseDev cd, int64_t e0, int64_t n, const double* __restrict__ x_e,
                             const double* __restrict__ n_e, const double* __restrict__ z_f,
                             const int* __restrict__ e2c, const double* __restrict__ hs,
                             const double* __restrict__ bf, double* __restrict__ vn) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int ld = cd.ld;
  if (t >= n * ld) return;
  const int64_t e = e0 + t / ld;
  const int k = (int)(t % ld);
  if (k >= cd.N) { vn[t] = 0.0; return; }
  double x = x_e[3 * e], y = x_e[3 * e + 1], z = x_e[3 * e + 2];
  double lnp, T, u;
  const double zz = hs ? z_f[k] + (0.5 * (hs[e2c[2 * e]] + hs[e2c[2 * e + 1]])) * bf[k] : z_f[k];
  analytic(cd, x, y, z, zz, lnp, T, u);
  if (cd.has_bump) {
    double cx = y * cd.bz - z * cd.by, cy = z * cd.bx - x * cd.bz, cz = x * cd.by - y * cd.bx;
    double r = kR * atan2(sqrt((cx * cx + cy * cy) + cz * cz), (x * cd.bx + y * cd.by) + z * cd.bz);
    double q = r / (kR / 10.0);
    u = u + cd.bamp * exp(-(q * q));
  }
  double cphi, sphi, elx, ely;
  basis(x, y, z, cphi, sphi, elx, ely);
  double proj = (elx * n_e[3 * e] + ely * n_e[3 * e + 1]) + 0.0 * n_e[3 * e + 2];
  vn[t] = u * proj;
}

__global__ void k_exner_ref(int N, const double* __restrict__ z_f, const double* __restrict__ dzh,
                            const double* __restrict__ wu, const double* __restrict__ wl, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double kap = kRd / kCpd;
  double th[512];
  for (int k = 0; k < N; ++k) {
    double lnp = log(kP0) - kGrav * z_f[k] / (kRd * 250.0);
    th[k] = 250.0 / exp(kap * (lnp - log(kP0)));
    if (k == N - 1) out[k] = exp(kap * (lnp - log(kP0)));
  }
  for (int k = N - 1; k > 0; --k) {
    double thic = wu[k] * th[k - 1] + wl[k] * th[k];
    out[k - 1] = out[k] - kGrav * dzh[k] / (kCpd * thic);
  }
}

double jet_B() {
  const double c45 = std::sqrt(0.5), U = 35.0, Tj = 288.0;
  return (U * U / (kR * c45) + 2.0 * kOmega * U) * kR / (kRd * Tj);
}

// FP64 fields in [entity][ld] layout -> mixed-mode storage: FP64 level-major
// prognostics, FP32 vn and FP32 shadows of S^n
// rows 0..n-1 of the [n][ld] FP64 arrays hold cells c0..c0+n-1
__global__ void k_mixed_cells(int64_t nc, int64_t c0, int64_t n, int N, int ld, const double* __restrict__ w,
                              const double* __restrict__ rho, const double* __restrict__ thv,
                              const double* __restrict__ ex, const double* __restrict__ ex_ref,
                              const double* __restrict__ exref_c, double* __restrict__ w_lm, double* __restrict__ rho_lm, double* __restrict__ thv_lm,
                              double* __restrict__ ex_lm, float* __restrict__ w32, float* __restrict__ rho32,
                              float* __restrict__ thv32, float* __restrict__ exp32) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int64_t c = c0 + t / ld;
  const int k = (int)(t % ld);
  const int64_t g = c * ld + k;
  if (k <= N) {
    w_lm[(int64_t)k * nc + c] = w[t];
    w32[g] = (float)w[t];
  } else {
    w32[g] = 0.0f;
  }
  if (k < N) {
    rho_lm[(int64_t)k * nc + c] = rho[t];
    thv_lm[(int64_t)k * nc + c] = thv[t];
    ex_lm[(int64_t)k * nc + c] = ex[t];
    rho32[g] = (float)rho[t];
    thv32[g] = (float)thv[t];
    exp32[g] = (float)(ex[t] - (exref_c ? exref_c[g] : ex_ref[k]));
  } else {
    rho32[g] = 0.0f;
    thv32[g] = 0.0f;
    exp32[g] = 0.0f;
  }
}

__global__ void k_half(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = 0.5 * a[i];
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// shadows of S^n from the level-major FP64 prognostics
__global__ void k_mixed_shadows(int64_t nc, int N, int ld, const double* __restrict__ w_lm,
                                const double* __restrict__ rho_lm, const double* __restrict__ thv_lm,
                                const double* __restrict__ ex_lm, const double* __restrict__ ex_ref,
                                const double* __restrict__ exref_c, float* __restrict__ w32, float* __restrict__ rho32, float* __restrict__ thv32,
                                float* __restrict__ exp32) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nc * ld) return;
  const int64_t c = t / ld;
  const int k = (int)(t % ld);
  w32[t] = k <= N ? (float)w_lm[(int64_t)k * nc + c] : 0.0f;
  if (k < N) {
    rho32[t] = (float)rho_lm[(int64_t)k * nc + c];
    thv32[t] = (float)thv_lm[(int64_t)k * nc + c];
    exp32[t] = (float)(ex_lm[(int64_t)k * nc + c] - (exref_c ? exref_c[t] : ex_ref[k]));
  }
}

}  // namespace

void mixed_cells_from_fp64(icon_state* st, int64_t c0, int64_t n, const double* w, const double* rho,
                           const double* thv, const double* ex, cudaStream_t stream) {
  const GridDev& g = st->grid->g;
  const Vertical& v = st->grid->vert;
  StateDev& s = st->s;
  k_mixed_cells<<<blocks_for(n * v.ld, 256), 256, 0, stream>>>(g.nc, c0, n, v.N, v.ld, w, rho, thv, ex, s.ex_ref,
                                                               s.topo.on ? s.topo.exref_c : nullptr,
                                                               s.w, s.rho, s.thv, s.ex, s.w32, s.rho32, s.thv32,
                                                               s.exp32);
}

void mixed_refresh_shadows(icon_state* st, cudaStream_t stream) {
  const GridDev& g = st->grid->g;
  const Vertical& v = st->grid->vert;
  StateDev& s = st->s;
  const int64_t ncl = g.nc * v.ld;
  k_mixed_shadows<<<blocks_for(ncl, 256), 256, 0, stream>>>(g.nc, v.N, v.ld, s.w, s.rho, s.thv, s.ex, s.ex_ref,
                                                            s.topo.on ? s.topo.exref_c : nullptr,
                                                            s.w32, s.rho32, s.thv32, s.exp32);
}

int init_state_device(icon_state* st, uint64_t seed, int case_id, const icon_case_params& p, cudaStream_t stream) {
  const icon_grid* grid = st->grid;
  const GridDev& g = grid->g;
  const Vertical& v = grid->vert;
  StateDev& s = st->s;
  CaseDev cd;
  cd.case_id = case_id;
  cd.N = v.N;
  cd.ld = v.ld;
  cd.noise = p.noise_K >= 0.0 ? p.noise_K : (case_id == ICON_CASE_SBR ? 0.01 : 0.0);
  cd.B = jet_B();
  cd.H0 = kRd * 288.0 / kGrav;
  cd.seed = seed;
  cd.has_bump = 0;
  cd.bamp = cd.bx = cd.by = cd.bz = 0.0;
  const double pi = 3.141592653589793;
  if (case_id == ICON_CASE_JET || case_id == ICON_CASE_MEMBER) {
    double amp = 1.0, lon = 20.0 * pi / 180.0, lat = 40.0 * pi / 180.0;
    if (case_id == ICON_CASE_MEMBER) {
      uint64_t ms = splitmix64(seed, (uint64_t)p.member);
      cd.seed = ms;
      amp = 0.5 + 1.5 * uniform01(ms, 0);
      lon = 2.0 * pi * uniform01(ms, 1);
      lat = std::asin(2.0 * uniform01(ms, 2) - 1.0);
    }
    cd.has_bump = 1;
    cd.bamp = amp;
    cd.bx = std::cos(lat) * std::cos(lon);
    cd.by = std::cos(lat) * std::sin(lon);
    cd.bz = std::sin(lat);
  }
  k_exner_ref<<<1, 1, 0, stream>>>(v.N, v.d_z_f, v.d_dzh, v.d_wu, v.d_wl, s.ex_ref);
  if (s.exref32) k_to_f32<<<1, 256, 0, stream>>>(s.ex_ref, s.exref32, v.ld);
  if (s.precision == ICON_FP64) {
    k_half<<<blocks_for(3 * g.nc, 256), 256, 0, stream>>>(g.kin_w, s.kin_w_h, 3 * g.nc);
    k_half<<<blocks_for(3 * g.nc, 256), 256, 0, stream>>>(g.div_wa, s.div_wa_h, 3 * g.nc);
    const TopoDev& T = s.topo;
    k_init_cells<<<blocks_for(g.nc, 128), 128, 0, stream>>>(cd, 0, g.nc, g.x_c, v.d_z_f, v.d_dzh, v.d_wu, v.d_wl,
                                                            T.on ? T.hs : nullptr, T.bf, T.wu_c, s.rho, s.thv,
                                                            s.ex, s.w);
    k_init_edges<<<blocks_for(g.ne * v.ld, 256), 256, 0, stream>>>(cd, 0, g.ne, g.x_e, g.n_e, v.d_z_f, g.e2c,
                                                                   T.on ? T.hs : nullptr, T.bf, s.vn);
    ICON_CUDA(cudaGetLastError());
    return ICON_OK;
  }
  // mixed: the same FP64 initial state, computed in chunks of at most 2^21 cells
  // (edges) into bounded temporaries, then converted to the mixed-mode storage
  DeviceArena T;
  T.al = st->arena.al;
  const int64_t CH = (int64_t)1 << 21;
  const int64_t cch = g.nc < CH ? g.nc : CH, ech = g.ne < CH ? g.ne : CH;
  const size_t C = (size_t)(cch * v.ld), E = (size_t)(ech * v.ld);
  double *rho = T.get_n<double>(C), *thv = T.get_n<double>(C), *ex = T.get_n<double>(C), *w = T.get_n<double>(C);
  double* vn = T.get_n<double>(E);
  if (T.failed) {
    T.release();
    set_error("out of device memory for the initial state");
    return ICON_ENOMEM;
  }
  for (int64_t c0 = 0; c0 < g.nc; c0 += CH) {
    const int64_t n = (g.nc - c0) < CH ? (g.nc - c0) : CH;
    k_init_cells<<<blocks_for(n, 128), 128, 0, stream>>>(cd, c0, n, g.x_c, v.d_z_f, v.d_dzh, v.d_wu, v.d_wl,
                                                         s.topo.on ? s.topo.hs : nullptr, s.topo.bf, s.topo.wu_c,
                                                         rho, thv, ex, w);
    mixed_cells_from_fp64(st, c0, n, w, rho, thv, ex, stream);
  }
  for (int64_t e0 = 0; e0 < g.ne; e0 += CH) {
    const int64_t n = (g.ne - e0) < CH ? (g.ne - e0) : CH;
    k_init_edges<<<blocks_for(n * v.ld, 256), 256, 0, stream>>>(cd, e0, n, g.x_e, g.n_e, v.d_z_f, g.e2c,
                                                                s.topo.on ? s.topo.hs : nullptr, s.topo.bf, vn);
    k_to_f32<<<blocks_for(n * v.ld, 256), 256, 0, stream>>>(vn, s.vn32 + e0 * v.ld, n * v.ld);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  T.release();
  if (e != cudaSuccess) return cuda_fail(e, "mixed initial state");
  return ICON_OK;
}

}  // namespace icon
