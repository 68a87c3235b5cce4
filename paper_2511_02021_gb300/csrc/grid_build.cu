// Grid/connectivity builder on the GPU (sm_103a).
//
// Builds the icosahedral-triangular C grid RnBk (n = 2: k+1 bisections of the
// icosahedron) that ICON computes on (paper: Sec. "Current State of the Art";
// sizes of the 10 km and 1.25 km grids in Table 2; dual of hexagons and 12
// pentagons in Sec. "Separation of Concerns"). Numbering and geometry:
//
//  * Cell id = root face * 4^L + base-4 child digits of the bisection, children
//    (a, m_ab, m_ca), (m_ab, b, m_bc), (m_ca, m_bc, c), (m_bc, m_ca, m_ab) with
//    m_ab = normalize(a + b). This Morton order is the locality order of every
//    table: neighbours of nearby cells are nearby in memory.
//  * A vertex is identified across cells by its integer barycentric lattice
//    coordinates on its root face, canonicalised on shared root edges and
//    corners (never by comparing floats). Vertex id = rank of the vertex's
//    lowest (cell id * 3 + corner slot) among all vertices; edges likewise with
//    the local edge slot s (corner s -> corner (s+1)%3), identified by the lattice
//    coordinates of their midpoint on the twice finer lattice. The lowest
//    incident (cell, slot) is found with atomicMin into a dense array indexed by
//    the canonical lattice index and the ids by an exclusive scan of
//    "is representative" flags: no sort, and the result is deterministic.
//  * Geometry in FP64 on the unit sphere scaled by R: circumcentres
//    normalize((b-a) x (c-a)), midpoints normalize(v1+v2), normals
//    normalize(v2 x v1) (from c1 to c2), tangents x_e x n_e, great-circle
//    lengths, spherical-excess areas; vertex lists counter-clockwise from the
//    lowest edge id by walking the cells around each vertex; Perot tangential
//    weights, kinetic-energy weights and least-squares vertex-velocity weights.
#include <cmath>
#include <cstdio>
#include <vector>
#include "icon_internal.h"

namespace icon {
namespace {

struct V3 { double x, y, z; };
__host__ __device__ inline V3 v3(double x, double y, double z) { V3 r; r.x = x; r.y = y; r.z = z; return r; }
__host__ __device__ inline V3 add(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ inline V3 sub(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ inline double dot(V3 a, V3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
__host__ __device__ inline V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline V3 normalize(V3 v) {
  double s = sqrt(dot(v, v));
  return v3(v.x / s, v.y / s, v.z / s);
}
__device__ inline double arc(V3 a, V3 b) {
  V3 c = cross(a, b);
  return atan2(sqrt(dot(c, c)), dot(a, b));
}
// spherical excess, tan(E/2) = |a.(b x c)| / (1 + a.b + b.c + c.a)
__device__ inline double excess(V3 a, V3 b, V3 c) {
  double num = fabs(dot(a, cross(b, c)));
  double den = ((1.0 + dot(a, b)) + dot(b, c)) + dot(c, a);
  return 2.0 * atan2(num, den);
}
__device__ inline V3 ld3(const double* p, int64_t i) { return v3(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }
__device__ inline void st3(double* p, int64_t i, V3 v) { p[3 * i] = v.x; p[3 * i + 1] = v.y; p[3 * i + 2] = v.z; }

// root icosahedron: vertex positions (set from the host), faces and root-edge index
__constant__ double c_root_pos[12 * 3];
__constant__ int c_faces[20 * 3];
__constant__ signed char c_redge[12 * 12];

// canonical index of the lattice point with root-corner weights (i, j, k), i+j+k = n,
// on root face f: 12 corners, then 30 root edges x (n-1), then 20 faces x interior
__device__ inline int64_t canon(int f, int64_t i, int64_t j, int64_t k, int64_t n) {
  const int F0 = c_faces[3 * f], F1 = c_faces[3 * f + 1], F2 = c_faces[3 * f + 2];
  if (i == n) return F0;
  if (j == n) return F1;
  if (k == n) return F2;
  if (i == 0 || j == 0 || k == 0) {
    int P, Q;
    int64_t wq;
    if (i == 0) { P = F1; Q = F2; wq = k; if (P > Q) { P = F2; Q = F1; wq = j; } }
    else if (j == 0) { P = F0; Q = F2; wq = k; if (P > Q) { P = F2; Q = F0; wq = i; } }
    else { P = F0; Q = F1; wq = j; if (P > Q) { P = F1; Q = F0; wq = i; } }
    return 12 + (int64_t)c_redge[P * 12 + Q] * (n - 1) + (wq - 1);
  }
  const int64_t I = (n - 1) * (n - 2) / 2;
  const int64_t a = i - 1, b = j - 1;
  return 12 + 30 * (n - 1) + (int64_t)f * I + a * (n - 2) - a * (a - 1) / 2 + b;
}

struct L3 { int64_t i, j, k; };

// one thread per cell: corner positions and canonical vertex / edge-midpoint indices
__global__ void k_cells(int L, int64_t nc, double* __restrict__ corner_pos,
                        unsigned* __restrict__ cv, unsigned* __restrict__ ce) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int f = (int)(c >> (2 * L));
  V3 P[3];
  L3 B[3];
  for (int s = 0; s < 3; ++s) {
    int rv = c_faces[3 * f + s];
    P[s] = v3(c_root_pos[3 * rv], c_root_pos[3 * rv + 1], c_root_pos[3 * rv + 2]);
    B[s].i = (s == 0); B[s].j = (s == 1); B[s].k = (s == 2);
  }
  for (int l = 0; l < L; ++l) {
    int d = (int)((c >> (2 * (L - 1 - l))) & 3);
    V3 a = P[0], b = P[1], cc = P[2];
    V3 mab = normalize(add(a, b)), mbc = normalize(add(b, cc)), mca = normalize(add(cc, a));
    L3 la = {2 * B[0].i, 2 * B[0].j, 2 * B[0].k}, lb = {2 * B[1].i, 2 * B[1].j, 2 * B[1].k},
       lc = {2 * B[2].i, 2 * B[2].j, 2 * B[2].k};
    L3 lab = {B[0].i + B[1].i, B[0].j + B[1].j, B[0].k + B[1].k};
    L3 lbc = {B[1].i + B[2].i, B[1].j + B[2].j, B[1].k + B[2].k};
    L3 lca = {B[2].i + B[0].i, B[2].j + B[0].j, B[2].k + B[0].k};
    if (d == 0) { P[0] = a; P[1] = mab; P[2] = mca; B[0] = la; B[1] = lab; B[2] = lca; }
    else if (d == 1) { P[0] = mab; P[1] = b; P[2] = mbc; B[0] = lab; B[1] = lb; B[2] = lbc; }
    else if (d == 2) { P[0] = mca; P[1] = mbc; P[2] = cc; B[0] = lca; B[1] = lbc; B[2] = lc; }
    else { P[0] = mbc; P[1] = mca; P[2] = mab; B[0] = lbc; B[1] = lca; B[2] = lab; }
  }
  const int64_t n = (int64_t)1 << L;
  for (int s = 0; s < 3; ++s) {
    // -0.0 and 0.0 are the same point; store +0.0 (as the oracle does)
    V3 p = v3(P[s].x + 0.0, P[s].y + 0.0, P[s].z + 0.0);
    st3(corner_pos, 3 * c + s, p);
    cv[3 * c + s] = (unsigned)canon(f, B[s].i, B[s].j, B[s].k, n);
    const L3 &u = B[s], &w = B[(s + 1) % 3];
    ce[3 * c + s] = (unsigned)canon(f, u.i + w.i, u.j + w.j, u.k + w.k, 2 * n);
  }
}

__global__ void k_fill_u32(unsigned* p, int64_t n, unsigned v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}
__global__ void k_min_rep(const unsigned* __restrict__ key, int64_t n, unsigned* __restrict__ best) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) atomicMin(&best[key[t]], (unsigned)t);
}
__global__ void k_flag_rep(const unsigned* __restrict__ key, int64_t n, const unsigned* __restrict__ best,
                           unsigned* __restrict__ flag) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) flag[t] = (best[key[t]] == (unsigned)t) ? 1u : 0u;
}

// block-wide exclusive scan of one value per thread (blockDim.x == 1024)
__device__ unsigned block_exclusive(unsigned v, unsigned* total) {
  __shared__ unsigned ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned s = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  unsigned off = wid ? ws[wid - 1] : 0u;
  *total = ws[31];
  __syncthreads();
  return off + x - v;
}

constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(1024) k_scan_tiles(const unsigned* __restrict__ in, int64_t n,
                                                     unsigned* __restrict__ tile_sum) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  unsigned s = 0;
  for (int q = 0; q < kScanPer; ++q) s += (base + q < n) ? in[base + q] : 0u;
  unsigned tot;
  block_exclusive(s, &tot);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}
__global__ void __launch_bounds__(1024) k_scan_sums(unsigned* __restrict__ sums, int64_t nt,
                                                    unsigned* __restrict__ total) {
  unsigned carry = 0;
  for (int64_t b = 0; b < nt; b += kScanThreads) {
    int64_t i = b + threadIdx.x;
    unsigned v = (i < nt) ? sums[i] : 0u, tot;
    unsigned ex = block_exclusive(v, &tot);
    if (i < nt) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}
__global__ void __launch_bounds__(1024) k_scan_apply(const unsigned* __restrict__ in, int64_t n,
                                                     const unsigned* __restrict__ tile_off,
                                                     unsigned* __restrict__ out) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  unsigned v[kScanPer], s = 0;
  for (int q = 0; q < kScanPer; ++q) { v[q] = (base + q < n) ? in[base + q] : 0u; s += v[q]; }
  unsigned tot;
  unsigned ex = block_exclusive(s, &tot) + tile_off[blockIdx.x];
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < n) out[base + q] = ex;
    ex += v[q];
  }
}

// vertex ids, positions and representatives
__global__ void k_assign_vertices(int64_t n3, const unsigned* __restrict__ cv, const unsigned* __restrict__ best,
                                  const unsigned* __restrict__ flag, const unsigned* __restrict__ scan,
                                  const double* __restrict__ corner_pos, int* __restrict__ c2v,
                                  double* __restrict__ x_v, unsigned* __restrict__ vrep) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n3) return;
  unsigned rep = best[cv[t]];
  c2v[t] = (int)scan[rep];
  if (flag[t]) {
    unsigned vid = scan[t];
    x_v[3 * (int64_t)vid] = corner_pos[3 * t];
    x_v[3 * (int64_t)vid + 1] = corner_pos[3 * t + 1];
    x_v[3 * (int64_t)vid + 2] = corner_pos[3 * t + 2];
    vrep[vid] = (unsigned)t;
  }
}
__global__ void k_assign_edges(int64_t n3, const unsigned* __restrict__ ce, const unsigned* __restrict__ best,
                               const unsigned* __restrict__ flag, const unsigned* __restrict__ scan,
                               const int* __restrict__ c2v, int* __restrict__ c2e, int* __restrict__ e2c,
                               int* __restrict__ e2v) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n3) return;
  unsigned rep = best[ce[t]];
  unsigned e = scan[rep];
  c2e[t] = (int)e;
  const int64_t c = t / 3;
  const int s = (int)(t % 3);
  if (flag[t]) {
    e2c[2 * (int64_t)e] = (int)c;
    e2v[2 * (int64_t)e] = c2v[3 * c + s];
    e2v[2 * (int64_t)e + 1] = c2v[3 * c + (s + 1) % 3];
  } else {
    e2c[2 * (int64_t)e + 1] = (int)c;
  }
}

__global__ void k_cell_geom(int64_t nc, const int* __restrict__ c2v, const double* __restrict__ x_v,
                            double* __restrict__ x_c, double* __restrict__ A_c) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  V3 a = ld3(x_v, c2v[3 * c]), b = ld3(x_v, c2v[3 * c + 1]), cc = ld3(x_v, c2v[3 * c + 2]);
  st3(x_c, c, normalize(cross(sub(b, a), sub(cc, a))));
  A_c[c] = (kR * kR) * excess(a, b, cc);
}

__device__ inline int opposite_corner(const int* c2v, int64_t c, int va, int vb) {
  for (int s = 0; s < 3; ++s) {
    int v = c2v[3 * c + s];
    if (v != va && v != vb) return v;
  }
  return -1;
}

__global__ void k_edge_geom(int64_t ne, const int* __restrict__ e2c, const int* __restrict__ e2v,
                            const int* __restrict__ c2v, const double* __restrict__ x_v,
                            const double* __restrict__ x_c, double* __restrict__ x_e, double* __restrict__ n_e,
                            double* __restrict__ t_e, double* __restrict__ l_e, double* __restrict__ d_e,
                            double* __restrict__ f_e, int* __restrict__ e2q, double* __restrict__ L34,
                            unsigned* __restrict__ err) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int c1 = e2c[2 * e], c2 = e2c[2 * e + 1];
  const int iv1 = e2v[2 * e], iv2 = e2v[2 * e + 1];
  if (c1 < 0 || c2 < 0 || c1 >= c2) { atomicOr(err, 1u); return; }
  V3 v1 = ld3(x_v, iv1), v2 = ld3(x_v, iv2);
  V3 xe = normalize(add(v1, v2));
  V3 nn = normalize(cross(v2, v1));
  V3 tt = cross(xe, nn);
  st3(x_e, e, xe);
  st3(n_e, e, nn);
  st3(t_e, e, tt);
  l_e[e] = kR * arc(v1, v2);
  d_e[e] = kR * arc(ld3(x_c, c1), ld3(x_c, c2));
  f_e[e] = (2.0 * kOmega) * xe.z;
  int v3i = opposite_corner(c2v, c1, iv1, iv2), v4i = opposite_corner(c2v, c2, iv1, iv2);
  if (v3i < 0 || v4i < 0) { atomicOr(err, 2u); return; }
  e2q[4 * e] = iv1; e2q[4 * e + 1] = iv2; e2q[4 * e + 2] = v3i; e2q[4 * e + 3] = v4i;
  L34[e] = kR * arc(ld3(x_v, v3i), ld3(x_v, v4i));
}

__global__ void k_cell_weights(int64_t nc, const int* __restrict__ c2e, const int* __restrict__ e2c,
                               const double* __restrict__ x_c, const double* __restrict__ x_e,
                               const double* __restrict__ l_e, double* __restrict__ kin_w,
                               double* __restrict__ s_ce, double* __restrict__ div_w) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  V3 xc = ld3(x_c, c);
  double w[3];
  for (int s = 0; s < 3; ++s) {
    int e = c2e[3 * c + s];
    w[s] = l_e[e] * (kR * arc(xc, ld3(x_e, e)));
    double sg = (e2c[2 * (int64_t)e] == (int)c) ? 1.0 : -1.0;
    s_ce[3 * c + s] = sg;
    div_w[3 * c + s] = sg * l_e[e];
  }
  double tot = (w[0] + w[1]) + w[2];
  for (int s = 0; s < 3; ++s) kin_w[3 * c + s] = w[s] / tot;
}

// one thread per vertex: counter-clockwise walk around the vertex, dual area,
// circulation signs and least-squares weights
__global__ void k_vertex(int64_t nv, const unsigned* __restrict__ vrep, const int* __restrict__ c2v,
                         const int* __restrict__ c2e, const int* __restrict__ e2c, const int* __restrict__ e2v,
                         const double* __restrict__ x_v, const double* __restrict__ x_c,
                         const double* __restrict__ n_e, const double* __restrict__ d_e,
                         int* __restrict__ v2e, int* __restrict__ v2c, int* __restrict__ vdeg,
                         double* __restrict__ A_v, double* __restrict__ s_ve, double* __restrict__ rot_w,
                         double* __restrict__ lsq_w, unsigned* __restrict__ err) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nv) return;
  int el[6], cl[6];
  const unsigned t0 = vrep[v];
  const int c0 = (int)(t0 / 3);
  int c = c0, s = (int)(t0 % 3), deg = 0;
  for (int j = 0; j < 6; ++j) {
    el[j] = c2e[3 * c + s];                       // edge leaving v (corner s -> s+1)
    cl[j] = c;                                    // cell counter-clockwise after it
    int ein = c2e[3 * c + (s + 2) % 3];           // edge entering v (corner s+2 -> s)
    int cn = (e2c[2 * ein] == c) ? e2c[2 * ein + 1] : e2c[2 * ein];
    if (cn == c0) { deg = j + 1; break; }
    int sn = -1;
    for (int q = 0; q < 3; ++q) if (c2v[3 * cn + q] == (int)v) sn = q;
    if (sn < 0) break;
    c = cn; s = sn;
  }
  if (deg != 5 && deg != 6) { atomicOr(err, 4u); return; }
  int j0 = 0;
  for (int j = 1; j < deg; ++j) if (el[j] < el[j0]) j0 = j;
  int E[6], C[6];
  for (int j = 0; j < deg; ++j) { E[j] = el[(j0 + j) % deg]; C[j] = cl[(j0 + j) % deg]; }
  if (deg == 5) { E[5] = E[0]; C[5] = C[0]; }
  vdeg[v] = deg;
  V3 xv = ld3(x_v, v);
  double area = 0.0;
  for (int j = 0; j < 6; ++j) {
    v2e[6 * v + j] = E[j];
    v2c[6 * v + j] = C[j];
    if (j < deg) area += excess(xv, ld3(x_c, C[j]), ld3(x_c, C[(j + 1) % deg]));
    else area += 0.0;
    double sg = (j < deg) ? ((e2v[2 * (int64_t)E[j]] == (int)v) ? -1.0 : 1.0) : 0.0;
    s_ve[6 * v + j] = sg;
    rot_w[6 * v + j] = sg * d_e[E[j]];
  }
  A_v[v] = area * (kR * kR);
  // least squares: u = argmin sum_j (u.n_j - vn_j)^2, u in the tangent plane at x_v
  V3 ref = (fabs(xv.z) < 0.9) ? v3(0.0, 0.0, 1.0) : v3(1.0, 0.0, 0.0);
  V3 e1 = normalize(cross(ref, xv));
  V3 e2 = cross(xv, e1);
  double p1[6], p2[6], m11 = 0.0, m12 = 0.0, m22 = 0.0;
  for (int j = 0; j < 6; ++j) {
    double valid = (j < deg) ? 1.0 : 0.0;
    V3 nj = ld3(n_e, E[j]);
    p1[j] = dot(nj, e1) * valid;
    p2[j] = dot(nj, e2) * valid;
  }
  for (int j = 0; j < 6; ++j) m11 += p1[j] * p1[j];
  for (int j = 0; j < 6; ++j) m12 += p1[j] * p2[j];
  for (int j = 0; j < 6; ++j) m22 += p2[j] * p2[j];
  double det = m11 * m22 - m12 * m12;
  double i11 = m22 / det, i12 = -m12 / det, i22 = m11 / det;
  for (int j = 0; j < 6; ++j) {
    double q1 = i11 * p1[j] + i12 * p2[j];
    double q2 = i12 * p1[j] + i22 * p2[j];
    lsq_w[18 * v + 3 * j + 0] = q1 * e1.x + q2 * e2.x;
    lsq_w[18 * v + 3 * j + 1] = q1 * e1.y + q2 * e2.y;
    lsq_w[18 * v + 3 * j + 2] = q1 * e1.z + q2 * e2.z;
  }
}

// Perot tangential-velocity stencil: own edge, two other edges of c1, of c2
__global__ void k_edge_vt(int64_t ne, const int* __restrict__ e2c, const int* __restrict__ c2e,
                          const double* __restrict__ s_ce, const double* __restrict__ l_e,
                          const double* __restrict__ x_e, const double* __restrict__ x_c,
                          const double* __restrict__ t_e, const double* __restrict__ A_c,
                          int* __restrict__ e2vt, double* __restrict__ vt_w) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  V3 te = ld3(t_e, e);
  double w0 = 0.0;
  e2vt[5 * e] = (int)e;
  for (int side = 0; side < 2; ++side) {
    const int cs = e2c[2 * e + side];
    const int col = 1 + 2 * side;
    V3 xc = ld3(x_c, cs);
    int q = 0;
    double own = 0.0;
    for (int s = 0; s < 3; ++s) {
      int ej = c2e[3 * (int64_t)cs + s];
      double coef = ((((0.5 * s_ce[3 * (int64_t)cs + s]) * l_e[ej]) * kR) * dot(sub(ld3(x_e, ej), xc), te)) / A_c[cs];
      if (ej == (int)e) {
        own = coef;
      } else {
        e2vt[5 * e + col + q] = ej;
        vt_w[5 * e + col + q] = coef;
        ++q;
      }
    }
    w0 = w0 + own;
  }
  vt_w[5 * e] = w0;
}

// FP32 coefficient tables for the mixed-precision stencils (area divisions folded in)
__global__ void k_mixed_tables(int64_t nc, int64_t ne, int64_t nv, const double* __restrict__ div_w,
                               const double* __restrict__ A_c, const double* __restrict__ rot_w,
                               const double* __restrict__ A_v, const double* __restrict__ vt_w,
                               const double* __restrict__ kin_w, const double* __restrict__ lsq_w,
                               const double* __restrict__ d_e, const double* __restrict__ l_e,
                               const double* __restrict__ f_e, const double* __restrict__ n_e,
                               const double* __restrict__ t_e, const double* __restrict__ L34,
                               const double* __restrict__ s_ce, float* __restrict__ div32,
                               float* __restrict__ rot32, float* __restrict__ vt32, float* __restrict__ kin32,
                               float* __restrict__ lsq32, float* __restrict__ ide32, float* __restrict__ ile32,
                               float* __restrict__ fe32, float* __restrict__ le32, float* __restrict__ ne32,
                               float* __restrict__ te32, float* __restrict__ i34_32, float* __restrict__ sce32,
                               double* __restrict__ invAc, double* __restrict__ div_wa, double* __restrict__ rot_wa,
                               double* __restrict__ inv_de, double* __restrict__ inv_le,
                               double* __restrict__ inv_L34) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nc) {
    for (int s = 0; s < 3; ++s) {
      div32[3 * i + s] = (float)(div_w[3 * i + s] / A_c[i]);
      kin32[3 * i + s] = (float)kin_w[3 * i + s];
      sce32[3 * i + s] = (float)s_ce[3 * i + s];
      div_wa[3 * i + s] = div_w[3 * i + s] / A_c[i];
    }
    invAc[i] = 1.0 / A_c[i];
  }
  if (i < nv) {
    for (int j = 0; j < 6; ++j) {
      rot_wa[6 * i + j] = rot_w[6 * i + j] / A_v[i];
      rot32[6 * i + j] = (float)rot_wa[6 * i + j];
    }
    for (int j = 0; j < 18; ++j) lsq32[18 * i + j] = (float)lsq_w[18 * i + j];
  }
  if (i < ne) {
    for (int j = 0; j < 5; ++j) vt32[5 * i + j] = (float)vt_w[5 * i + j];
    ide32[i] = (float)(1.0 / d_e[i]);
    ile32[i] = (float)(1.0 / l_e[i]);
    fe32[i] = (float)f_e[i];
    le32[i] = (float)l_e[i];
    i34_32[i] = (float)(1.0 / L34[i]);
    inv_de[i] = 1.0 / d_e[i];
    inv_le[i] = 1.0 / l_e[i];
    inv_L34[i] = 1.0 / L34[i];
    for (int j = 0; j < 3; ++j) {
      ne32[3 * i + j] = (float)n_e[3 * i + j];
      te32[3 * i + j] = (float)t_e[3 * i + j];
    }
  }
}

void root_tables(double pos[36], int faces[60], signed char redge[144]) {
  pos[0] = 0.0; pos[1] = 0.0; pos[2] = 1.0;
  const double lat = std::atan(0.5);
  const double pi = 3.141592653589793;
  for (int i = 0; i < 5; ++i) {
    double ln = 2.0 * pi * i / 5.0;
    double ls = 2.0 * pi * (i + 0.5) / 5.0;
    pos[3 * (1 + i) + 0] = std::cos(lat) * std::cos(ln);
    pos[3 * (1 + i) + 1] = std::cos(lat) * std::sin(ln);
    pos[3 * (1 + i) + 2] = std::sin(lat);
    pos[3 * (6 + i) + 0] = std::cos(lat) * std::cos(ls);
    pos[3 * (6 + i) + 1] = std::cos(lat) * std::sin(ls);
    pos[3 * (6 + i) + 2] = -std::sin(lat);
  }
  pos[33] = 0.0; pos[34] = 0.0; pos[35] = -1.0;
  int f = 0;
  for (int i = 0; i < 5; ++i) { faces[3 * f] = 0; faces[3 * f + 1] = 1 + i; faces[3 * f + 2] = 1 + (i + 1) % 5; ++f; }
  for (int i = 0; i < 5; ++i) {
    faces[3 * f] = 1 + i; faces[3 * f + 1] = 6 + i; faces[3 * f + 2] = 1 + (i + 1) % 5; ++f;
    faces[3 * f] = 1 + (i + 1) % 5; faces[3 * f + 1] = 6 + i; faces[3 * f + 2] = 6 + (i + 1) % 5; ++f;
  }
  for (int i = 0; i < 5; ++i) { faces[3 * f] = 11; faces[3 * f + 1] = 6 + (i + 1) % 5; faces[3 * f + 2] = 6 + i; ++f; }
  for (int i = 0; i < 144; ++i) redge[i] = -1;
  int ne = 0;
  for (int q = 0; q < 20; ++q)
    for (int s = 0; s < 3; ++s) {
      int a = faces[3 * q + s], b = faces[3 * q + (s + 1) % 3];
      int P = a < b ? a : b, Q = a < b ? b : a;
      if (redge[P * 12 + Q] < 0) redge[P * 12 + Q] = (signed char)(ne++);
    }
}


// Tables of the tracer transport (built on demand): the neighbour across each cell
// edge, least-squares gradient weights per (cell, neighbour) as 3-vectors in the tangent
// plane at the cell centre, and the offsets R (x_e - x_c1), R (x_e - x_c2) of every edge.
// Least squares: g = argmin sum_s (q_s - q_c - g . d_s)^2 with d_s the neighbour offset
// R (x_s - x_c) projected on the tangent plane, solved in the basis e1 = normalize(ref x
// x_c) (ref the z axis unless |z_c| >= 0.9, else the x axis), e2 = x_c x e1.
__global__ void k_tracer_cells(int64_t nc, const int* __restrict__ c2e, const int* __restrict__ e2c,
                               const double* __restrict__ x_c, double R, int* __restrict__ c2c,
                               double* __restrict__ lsq_c) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const V3 xc = ld3(x_c, c);
  V3 d[3];
  for (int s = 0; s < 3; ++s) {
    const int e = c2e[3 * c + s];
    const int a = e2c[2 * e], b = e2c[2 * e + 1];
    const int nb = (a == (int)c) ? b : a;
    c2c[3 * c + s] = nb;
    const V3 xs = ld3(x_c, nb);
    V3 v = v3((xs.x - xc.x) * R, (xs.y - xc.y) * R, (xs.z - xc.z) * R);
    const double vn = dot(v, xc);
    d[s] = v3(v.x - vn * xc.x, v.y - vn * xc.y, v.z - vn * xc.z);
  }
  const V3 ref = fabs(xc.z) < 0.9 ? v3(0.0, 0.0, 1.0) : v3(1.0, 0.0, 0.0);
  const V3 e1 = normalize(cross(ref, xc));
  const V3 e2 = cross(xc, e1);
  double p1[3], p2[3];
  for (int s = 0; s < 3; ++s) {
    p1[s] = dot(d[s], e1);
    p2[s] = dot(d[s], e2);
  }
  const double m11 = (p1[0] * p1[0] + p1[1] * p1[1]) + p1[2] * p1[2];
  const double m12 = (p1[0] * p2[0] + p1[1] * p2[1]) + p1[2] * p2[2];
  const double m22 = (p2[0] * p2[0] + p2[1] * p2[1]) + p2[2] * p2[2];
  const double det = m11 * m22 - m12 * m12;
  const double i11 = m22 / det, i12 = -m12 / det, i22 = m11 / det;
  for (int s = 0; s < 3; ++s) {
    const double q1 = i11 * p1[s] + i12 * p2[s];
    const double q2 = i12 * p1[s] + i22 * p2[s];
    st3(lsq_c, 3 * c + s, v3(q1 * e1.x + q2 * e2.x, q1 * e1.y + q2 * e2.y, q1 * e1.z + q2 * e2.z));
  }
}

__global__ void k_tracer_edges(int64_t ne, const int* __restrict__ e2c, const double* __restrict__ x_c,
                               const double* __restrict__ x_e, double R, double* __restrict__ roff) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const V3 xe = ld3(x_e, e);
  for (int j = 0; j < 2; ++j) {
    const V3 xc = ld3(x_c, e2c[2 * e + j]);
    st3(roff, 2 * e + j, v3((xe.x - xc.x) * R, (xe.y - xc.y) * R, (xe.z - xc.z) * R));
  }
}
}  // namespace

int exclusive_scan_u32(const unsigned* in, unsigned* out, int64_t n, unsigned* total_dev, DeviceArena& tmp,
                       cudaStream_t st) {
  int64_t nt = (n + kScanTile - 1) / kScanTile;
  unsigned* sums = tmp.get_n<unsigned>((size_t)nt + 1);
  if (!sums) { set_error("scan: out of device memory"); return ICON_ENOMEM; }
  k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, st>>>(in, n, sums);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nt, total_dev);
  k_scan_apply<<<(unsigned)nt, kScanThreads, 0, st>>>(in, n, sums, out);
  ICON_CUDA(cudaGetLastError());
  return ICON_OK;
}

int build_grid_device(icon_grid* grid, cudaStream_t st) {
  GridDev& g = grid->g;
  const int L = grid->bisections + 1;
  g.L = L;
  const int64_t n = (int64_t)1 << L;
  g.nc = 20 * n * n;
  g.ne = 30 * n * n;
  g.nv = 10 * n * n + 2;
  const int64_t nc = g.nc, ne = g.ne, nv = g.nv, n3 = 3 * nc;
  const int64_t nvcan = nv, necan = 10 * (2 * n) * (2 * n) + 2;

  double pos[36];
  int faces[60];
  signed char redge[144];
  root_tables(pos, faces, redge);
  ICON_CUDA(cudaMemcpyToSymbolAsync(c_root_pos, pos, sizeof(pos), 0, cudaMemcpyHostToDevice, st));
  ICON_CUDA(cudaMemcpyToSymbolAsync(c_faces, faces, sizeof(faces), 0, cudaMemcpyHostToDevice, st));
  ICON_CUDA(cudaMemcpyToSymbolAsync(c_redge, redge, sizeof(redge), 0, cudaMemcpyHostToDevice, st));

  DeviceArena& A = grid->arena;
  DeviceArena T;                    // temporaries of the build
  T.al = A.al;
  struct TmpGuard { DeviceArena& t; ~TmpGuard() { t.release(); } } guard{T};

  g.c2v = A.get_n<int>(n3); g.c2e = A.get_n<int>(n3);
  g.e2c = A.get_n<int>(2 * ne); g.e2v = A.get_n<int>(2 * ne);
  g.v2e = A.get_n<int>(6 * nv); g.v2c = A.get_n<int>(6 * nv); g.vdeg = A.get_n<int>(nv);
  g.e2vt = A.get_n<int>(5 * ne); g.e2q = A.get_n<int>(4 * ne);
  g.x_c = A.get_n<double>(3 * nc); g.x_e = A.get_n<double>(3 * ne); g.x_v = A.get_n<double>(3 * nv);
  g.n_e = A.get_n<double>(3 * ne); g.t_e = A.get_n<double>(3 * ne);
  g.l_e = A.get_n<double>(ne); g.d_e = A.get_n<double>(ne); g.A_c = A.get_n<double>(nc);
  g.A_v = A.get_n<double>(nv); g.f_e = A.get_n<double>(ne);
  g.vt_w = A.get_n<double>(5 * ne); g.kin_w = A.get_n<double>(3 * nc); g.lsq_w = A.get_n<double>(18 * nv);
  g.L34 = A.get_n<double>(ne); g.s_ce = A.get_n<double>(3 * nc); g.s_ve = A.get_n<double>(6 * nv);
  g.div_w = A.get_n<double>(3 * nc); g.rot_w = A.get_n<double>(6 * nv);
  g.vt_w32 = A.get_n<float>(5 * ne); g.kin_w32 = A.get_n<float>(3 * nc); g.lsq_w32 = A.get_n<float>(18 * nv);
  g.div_w32 = A.get_n<float>(3 * nc); g.rot_w32 = A.get_n<float>(6 * nv);
  g.inv_de32 = A.get_n<float>(ne); g.inv_le32 = A.get_n<float>(ne); g.f_e32 = A.get_n<float>(ne);
  g.l_e32 = A.get_n<float>(ne); g.n_e32 = A.get_n<float>(3 * ne); g.t_e32 = A.get_n<float>(3 * ne);
  g.L34inv32 = A.get_n<float>(ne); g.s_ce32 = A.get_n<float>(3 * nc); g.inv_Ac = A.get_n<double>(nc);
  g.div_wa = A.get_n<double>(3 * nc); g.rot_wa = A.get_n<double>(6 * nv);
  g.inv_de = A.get_n<double>(ne); g.inv_le = A.get_n<double>(ne); g.inv_L34 = A.get_n<double>(ne);
  double* corner_pos = T.get_n<double>(9 * nc);
  unsigned* cv = T.get_n<unsigned>(n3);
  unsigned* ce = T.get_n<unsigned>(n3);
  unsigned* vbest = T.get_n<unsigned>(nvcan);
  unsigned* ebest = T.get_n<unsigned>(necan);
  unsigned* flag = T.get_n<unsigned>(n3);
  unsigned* scan = T.get_n<unsigned>(n3);
  unsigned* vrep = T.get_n<unsigned>(nv);
  unsigned* dev_u = T.get_n<unsigned>(4);   // [0] vertex total, [1] edge total, [2] error bits
  if (A.failed || T.failed) { set_error("grid build: out of device memory"); return ICON_ENOMEM; }
  ICON_CUDA(cudaMemsetAsync(dev_u, 0, 4 * sizeof(unsigned), st));

  const int TB = 256;
  k_cells<<<blocks_for(nc, TB), TB, 0, st>>>(L, nc, corner_pos, cv, ce);
  // vertices
  k_fill_u32<<<blocks_for(nvcan, TB), TB, 0, st>>>(vbest, nvcan, 0xffffffffu);
  k_min_rep<<<blocks_for(n3, TB), TB, 0, st>>>(cv, n3, vbest);
  k_flag_rep<<<blocks_for(n3, TB), TB, 0, st>>>(cv, n3, vbest, flag);
  int rc = exclusive_scan_u32(flag, scan, n3, dev_u + 0, T, st);
  if (rc) return rc;
  k_assign_vertices<<<blocks_for(n3, TB), TB, 0, st>>>(n3, cv, vbest, flag, scan, corner_pos, g.c2v, g.x_v, vrep);
  // edges
  k_fill_u32<<<blocks_for(necan, TB), TB, 0, st>>>(ebest, necan, 0xffffffffu);
  k_min_rep<<<blocks_for(n3, TB), TB, 0, st>>>(ce, n3, ebest);
  k_flag_rep<<<blocks_for(n3, TB), TB, 0, st>>>(ce, n3, ebest, flag);
  rc = exclusive_scan_u32(flag, scan, n3, dev_u + 1, T, st);
  if (rc) return rc;
  ICON_CUDA(cudaMemsetAsync(g.e2c, 0xff, 2 * ne * sizeof(int), st));
  k_assign_edges<<<blocks_for(n3, TB), TB, 0, st>>>(n3, ce, ebest, flag, scan, g.c2v, g.c2e, g.e2c, g.e2v);
  // geometry and weights
  k_cell_geom<<<blocks_for(nc, TB), TB, 0, st>>>(nc, g.c2v, g.x_v, g.x_c, g.A_c);
  k_edge_geom<<<blocks_for(ne, TB), TB, 0, st>>>(ne, g.e2c, g.e2v, g.c2v, g.x_v, g.x_c, g.x_e, g.n_e, g.t_e,
                                                  g.l_e, g.d_e, g.f_e, g.e2q, g.L34, dev_u + 2);
  k_cell_weights<<<blocks_for(nc, TB), TB, 0, st>>>(nc, g.c2e, g.e2c, g.x_c, g.x_e, g.l_e, g.kin_w, g.s_ce,
                                                     g.div_w);
  k_vertex<<<blocks_for(nv, 128), 128, 0, st>>>(nv, vrep, g.c2v, g.c2e, g.e2c, g.e2v, g.x_v, g.x_c, g.n_e,
                                                 g.d_e, g.v2e, g.v2c, g.vdeg, g.A_v, g.s_ve, g.rot_w, g.lsq_w,
                                                 dev_u + 2);
  k_edge_vt<<<blocks_for(ne, TB), TB, 0, st>>>(ne, g.e2c, g.c2e, g.s_ce, g.l_e, g.x_e, g.x_c, g.t_e, g.A_c,
                                                g.e2vt, g.vt_w);
  int64_t nmax = nc > ne ? (nc > nv ? nc : nv) : (ne > nv ? ne : nv);
  k_mixed_tables<<<blocks_for(nmax, TB), TB, 0, st>>>(nc, ne, nv, g.div_w, g.A_c, g.rot_w, g.A_v, g.vt_w,
                                                       g.kin_w, g.lsq_w, g.d_e, g.l_e, g.f_e, g.n_e, g.t_e,
                                                       g.L34, g.s_ce, g.div_w32, g.rot_w32, g.vt_w32, g.kin_w32,
                                                       g.lsq_w32, g.inv_de32, g.inv_le32, g.f_e32, g.l_e32,
                                                       g.n_e32, g.t_e32, g.L34inv32, g.s_ce32, g.inv_Ac,
                                                       g.div_wa, g.rot_wa, g.inv_de, g.inv_le, g.inv_L34);
  ICON_CUDA(cudaGetLastError());
  unsigned host_u[4];
  ICON_CUDA(cudaMemcpyAsync(host_u, dev_u, sizeof(host_u), cudaMemcpyDeviceToHost, st));
  ICON_CUDA(cudaStreamSynchronize(st));
  if (host_u[0] != (unsigned)nv || host_u[1] != (unsigned)ne || host_u[2] != 0) {
    set_error("grid build: inconsistent connectivity (vertices %u/%lld, edges %u/%lld, flags %u)", host_u[0],
              (long long)nv, host_u[1], (long long)ne, host_u[2]);
    return ICON_EINDEX;
  }
  return ICON_OK;
}

int build_tracer_tables(icon_grid* grid, cudaStream_t st) {
  GridDev& g = grid->g;
  if (g.c2c) return ICON_OK;
  DeviceArena& A = grid->arena;
  int* c2c = A.get_n<int>(3 * g.nc);
  double* lsq_c = A.get_n<double>(9 * g.nc);
  double* roff = A.get_n<double>(6 * g.ne);
  const Vertical& v = grid->vert;
  std::vector<double> lev(3 * (size_t)v.ld, 0.0);
  for (int k = 1; k + 1 < v.N; ++k) lev[k] = 1.0 / (v.z_f[k - 1] - v.z_f[k + 1]);
  for (int h = 1; h < v.N; ++h) {
    lev[v.ld + h] = v.z_h[h] - v.z_f[h];
    lev[2 * v.ld + h] = v.z_h[h] - v.z_f[h - 1];
  }
  double* tr_lev = A.get_n<double>(3 * (size_t)v.ld);
  if (!c2c || !lsq_c || !roff || !tr_lev) {
    set_error("out of device memory (tracer tables)");
    return ICON_ENOMEM;
  }
  const int TB = 256;
  k_tracer_cells<<<blocks_for(g.nc, TB), TB, 0, st>>>(g.nc, g.c2e, g.e2c, g.x_c, kR, c2c, lsq_c);
  k_tracer_edges<<<blocks_for(g.ne, TB), TB, 0, st>>>(g.ne, g.e2c, g.x_c, g.x_e, kR, roff);
  ICON_CUDA(cudaMemcpyAsync(tr_lev, lev.data(), sizeof(double) * lev.size(), cudaMemcpyHostToDevice, st));
  ICON_CUDA(cudaGetLastError());
  ICON_CUDA(cudaStreamSynchronize(st));
  g.tr_lev = tr_lev;
  g.c2c = c2c;
  g.lsq_c = lsq_c;
  g.roff = roff;
  return ICON_OK;
}

}  // namespace icon
