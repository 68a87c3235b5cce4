// Horizontal domain decomposition of the FP64 step with halo exchanges.
//
// The paper's model runs the atmosphere decomposed horizontally over thousands of GPUs,
// exchanging subdomain halos point to point after its stencil phases (Sec. "Exploiting
// the Earth System's Complexity to Flexibly Utilize System Parallelism"). Here:
//
//  * Partition: part p owns the contiguous range [p Nc/P, (p+1) Nc/P) of the Morton cell
//    order (the locality order of the grid), the edges whose first cell c1 (the lower cell
//    id) it owns and the vertices whose lowest incident cell it owns. Every entity has
//    exactly one owner.
//  * Halo: the local cells of a part are its owned cells and every cell within R vertex
//    rings of them (a ring adds the cells sharing a vertex with the set); the local edges
//    and vertices are those of the local cells. Local numbering: owned entities first, then
//    halo entities, each in ascending global order, so the owned rows of a part are the
//    contiguous prefix of its arrays. Neighbour tables keep the global slot order (remapped
//    to local ids); a neighbour outside the local set points at local entity 0, which
//    keeps every access in bounds (the values computed there are discarded: they lie in
//    the outer halo and are overwritten by the next exchange).
//  * Step: every part runs the same kernels as the single-domain step on its local grid
//    (the divergence damping with the global grid's mean cell area); after each predictor
//    and corrector stage the halo rows of the stage's outputs (vn on edges; w, rho,
//    theta_v, Exner on cells) are copied from their owners, and after the diffusion the
//    halo rows of vn, theta_v and Exner. With R >= 3 the owned entities of every stage
//    read only values that are correct, so each part's owned results are bit-identical to
//    the single-domain step's (the kernels compute every entity in the same order from
//    the same inputs).
//  * Mass: each part sums its owned cells (fixed order), the P partial sums are added in
//    part order on the host (the scalar all-reduce of a multi-GPU run).
//
// On one GPU the parts are states in one process and an exchange is a gather kernel that
// reads the owners' rows directly; across GPUs the same lists would drive peer copies.
#include <algorithm>
#include <cstring>
#include <vector>
#include "icon_internal.h"

namespace icon {
namespace {

// the plan of one part from host connectivity tables
struct PartPlan {
  int64_t own[3] = {0, 0, 0};              // owned cells, edges, vertices
  std::vector<int> g[3];                   // local -> global id (cells, edges, vertices)
};

struct GlobalOwners {
  std::vector<int> owner[3];               // owning part of every cell, edge, vertex
  std::vector<int> oidx[3];                // local index of the entity in its owner's arrays
};

int64_t part_lo(int64_t nc, int P, int p) { return (int64_t)p * nc / P; }

int cell_owner(int64_t c, int64_t nc, int P) {
  int p = (int)((c * P) / nc);
  while (p + 1 < P && part_lo(nc, P, p + 1) <= c) ++p;
  while (p > 0 && part_lo(nc, P, p) > c) --p;
  return p;
}

void global_owners(int64_t nc, int64_t ne, int64_t nv, const int* e2c, const int* v2c, const int* vdeg, int P,
                   GlobalOwners& O) {
  O.owner[0].resize(nc); O.owner[1].resize(ne); O.owner[2].resize(nv);
  O.oidx[0].resize(nc); O.oidx[1].resize(ne); O.oidx[2].resize(nv);
  for (int64_t c = 0; c < nc; ++c) {
    O.owner[0][c] = cell_owner(c, nc, P);
    O.oidx[0][c] = (int)(c - part_lo(nc, P, O.owner[0][c]));
  }
  std::vector<int> cnt(P, 0);
  for (int64_t e = 0; e < ne; ++e) {
    const int p = O.owner[0][e2c[2 * e]];
    O.owner[1][e] = p;
    O.oidx[1][e] = cnt[p]++;
  }
  std::fill(cnt.begin(), cnt.end(), 0);
  for (int64_t v = 0; v < nv; ++v) {
    int cmin = v2c[6 * v];
    for (int j = 1; j < vdeg[v]; ++j) cmin = std::min(cmin, v2c[6 * v + j]);
    const int p = O.owner[0][cmin];
    O.owner[2][v] = p;
    O.oidx[2][v] = cnt[p]++;
  }
}

int build_plan(int64_t nc, int64_t ne, int64_t nv, const int* c2e, const int* c2v, const int* v2c,
               const int* vdeg, const GlobalOwners& O, int P, int part, int rings, PartPlan& plan) {
  std::vector<char> inC(nc, 0), inE(ne, 0), inV(nv, 0);
  const int64_t lo = part_lo(nc, P, part), hi = part_lo(nc, P, part + 1);
  std::vector<int> frontier;
  for (int64_t c = lo; c < hi; ++c) {
    inC[c] = 1;
    frontier.push_back((int)c);
  }
  for (int r = 0; r < rings; ++r) {
    std::vector<int> next;
    for (int c : frontier)
      for (int s = 0; s < 3; ++s) {
        const int v = c2v[3 * c + s];
        for (int j = 0; j < vdeg[v]; ++j) {
          const int cn = v2c[6 * v + j];
          if (!inC[cn]) {
            inC[cn] = 1;
            next.push_back(cn);
          }
        }
      }
    frontier.swap(next);
  }
  for (int64_t c = 0; c < nc; ++c)
    if (inC[c])
      for (int s = 0; s < 3; ++s) {
        inE[c2e[3 * c + s]] = 1;
        inV[c2v[3 * c + s]] = 1;
      }
  const char* in[3] = {inC.data(), inE.data(), inV.data()};
  const int64_t n[3] = {nc, ne, nv};
  for (int t = 0; t < 3; ++t) {
    plan.g[t].clear();
    for (int64_t i = 0; i < n[t]; ++i)
      if (in[t][i] && O.owner[t][i] == part) plan.g[t].push_back((int)i);
    plan.own[t] = (int64_t)plan.g[t].size();
    for (int64_t i = 0; i < n[t]; ++i)
      if (in[t][i] && O.owner[t][i] != part) plan.g[t].push_back((int)i);
  }
  // every owned entity must be local (an owned edge or vertex belongs to an owned cell)
  for (int t = 1; t < 3; ++t) {
    int64_t owned_total = 0;
    for (int64_t i = 0; i < n[t]; ++i) owned_total += O.owner[t][i] == part;
    if (owned_total != plan.own[t]) {
      set_error("domain plan: part %d owns %lld entities of kind %d but only %lld are local", part,
                (long long)owned_total, t, (long long)plan.own[t]);
      return ICON_EINDEX;
    }
  }
  return ICON_OK;
}

// ---------------------------------------------------------------- device helpers
template <class T>
__global__ void k_gather_rows(int64_t n, int width, const int* __restrict__ map, const T* __restrict__ src,
                              T* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * width) return;
  const int64_t r = i / width;
  const int j = (int)(i % width);
  dst[i] = src[(int64_t)map[r] * width + j];
}

// local neighbour table: global ids of the rows map[], translated by g2l (-1 -> 0)
__global__ void k_remap_rows(int64_t n, int width, const int* __restrict__ map, const int* __restrict__ src,
                             const int* __restrict__ g2l, int* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * width) return;
  const int64_t r = i / width;
  const int j = (int)(i % width);
  const int l = g2l[src[(int64_t)map[r] * width + j]];
  dst[i] = l >= 0 ? l : 0;
}

// halo exchange of [n][ld] rows: row loc[i] of dst <- row oidx[i] of the owner's array src[own[i]]
__global__ void k_halo_rows(int64_t nh, int ld, const int* __restrict__ loc, const int* __restrict__ own,
                            const int* __restrict__ oidx, const double* const* __restrict__ src,
                            double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= nh) return;
  const double* __restrict__ s = src[own[i]] + (int64_t)oidx[i] * ld;
  double* __restrict__ d = dst + (int64_t)loc[i] * ld;
  for (int k = threadIdx.x & 31; k < ld; k += 32) d[k] = s[k];
}

// mass of the first n cells (owned), fixed order: one partial per block of 1024 cells
constexpr int kDomMassCells = 1024;
__global__ void __launch_bounds__(256) k_dom_mass_partial(int64_t n, int N, int ld, const double* __restrict__ rho,
                                                          const double* __restrict__ dz, const double* __restrict__ A_c,
                                                          double* __restrict__ part) {
  __shared__ double ws[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kDomMassCells;
  const int64_t c1 = c0 + kDomMassCells < n ? c0 + kDomMassCells : n;
  double acc = 0.0;
  for (int64_t c = c0 + wid; c < c1; c += 8) {
    double col = 0.0;
    for (int k = lane; k < N; k += 32) col += rho[c * ld + k] * dz[k];
    for (int o = 16; o > 0; o >>= 1) col += __shfl_xor_sync(0xffffffffu, col, o);
    acc += A_c[c] * col;
  }
  if (lane == 0) ws[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += ws[i];
    part[blockIdx.x] = s;
  }
}

__global__ void k_dom_mass_final(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    out[0] = s;
  }
}

}  // namespace
}  // namespace icon

struct icon_domain {
  const icon_grid* grid = nullptr;
  int nparts = 0, rings = 0;
  icon::DeviceArena arena;                                  // pointer tables, exchange lists, mass
  std::vector<icon::PartPlan> plans;
  std::vector<icon_grid*> grids;                            // local grids (own arenas)
  std::vector<icon_state*> states;
  // halo lists per part and kind (0 cells, 1 edges): local index, owner part, owner's index
  std::vector<int*> hloc[2], hown[2], hoidx[2];
  std::vector<int64_t> nh[2];
  // device tables of the parts' field pointers, one per exchanged field
  enum { FC_W = 0, FC_RHO, FC_THV, FC_EX, FC_W_S, FC_RHO_S, FC_THV_S, FC_EX_S, FE_VN, FE_VN_S, F_COUNT };
  double** ptrs = nullptr;                                  // [F_COUNT][nparts]
  double* mass_part = nullptr;
  int mass_nblk = 0;
  double* mass_out = nullptr;                               // [nparts]
};

namespace icon {
namespace {

int copy_table_host(const icon_grid* grid, int id, std::vector<int>& out, size_t n) {
  out.resize(n);
  return icon_grid_copy_table(grid, id, out.data(), n * sizeof(int));
}

// build the local grid of one part: remapped connectivity, gathered geometry and weights,
// the global vertical grid (device arrays shared with the global grid)
int build_local_grid(const icon_grid* G, const PartPlan& plan, icon_grid* L, cudaStream_t st) {
  const GridDev& g = G->g;
  GridDev& l = L->g;
  DeviceArena& A = L->arena;
  L->root = G->root;
  L->bisections = G->bisections;
  L->device = G->device;
  L->vert = G->vert;
  l.nc = (int64_t)plan.g[0].size();
  l.ne = (int64_t)plan.g[1].size();
  l.nv = (int64_t)plan.g[2].size();
  l.L = g.L;
  int* map[3];
  int* g2l[3];
  const int64_t n_g[3] = {g.nc, g.ne, g.nv};
  const int64_t n_l[3] = {l.nc, l.ne, l.nv};
  for (int t = 0; t < 3; ++t) {
    map[t] = A.get_n<int>(n_l[t]);
    g2l[t] = A.get_n<int>(n_g[t]);
    if (A.failed) return ICON_ENOMEM;
    std::vector<int> h(n_g[t], -1);
    for (int64_t i = 0; i < n_l[t]; ++i) h[plan.g[t][i]] = (int)i;
    ICON_CUDA(cudaMemcpyAsync(map[t], plan.g[t].data(), sizeof(int) * n_l[t], cudaMemcpyHostToDevice, st));
    ICON_CUDA(cudaMemcpyAsync(g2l[t], h.data(), sizeof(int) * n_g[t], cudaMemcpyHostToDevice, st));
    ICON_CUDA(cudaStreamSynchronize(st));           // the host vectors go out of scope
  }
  // connectivity: rows of kind `row`, entries of kind `ent`
  struct IT { int** dst; const int* src; int row, ent, width; };
  const IT its[] = {{&l.c2v, g.c2v, 0, 2, 3}, {&l.c2e, g.c2e, 0, 1, 3}, {&l.e2c, g.e2c, 1, 0, 2},
                    {&l.e2v, g.e2v, 1, 2, 2}, {&l.v2e, g.v2e, 2, 1, 6}, {&l.v2c, g.v2c, 2, 0, 6},
                    {&l.e2vt, g.e2vt, 1, 1, 5}, {&l.e2q, g.e2q, 1, 2, 4}};
  for (const IT& it : its) {
    *it.dst = A.get_n<int>((size_t)n_l[it.row] * it.width);
    if (!*it.dst) return ICON_ENOMEM;
    const int64_t n = n_l[it.row];
    k_remap_rows<<<blocks_for(n * it.width, 256), 256, 0, st>>>(n, it.width, map[it.row], it.src, g2l[it.ent],
                                                               *it.dst);
  }
  l.vdeg = A.get_n<int>(l.nv);
  if (!l.vdeg) return ICON_ENOMEM;
  k_gather_rows<int><<<blocks_for(l.nv, 256), 256, 0, st>>>(l.nv, 1, map[2], g.vdeg, l.vdeg);
  // geometry and weights (FP64)
  struct DT { double** dst; const double* src; int row, width; };
  const DT dts[] = {{&l.x_c, g.x_c, 0, 3}, {&l.x_e, g.x_e, 1, 3}, {&l.x_v, g.x_v, 2, 3}, {&l.n_e, g.n_e, 1, 3},
                    {&l.t_e, g.t_e, 1, 3}, {&l.l_e, g.l_e, 1, 1}, {&l.d_e, g.d_e, 1, 1}, {&l.A_c, g.A_c, 0, 1},
                    {&l.A_v, g.A_v, 2, 1}, {&l.f_e, g.f_e, 1, 1}, {&l.vt_w, g.vt_w, 1, 5},
                    {&l.kin_w, g.kin_w, 0, 3}, {&l.lsq_w, g.lsq_w, 2, 18}, {&l.L34, g.L34, 1, 1},
                    {&l.s_ce, g.s_ce, 0, 3}, {&l.s_ve, g.s_ve, 2, 6}, {&l.div_w, g.div_w, 0, 3},
                    {&l.rot_w, g.rot_w, 2, 6}, {&l.inv_Ac, g.inv_Ac, 0, 1}, {&l.div_wa, g.div_wa, 0, 3},
                    {&l.rot_wa, g.rot_wa, 2, 6}, {&l.inv_de, g.inv_de, 1, 1}, {&l.inv_le, g.inv_le, 1, 1},
                    {&l.inv_L34, g.inv_L34, 1, 1}};
  for (const DT& d : dts) {
    if (!d.src) continue;
    *d.dst = A.get_n<double>((size_t)n_l[d.row] * d.width);
    if (!*d.dst) return ICON_ENOMEM;
    const int64_t n = n_l[d.row];
    k_gather_rows<double><<<blocks_for(n * d.width, 256), 256, 0, st>>>(n, d.width, map[d.row], d.src, *d.dst);
  }
  ICON_CUDA(cudaGetLastError());
  ICON_CUDA(cudaStreamSynchronize(st));
  return ICON_OK;
}

double* field_ptr(icon_state* st, int f) {
  StateDev& s = st->s;
  switch (f) {
    case icon_domain::FC_W: return s.w;
    case icon_domain::FC_RHO: return s.rho;
    case icon_domain::FC_THV: return s.thv;
    case icon_domain::FC_EX: return s.ex;
    case icon_domain::FC_W_S: return s.w_s;
    case icon_domain::FC_RHO_S: return s.rho_s;
    case icon_domain::FC_THV_S: return s.thv_s;
    case icon_domain::FC_EX_S: return s.ex_s;
    case icon_domain::FE_VN: return s.vn;
    case icon_domain::FE_VN_S: return s.vn_s;
    default: return nullptr;
  }
}

void exchange(icon_domain* D, std::initializer_list<int> fields, cudaStream_t st) {
  const int ld = D->grid->vert.ld;
  for (int f : fields) {
    const int kind = f >= icon_domain::FE_VN ? 1 : 0;
    for (int p = 0; p < D->nparts; ++p) {
      const int64_t nh = D->nh[kind][p];
      if (nh == 0) continue;
      k_halo_rows<<<blocks_for(nh, 8), 256, 0, st>>>(nh, ld, D->hloc[kind][p], D->hown[kind][p], D->hoidx[kind][p],
                                                      D->ptrs + (size_t)f * D->nparts, field_ptr(D->states[p], f));
    }
  }
}

// the global connectivity on the host and the owners of every entity
int host_tables(const icon_grid* grid, std::vector<int>& c2e, std::vector<int>& e2c, std::vector<int>& c2v,
                std::vector<int>& v2c, std::vector<int>& vdeg) {
  const GridDev& g = grid->g;
  int rc = copy_table_host(grid, ICON_T_C2E, c2e, 3 * g.nc);
  if (rc == ICON_OK) rc = copy_table_host(grid, ICON_T_E2C, e2c, 2 * g.ne);
  if (rc == ICON_OK) rc = copy_table_host(grid, ICON_T_C2V, c2v, 3 * g.nc);
  if (rc == ICON_OK) rc = copy_table_host(grid, ICON_T_V2C, v2c, 6 * g.nv);
  if (rc == ICON_OK) rc = copy_table_host(grid, ICON_T_VDEG, vdeg, g.nv);
  return rc;
}

void domain_release(icon_domain* D) {
  cudaStream_t st = current_stream();
  cudaStreamSynchronize(st);
  for (icon_state* s : D->states) icon_state_free(s);
  for (icon_grid* g : D->grids) {
    g->arena.release();
    delete g;
  }
  D->arena.release();
  delete D;
}

}  // namespace
}  // namespace icon

extern "C" {

int icon_partition_plan(int64_t nc, int64_t ne, int64_t nv, const int32_t* host_c2e, const int32_t* host_e2c,
                        const int32_t* host_c2v, const int32_t* host_v2c, const int32_t* host_vdeg, int nparts,
                        int part, int halo_rings, int64_t* host_counts, int32_t* host_local, int32_t* host_owner,
                        int32_t* host_owner_index) {
  using namespace icon;
  if (!host_c2e || !host_e2c || !host_c2v || !host_v2c || !host_vdeg || !host_counts || nc <= 0 || ne <= 0 ||
      nv <= 0) {
    set_error("icon_partition_plan: NULL argument or empty grid");
    return ICON_EINVAL;
  }
  if (nparts < 1 || nparts > nc || part < 0 || part >= nparts || halo_rings < 0 || halo_rings > 16) {
    set_error("icon_partition_plan: need 1 <= nparts <= Nc, 0 <= part < nparts, 0 <= halo_rings <= 16");
    return ICON_EINVAL;
  }
  GlobalOwners O;
  global_owners(nc, ne, nv, host_e2c, host_v2c, host_vdeg, nparts, O);
  PartPlan plan;
  const int rc = build_plan(nc, ne, nv, host_c2e, host_c2v, host_v2c, host_vdeg, O, nparts, part, halo_rings, plan);
  if (rc != ICON_OK) return rc;
  for (int t = 0; t < 3; ++t) {
    host_counts[t] = plan.own[t];
    host_counts[3 + t] = (int64_t)plan.g[t].size();
  }
  if (host_local) {
    size_t o = 0;
    for (int t = 0; t < 3; ++t)
      for (size_t i = 0; i < plan.g[t].size(); ++i, ++o) {
        const int gi = plan.g[t][i];
        host_local[o] = gi;
        if (host_owner) host_owner[o] = O.owner[t][gi];
        if (host_owner_index) host_owner_index[o] = O.oidx[t][gi];
      }
  }
  return ICON_OK;
}

int icon_domain_create(const icon_state* global_state, int nparts, int halo_rings, icon_domain** out) {
  using namespace icon;
  if (!global_state || !out) {
    set_error("icon_domain_create: NULL argument");
    return ICON_EINVAL;
  }
  const icon_grid* grid = global_state->grid;
  const StateDev& gs = global_state->s;
  if (gs.precision != ICON_FP64 || gs.topo.on || gs.ntr > 0 || global_state->diff4 > 0.0 ||
      global_state->upwind_theta) {
    set_error("icon_domain_create: decomposes FP64 states on flat levels without tracers, background diffusion "
              "or upwind theta");
    return ICON_EINVAL;
  }
  if (nparts < 1 || nparts > 64 || nparts > grid->g.nc || halo_rings < 3 || halo_rings > 16) {
    set_error("icon_domain_create: need 1 <= nparts <= 64 and 3 <= halo_rings <= 16 (got %d, %d)", nparts,
              halo_rings);
    return ICON_EINVAL;
  }
  cudaStream_t st = current_stream();
  std::vector<int> c2e, e2c, c2v, v2c, vdeg;
  int rc = host_tables(grid, c2e, e2c, c2v, v2c, vdeg);
  if (rc != ICON_OK) return rc;
  const GridDev& g = grid->g;
  GlobalOwners O;
  global_owners(g.nc, g.ne, g.nv, e2c.data(), v2c.data(), vdeg.data(), nparts, O);
  icon_domain* D = new icon_domain();
  D->grid = grid;
  D->nparts = nparts;
  D->rings = halo_rings;
  D->arena.al = current_allocator();
  D->plans.resize(nparts);
  for (int k = 0; k < 2; ++k) {
    D->hloc[k].assign(nparts, nullptr);
    D->hown[k].assign(nparts, nullptr);
    D->hoidx[k].assign(nparts, nullptr);
    D->nh[k].assign(nparts, 0);
  }
  const int N = grid->vert.N, ld = grid->vert.ld;
  for (int p = 0; p < nparts && rc == ICON_OK; ++p) {
    rc = build_plan(g.nc, g.ne, g.nv, c2e.data(), c2v.data(), v2c.data(), vdeg.data(), O, nparts, p, halo_rings,
                    D->plans[p]);
    if (rc != ICON_OK) break;
    icon_grid* L = new icon_grid();
    L->arena.al = current_allocator();
    D->grids.push_back(L);
    rc = build_local_grid(grid, D->plans[p], L, st);
    if (rc == ICON_ENOMEM) set_error("icon_domain_create: out of device memory (local grid %d)", p);
    if (rc != ICON_OK) break;
    // the part's state: allocated and set up on the local grid, fields from the global state
    icon_case_params cp;
    cp.noise_K = 0.0; cp.top_m = -1.0; cp.stretch_s = -1.0; cp.damp_m = -1.0; cp.precision = ICON_FP64;
    cp.member = 0; cp.topo_height_m = 0.0; cp.topo_radius_m = 0.0;
    icon_state* ps = nullptr;
    rc = icon_state_init_ex(L, 0, ICON_CASE_REST, &cp, &ps);
    if (rc != ICON_OK) break;
    D->states.push_back(ps);
    // the damping's length scale is the global grid's mean cell area
    ps->abar = global_state->abar;
    ps->divdamp4 = global_state->divdamp4;
    const PartPlan& pl = D->plans[p];
    const DeviceArena& LA = L->arena;
    (void)LA;
    int* map[2];
    for (int k = 0; k < 2; ++k) {
      map[k] = D->arena.get_n<int>(pl.g[k].size());
      if (!map[k]) { rc = ICON_ENOMEM; break; }
      ICON_CUDA(cudaMemcpyAsync(map[k], pl.g[k].data(), sizeof(int) * pl.g[k].size(), cudaMemcpyHostToDevice, st));
    }
    if (rc != ICON_OK) { set_error("icon_domain_create: out of device memory"); break; }
    const int64_t lc = (int64_t)pl.g[0].size(), le = (int64_t)pl.g[1].size();
    struct FT { double* dst; const double* src; int kind; };
    const FT fts[] = {{ps->s.vn, gs.vn, 1}, {ps->s.w, gs.w, 0}, {ps->s.rho, gs.rho, 0}, {ps->s.thv, gs.thv, 0},
                      {ps->s.ex, gs.ex, 0}};
    for (const FT& f : fts) {
      const int64_t n = f.kind ? le : lc;
      k_gather_rows<double><<<blocks_for(n * ld, 256), 256, 0, st>>>(n, ld, map[f.kind], f.src, f.dst);
    }
    // halo lists (cells, edges)
    for (int k = 0; k < 2; ++k) {
      const int64_t nh = (int64_t)pl.g[k].size() - pl.own[k];
      D->nh[k][p] = nh;
      if (nh == 0) continue;
      std::vector<int> loc(nh), own(nh), oix(nh);
      for (int64_t i = 0; i < nh; ++i) {
        const int gi = pl.g[k][pl.own[k] + i];
        loc[i] = (int)(pl.own[k] + i);
        own[i] = O.owner[k][gi];
        oix[i] = O.oidx[k][gi];
      }
      D->hloc[k][p] = D->arena.get_n<int>(nh);
      D->hown[k][p] = D->arena.get_n<int>(nh);
      D->hoidx[k][p] = D->arena.get_n<int>(nh);
      if (D->arena.failed) { rc = ICON_ENOMEM; set_error("icon_domain_create: out of device memory"); break; }
      ICON_CUDA(cudaMemcpyAsync(D->hloc[k][p], loc.data(), sizeof(int) * nh, cudaMemcpyHostToDevice, st));
      ICON_CUDA(cudaMemcpyAsync(D->hown[k][p], own.data(), sizeof(int) * nh, cudaMemcpyHostToDevice, st));
      ICON_CUDA(cudaMemcpyAsync(D->hoidx[k][p], oix.data(), sizeof(int) * nh, cudaMemcpyHostToDevice, st));
      ICON_CUDA(cudaStreamSynchronize(st));
    }
    if (rc == ICON_OK) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = cuda_fail(e, "icon_domain_create");
    }
  }
  if (rc == ICON_OK) {
    std::vector<double*> hp((size_t)icon_domain::F_COUNT * nparts);
    for (int f = 0; f < icon_domain::F_COUNT; ++f)
      for (int p = 0; p < nparts; ++p) hp[(size_t)f * nparts + p] = field_ptr(D->states[p], f);
    D->ptrs = static_cast<double**>(D->arena.get(sizeof(double*) * hp.size()));
    int64_t maxown = 0;
    for (int p = 0; p < nparts; ++p) maxown = std::max(maxown, D->plans[p].own[0]);
    D->mass_nblk = (int)((maxown + kDomMassCells - 1) / kDomMassCells);
    D->mass_part = D->arena.get_n<double>((size_t)D->mass_nblk * nparts);
    D->mass_out = D->arena.get_n<double>(nparts);
    if (D->arena.failed) {
      rc = ICON_ENOMEM;
      set_error("icon_domain_create: out of device memory");
    } else {
      cudaError_t e = cudaMemcpyAsync(D->ptrs, hp.data(), sizeof(double*) * hp.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = cuda_fail(e, "icon_domain_create");
    }
  }
  (void)N;
  if (rc != ICON_OK) {
    domain_release(D);
    return rc;
  }
  *out = D;
  return ICON_OK;
}

int icon_domain_step(icon_domain* D, double dt, int nsubsteps) {
  using namespace icon;
  if (!D || !(dt > 0.0) || nsubsteps < 1 || nsubsteps > 64) {
    set_error("icon_domain_step: bad arguments");
    return ICON_EINVAL;
  }
  cudaStream_t st = current_stream();
  for (icon_state* s : D->states) fp64_step_begin(s, dt, nsubsteps, st);
  for (int it = 0; it < nsubsteps; ++it)
    for (int stage = 0; stage < 2; ++stage) {
      const bool corr = stage == 1;
      for (icon_state* s : D->states) fp64_step_stage(s, dt, nsubsteps, corr, st);
      if (corr)
        exchange(D, {icon_domain::FE_VN, icon_domain::FC_W, icon_domain::FC_RHO, icon_domain::FC_THV,
                     icon_domain::FC_EX}, st);
      else
        exchange(D, {icon_domain::FE_VN_S, icon_domain::FC_W_S, icon_domain::FC_RHO_S, icon_domain::FC_THV_S,
                     icon_domain::FC_EX_S}, st);
    }
  for (icon_state* s : D->states) fp64_step_diffusion(s, dt, st);
  exchange(D, {icon_domain::FE_VN, icon_domain::FC_THV, icon_domain::FC_EX}, st);
  ICON_CUDA(cudaGetLastError());
  ICON_CUDA(cudaStreamSynchronize(st));
  // non-finite values in owned rows show up in the parts' status words (halo rows are
  // overwritten copies of owned rows, so they add nothing)
  int worst = ICON_OK;
  for (icon_state* s : D->states) {
    const int r = icon_state_status(s);
    if (r != ICON_OK) worst = r;
  }
  return worst;
}

int icon_domain_global_mass(icon_domain* D, double* host_out) {
  using namespace icon;
  if (!D || !host_out) {
    set_error("icon_domain_global_mass: NULL argument");
    return ICON_EINVAL;
  }
  cudaStream_t st = current_stream();
  const Vertical& v = D->grid->vert;
  for (int p = 0; p < D->nparts; ++p) {
    const int64_t own = D->plans[p].own[0];
    const int nb = (int)((own + kDomMassCells - 1) / kDomMassCells);
    double* part = D->mass_part + (size_t)p * D->mass_nblk;
    k_dom_mass_partial<<<nb, 256, 0, st>>>(own, v.N, v.ld, D->states[p]->s.rho, v.d_dz, D->grids[p]->g.A_c, part);
    k_dom_mass_final<<<1, 32, 0, st>>>(part, nb, D->mass_out + p);
  }
  std::vector<double> m(D->nparts);
  ICON_CUDA(cudaMemcpyAsync(m.data(), D->mass_out, sizeof(double) * D->nparts, cudaMemcpyDeviceToHost, st));
  ICON_CUDA(cudaStreamSynchronize(st));
  double s = 0.0;
  for (double x : m) s += x;               // the all-reduce, in part order
  *host_out = s;
  return ICON_OK;
}

int icon_domain_copy_field(icon_domain* D, int field_id, double* host_dst, size_t count) {
  using namespace icon;
  if (!D || !host_dst) {
    set_error("icon_domain_copy_field: NULL argument");
    return ICON_EINVAL;
  }
  const GridDev& g = D->grid->g;
  const int N = D->grid->vert.N;
  int kind, cols;
  switch (field_id) {
    case ICON_F_VN: case ICON_F_MFLX: kind = 1; cols = N; break;
    case ICON_F_W: case ICON_F_WFLX: kind = 0; cols = N + 1; break;
    case ICON_F_RHO: case ICON_F_THETA_V: case ICON_F_EXNER: kind = 0; cols = N; break;
    default: set_error("icon_domain_copy_field: unknown field %d", field_id); return ICON_EINVAL;
  }
  const int64_t n = kind ? g.ne : g.nc;
  if (count != (size_t)(n * cols)) {
    set_error("icon_domain_copy_field: field %d has %lld values, got %zu", field_id, (long long)(n * cols), count);
    return ICON_EINVAL;
  }
  for (int p = 0; p < D->nparts; ++p) {
    const PartPlan& pl = D->plans[p];
    const int64_t nl = (int64_t)pl.g[kind].size();
    std::vector<double> buf((size_t)nl * cols);
    const int rc = icon_state_copy_field(D->states[p], field_id, buf.data(), buf.size());
    if (rc != ICON_OK) return rc;
    for (int64_t i = 0; i < pl.own[kind]; ++i)
      std::memcpy(host_dst + (size_t)pl.g[kind][i] * cols, buf.data() + (size_t)i * cols, sizeof(double) * cols);
  }
  return ICON_OK;
}

int icon_domain_part_counts(const icon_domain* D, int part, int64_t* host_counts) {
  using namespace icon;
  if (!D || !host_counts || part < 0 || part >= D->nparts) {
    set_error("icon_domain_part_counts: bad arguments");
    return ICON_EINVAL;
  }
  for (int t = 0; t < 3; ++t) {
    host_counts[t] = D->plans[part].own[t];
    host_counts[3 + t] = (int64_t)D->plans[part].g[t].size();
  }
  return ICON_OK;
}

void icon_domain_free(icon_domain* D) {
  if (D) icon::domain_release(D);
}

}  // extern "C"
