// Global air mass  M = sum_c A_c sum_k dz_k rho_ck  in FP64 (both precision modes).
//
// Deterministic: a fixed launch shape assigns cells to warps in a fixed pattern,
// each warp reduces a column over levels with a fixed shuffle tree, each block
// reduces its warps in a fixed order into one partial, and a single block sums
// the partials in a fixed tree. Repeated calls on the same device give
// bit-identical results.
#include "icon_internal.h"

namespace icon {
namespace {

constexpr int kMassBlocks = 608;      // 4 x 152 SMs
constexpr int kMassThreads = 256;

__global__ void __launch_bounds__(kMassThreads) k_mass_partial(int64_t nc, int N, int ld,
                                                               const double* __restrict__ rho,
                                                               const double* __restrict__ dz,
                                                               const double* __restrict__ A_c,
                                                               double* __restrict__ part) {
  __shared__ double ws[kMassThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (kMassThreads / 32);
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * (kMassThreads / 32) + wid; c < nc; c += nwarps) {
    double col = 0.0;
    for (int k = lane; k < N; k += 32) col += rho[c * ld + k] * dz[k];
    for (int o = 16; o > 0; o >>= 1) col += __shfl_xor_sync(0xffffffffu, col, o);
    acc += A_c[c] * col;
  }
  if (lane == 0) ws[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kMassThreads / 32; ++i) s += ws[i];
    part[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(1024) k_mass_final(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

int mass_partials_count(int64_t) { return kMassBlocks; }

void enqueue_mass(const icon_state* st, double* d_out, cudaStream_t stream) {
  const icon_grid* grid = st->grid;
  prof_begin(stream, K_MASS);
  k_mass_partial<<<kMassBlocks, kMassThreads, 0, stream>>>(grid->g.nc, grid->vert.N, grid->vert.ld, st->s.rho,
                                                           grid->vert.d_dz, grid->g.A_c, st->s.mass_part);
  k_mass_final<<<1, 1024, 0, stream>>>(st->s.mass_part, kMassBlocks, d_out);
  prof_end(stream);
}

}  // namespace icon
