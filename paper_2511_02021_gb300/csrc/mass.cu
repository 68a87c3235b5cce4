// Global air mass  M = sum_c A_c sum_k dz_ck rho_ck  in FP64 (both precision modes; dz_ck
// = dz_k on flat levels).
//
// Deterministic: a fixed launch shape assigns cells to warps in a fixed pattern,
// each warp reduces a column over levels with a fixed shuffle tree, each block
// reduces its warps in a fixed order into one partial, and a single block sums
// the partials in a fixed tree. Repeated calls on the same device give
// bit-identical results.
#include <mutex>
#include "icon_internal.h"

namespace icon {
namespace {

constexpr int kMassBlocks = 608;      // 4 x 152 SMs
constexpr int kMassThreads = 256;

__global__ void __launch_bounds__(kMassThreads) k_mass_partial(int64_t nc, int N, int ld,
                                                               const double* __restrict__ rho,
                                                               const double* __restrict__ dz,
                                                               const double* __restrict__ dzc,
                                                               const double* __restrict__ A_c,
                                                               double* __restrict__ part) {
  __shared__ double ws[kMassThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (kMassThreads / 32);
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * (kMassThreads / 32) + wid; c < nc; c += nwarps) {
    double col = 0.0;
    // dzc: each cell's own layer thickness on terrain-following levels
    if (dzc)
      for (int k = lane; k < N; k += 32) col += rho[c * ld + k] * dzc[c * ld + k];
    else
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

// level-major density [k][Nc]: one thread per column, same fixed assignment and tree
__global__ void __launch_bounds__(kMassThreads) k_mass_partial_lm(int64_t nc, int N, int ld,
                                                                  const double* __restrict__ rho,
                                                                  const double* __restrict__ dz,
                                                                  const double* __restrict__ dzc,
                                                                  const double* __restrict__ A_c,
                                                                  double* __restrict__ part) {
  __shared__ double ws[kMassThreads];
  const int64_t nthr = (int64_t)gridDim.x * kMassThreads;
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * kMassThreads + threadIdx.x; c < nc; c += nthr) {
    double col = 0.0;
    if (dzc)
      for (int k = 0; k < N; ++k) col += rho[(int64_t)k * nc + c] * dzc[c * ld + k];
    else
      for (int k = 0; k < N; ++k) col += rho[(int64_t)k * nc + c] * dz[k];
    acc += A_c[c] * col;
  }
  ws[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kMassThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) ws[threadIdx.x] += ws[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = ws[0];
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
  if (st->s.level_major)
    k_mass_partial_lm<<<kMassBlocks, kMassThreads, 0, stream>>>(grid->g.nc, grid->vert.N, grid->vert.ld, st->s.rho,
                                                                grid->vert.d_dz,
                                                                st->s.topo.on ? st->s.topo.dz_c : nullptr,
                                                                grid->g.A_c, st->s.mass_part);
  else
    k_mass_partial<<<kMassBlocks, kMassThreads, 0, stream>>>(grid->g.nc, grid->vert.N, grid->vert.ld, st->s.rho,
                                                             grid->vert.d_dz, st->s.topo.on ? st->s.topo.dz_c : nullptr,
                                                             grid->g.A_c, st->s.mass_part);
  k_mass_final<<<1, 1024, 0, stream>>>(st->s.mass_part, kMassBlocks, d_out);
  prof_end(stream);
}

}  // namespace icon

// ---------------------------------------------------------------- allocation-free variant
//
// Some callers cannot allocate device memory at all when they need the mass
// integral: a component embedded in a host model whose device memory is owned by
// that model's pool allocator, or a latency-bound loop that forbids allocations
// after start-up. For them icon_global_mass_noalloc reduces a caller-owned density
// array with its partial sums in the fixed device array below, which every GPU
// that loads this library holds until the process exits.
namespace icon {
namespace {

constexpr int kNoAllocCellsPerBlock = 1024;
constexpr int kNoAllocMaxPartials = 16384;                       // 128 KiB of partial sums
constexpr int64_t kNoAllocMaxCells = (int64_t)kNoAllocCellsPerBlock * kNoAllocMaxPartials;
constexpr int kNoAllocMaxDevices = 64;

// partial sums [0, nblk) and the result [kNoAllocMaxPartials]; shared by every call
static __device__ __align__(256) double g_mass_scratch[kNoAllocMaxPartials + 1];

// block b sums the cells [b * 1024, (b + 1) * 1024) in a fixed order; the layer thickness
// is per level (dz_lev[k], flat levels) or per cell and level (dz_cell[c * ld + k])
__global__ void __launch_bounds__(kMassThreads) k_mass_partial_blocked(int64_t nc, int N, int ld,
                                                                       const double* __restrict__ rho,
                                                                       const double* __restrict__ dz_lev,
                                                                       const double* __restrict__ dz_cell,
                                                                       const double* __restrict__ A_c,
                                                                       double* __restrict__ part) {
  __shared__ double ws[kMassThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kNoAllocCellsPerBlock;
  const int64_t c1 = c0 + kNoAllocCellsPerBlock < nc ? c0 + kNoAllocCellsPerBlock : nc;
  double acc = 0.0;
  for (int64_t c = c0 + wid; c < c1; c += kMassThreads / 32) {
    double col = 0.0;
    if (dz_cell) {
      for (int k = lane; k < N; k += 32) col += rho[c * ld + k] * dz_cell[c * ld + k];
    } else {
      for (int k = lane; k < N; k += 32) col += rho[c * ld + k] * dz_lev[k];
    }
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

// true if p is device (or managed) memory of device dev; the query allocates nothing
bool device_pointer_on(const void* p, int dev) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.device == dev;
}

std::once_flag g_noalloc_once[kNoAllocMaxDevices];
double* g_noalloc_ptr[kNoAllocMaxDevices];
cudaError_t g_noalloc_err[kNoAllocMaxDevices];

}  // namespace
}  // namespace icon

extern "C" int icon_global_mass_noalloc(const icon_grid* grid, const double* dev_rho, const double* dev_dz, int ld,
                                        double* host_out) {
  using namespace icon;
  if (!grid || !dev_rho || !host_out) {
    set_error("icon_global_mass_noalloc: NULL argument");
    return ICON_EINVAL;
  }
  const int N = grid->vert.N;
  const int64_t nc = grid->g.nc;
  if (ld < N) {
    set_error("icon_global_mass_noalloc: row stride %d is smaller than the %d levels", ld, N);
    return ICON_EINVAL;
  }
  if (nc > kNoAllocMaxCells) {
    set_error("icon_global_mass_noalloc: %lld cells exceed the maximum of %lld (fixed scratch of %d partial "
              "sums of %d cells each); use icon_global_mass", (long long)nc, (long long)kNoAllocMaxCells,
              kNoAllocMaxPartials, kNoAllocCellsPerBlock);
    return ICON_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("icon_global_mass_noalloc: device %d is beyond the %d supported devices", dev, kNoAllocMaxDevices);
    return ICON_EINVAL;
  }
  if (grid->device != dev) {
    set_error("icon_global_mass_noalloc: the grid was built on device %d but device %d is current", grid->device,
              dev);
    return ICON_EINVAL;
  }
  if (!device_pointer_on(dev_rho, dev) || (dev_dz && !device_pointer_on(dev_dz, dev))) {
    set_error("icon_global_mass_noalloc: %s is not device memory of the current device %d",
              device_pointer_on(dev_rho, dev) ? "dev_dz" : "dev_rho", dev);
    return ICON_EINVAL;
  }
  // once per device, with that device current: the device address of the scratch array
  std::call_once(g_noalloc_once[dev], [dev]() {
    g_noalloc_err[dev] = cudaGetSymbolAddress((void**)&g_noalloc_ptr[dev], g_mass_scratch);
  });
  if (g_noalloc_err[dev] != cudaSuccess) return cuda_fail(g_noalloc_err[dev], "cudaGetSymbolAddress");
  double* scratch = g_noalloc_ptr[dev];
  const int nblk = (int)((nc + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock);
  cudaStream_t stream = current_stream();
  k_mass_partial_blocked<<<nblk, kMassThreads, 0, stream>>>(nc, N, ld, dev_rho, grid->vert.d_dz, dev_dz,
                                                            grid->g.A_c, scratch);
  k_mass_final<<<1, 1024, 0, stream>>>(scratch, nblk, scratch + kNoAllocMaxPartials);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "icon_global_mass_noalloc launch");
  double h = 0.0;
  e = cudaMemcpyAsync(&h, scratch + kNoAllocMaxPartials, sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "icon_global_mass_noalloc");
  *host_out = h;
  return ICON_OK;
}
