// Measured FP64 instruction throughput of the current GPU.
//
// The FP64 step and the FP64 parts of the mixed step are bound by the rate at which
// the GPU issues FP64 instructions; the roofline of those kernels divides by this
// measured rate. Each thread runs eight independent dependency chains of FP64
// fused multiply-adds (or adds), enough to keep the FP64 pipe busy; the grid holds
// 16 blocks of 256 threads per SM. The rate counts instructions: a fused multiply-add
// is one.
#include "icon_internal.h"

namespace icon {
namespace {

constexpr int kProbeChains = 8;

template <bool FMA>
__global__ void __launch_bounds__(256) k_probe_fp64(int iters, double m, double c, double* out) {
  double a[kProbeChains];
  for (int i = 0; i < kProbeChains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = FMA ? fma(a[i], m, c) : a[i] + c;
  }
  double s = 0.0;
  for (int i = 0; i < kProbeChains; ++i) s += a[i];
  if (s == -1.0) out[0] = s;   // never true; keeps the chains alive
}

template <bool FMA>
int probe_rate(int sms, double* dev_out, cudaStream_t st, double* rate) {
  const int blocks = sms * 16, threads = 256, iters = 4096;
  cudaEvent_t e0, e1;
  ICON_CUDA(cudaEventCreate(&e0));
  ICON_CUDA(cudaEventCreate(&e1));
  k_probe_fp64<FMA><<<blocks, threads, 0, st>>>(iters / 8, 0.9999999, 1e-9, dev_out);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, st);
    k_probe_fp64<FMA><<<blocks, threads, 0, st>>>(iters, 0.9999999, 1e-9, dev_out);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ICON_CUDA(cudaGetLastError());
  const double instr = (double)blocks * threads * iters * kProbeChains;
  *rate = instr / (best * 1e-3);
  return ICON_OK;
}

}  // namespace
}  // namespace icon

extern "C" int icon_probe_fp64_rate(double* fma_per_s, double* add_per_s) {
  using namespace icon;
  if (!fma_per_s || !add_per_s) {
    set_error("icon_probe_fp64_rate: NULL argument");
    return ICON_EINVAL;
  }
  int dev = 0;
  ICON_CUDA(cudaGetDevice(&dev));
  int sms = 0;
  ICON_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* d = nullptr;
  ICON_CUDA(cudaMalloc(&d, sizeof(double)));
  cudaStream_t st = current_stream();
  double f = 0.0, a = 0.0;
  int rc = probe_rate<true>(sms, d, st, &f);
  if (rc == ICON_OK) rc = probe_rate<false>(sms, d, st, &a);
  cudaFree(d);
  if (rc != ICON_OK) return rc;
  *fma_per_s = f;
  *add_per_s = a;
  return ICON_OK;
}
