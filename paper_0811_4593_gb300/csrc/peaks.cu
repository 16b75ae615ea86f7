// peaks.cu -- measurement helper: the device's FP64 fused multiply-add rate.
//
// The FP64 sweep is bound by the FP64 pipe, so its roofline is the rate at which the
// device retires double-precision FMAs. The kernel keeps every resident warp busy with
// eight independent FMA chains per thread (enough to cover the pipe's latency) and is
// timed with CUDA events; the result is thread-level DFMA operations per second.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) dfma_chains_kernel(int iters, double seed, double* sink) {
  double v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 0.999999, d = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = __fma_rn(v[c], m, d);
  }
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) t += v[c];
  if (t == 123.456) sink[blockIdx.x * kThreads + threadIdx.x] = t;  // never true; keeps the chains
}

}  // namespace

extern "C" LBM_API lbm_status lbm_fp64_fma_rate(int iters, double* fma_per_s, double* ms) {
  if (iters < 1 || !fma_per_s) {
    lbm::record_error("lbm_fp64_fma_rate: iters must be >= 1 and fma_per_s non-NULL");
    return LBM_ERR_ARG;
  }
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dfma_chains_kernel, kThreads, 0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float t_ms = 0.0f;
  const int grid = sms * (per > 0 ? per : 1);
  if (e == cudaSuccess) {
    dfma_chains_kernel<<<grid, kThreads>>>(iters / 10 + 1, 1.0, nullptr);  // warm-up
    e = cudaEventRecord(e0);
    if (e == cudaSuccess) dfma_chains_kernel<<<grid, kThreads>>>(iters, 1.0, nullptr);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || t_ms <= 0.0f) {
    char buf[256];
    snprintf(buf, sizeof buf, "lbm_fp64_fma_rate: %s", cudaGetErrorString(e));
    lbm::record_error(buf);
    return LBM_ERR_CUDA;
  }
  *fma_per_s = double(grid) * kThreads * kChains * double(iters) / (double(t_ms) * 1e-3);
  if (ms) *ms = t_ms;
  return LBM_OK;
}
