// static_reduce.cu -- lbm_reduce_state_static: the state reduction of lbm_residual for
// callers that cannot allocate device memory.
//
// Its only scratch, the per-block partial sums, lives in the file-scope device array
// below, so a call allocates nothing. The array's name is only a host-side stand-in in
// host code; its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"
#include "kernels.cuh"

namespace {

// 65,536 blocks of 256 nodes: lattices up to 16,777,216 nodes (256^3); 2 MiB per device.
constexpr uint32_t kStaticBlocks = 65536;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_static_partials[4 * kStaticBlocks];

std::mutex g_setup_mu;
void* g_partials_addr[kMaxDevices] = {};

lbm_status fail(lbm_status st, const char* msg) {
  lbm::record_error(msg);
  return st;
}

// Device address of g_static_partials on the current device (looked up on the first
// call made with that device current).
lbm_status static_partials(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "lbm_reduce_state_static: cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_ARG, "lbm_reduce_state_static: device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess || !p) {
      char buf[256];
      snprintf(buf, sizeof buf, "lbm_reduce_state_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return fail(LBM_ERR_CUDA, buf);
    }
    g_partials_addr[dev] = p;
  }
  *out = g_partials_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" LBM_API lbm_status lbm_reduce_state_static(const void* populations, int nx, int ny, int nz,
                                                      lbm_precision prec, double rho0, void* velocity_snapshot,
                                                      double* sums, void* cuda_stream) {
  if (!populations || !velocity_snapshot || !sums)
    return fail(LBM_ERR_ARG, "lbm_reduce_state_static: a pointer argument is NULL");
  if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_ERR_ARG, "lbm_reduce_state_static: dimensions must be >= 1");
  if (prec < LBM_F64 || prec > LBM_F16_SHIFTED) return fail(LBM_ERR_ARG, "lbm_reduce_state_static: unknown precision");
  const unsigned long long n = 1ull * nx * ny * nz;
  if (n > 1ull * kStaticBlocks * lbm::SWEEP_THREADS) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "lbm_reduce_state_static: %llu nodes exceed the static scratch limit of %u nodes "
             "(use lbm_residual on a context instead)",
             n, kStaticBlocks * lbm::SWEEP_THREADS);
    return fail(LBM_ERR_ARG, buf);
  }
  void* scratch = nullptr;
  lbm_status st = static_partials(&scratch);
  if (st != LBM_OK) return st;
  const uint32_t N = uint32_t(n);
  const uint32_t blocks = lbm::sweep_blocks(N);
  double* partials = static_cast<double*>(scratch);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // Every block writes its own partial sums before the final fold reads them, so the
  // array needs no clearing between calls.
  switch (prec) {
    case LBM_F64:
      lbm::state_reduce_kernel<double><<<blocks, lbm::SWEEP_THREADS, 0, s>>>(
          static_cast<const double*>(populations), N, rho0, velocity_snapshot, partials);
      break;
    case LBM_F32:
      lbm::state_reduce_kernel<float><<<blocks, lbm::SWEEP_THREADS, 0, s>>>(
          static_cast<const float*>(populations), N, rho0, velocity_snapshot, partials);
      break;
    default:
      lbm::state_reduce_kernel<__half><<<blocks, lbm::SWEEP_THREADS, 0, s>>>(
          static_cast<const __half*>(populations), N, rho0, velocity_snapshot, partials);
      break;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = lbm::launch_final_reduce(partials, blocks, sums, s);
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof buf, "lbm_reduce_state_static: launch failed: %s", cudaGetErrorString(e));
    return fail(LBM_ERR_CUDA, buf);
  }
  return LBM_OK;
}
