// reduce.cuh -- fixed-order fold of per-block partial sums, shared by the single-lattice
// and the batched final reductions so that a lattice reduces to the same bits in both.
#pragma once
#include "lbm_internal.h"

namespace lbm {

// One block of REDUCE_THREADS folds partials[nblocks][4] into out[4]: thread t sums
// blocks t, t + REDUCE_THREADS, ... in ascending order, then a fixed pairwise tree over
// the threads. The order depends only on nblocks.
__device__ __forceinline__ void fold_partials(const double* __restrict__ partials, uint32_t nblocks,
                                              double* __restrict__ out) {
  __shared__ double s[4][REDUCE_THREADS];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t b = threadIdx.x; b < nblocks; b += REDUCE_THREADS)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] += partials[4ull * b + j];
#pragma unroll
  for (int j = 0; j < 4; ++j) s[j][threadIdx.x] = v[j];
  __syncthreads();
  for (int w = REDUCE_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int j = 0; j < 4; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = s[threadIdx.x][0];
}

}  // namespace lbm
