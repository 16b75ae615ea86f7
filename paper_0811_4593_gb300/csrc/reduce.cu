// reduce.cu -- final reduction of one lattice's per-block partial sums.
#include "reduce.cuh"

namespace lbm {

__global__ void __launch_bounds__(REDUCE_THREADS)
    final_reduce_kernel(const double* __restrict__ partials, uint32_t nblocks, double* __restrict__ out) {
  fold_partials(partials, nblocks, out);
}

cudaError_t launch_final_reduce(const double* partials, uint32_t nblocks, double* out, cudaStream_t s) {
  final_reduce_kernel<<<1, REDUCE_THREADS, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

// Final reduction of every lattice of a batch: block i folds entry i's partials into
// results[slot][4]; blocks past the entries in use return at once.
__global__ void __launch_bounds__(REDUCE_THREADS)
    batch_final_reduce_kernel(const BatchHeader* __restrict__ hdr, const BatchEntry* __restrict__ ents,
                              double* __restrict__ results) {
  if (blockIdx.x >= hdr->nentries) return;
  const BatchEntry& e = ents[blockIdx.x];
  fold_partials(e.a.partials, e.nblocks, results + 4ull * e.slot);
}

cudaError_t launch_batch_final_reduce(const BatchHeader* hdr, const BatchEntry* ents, int capacity, double* results,
                                      cudaStream_t s) {
  batch_final_reduce_kernel<<<capacity, REDUCE_THREADS, 0, s>>>(hdr, ents, results);
  return cudaGetLastError();
}

}  // namespace lbm
