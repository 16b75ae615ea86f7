// lbm_internal.h -- interface between the C-ABI runtime (runtime.cu) and the kernel
// translation units (sweep_f64.cu, sweep_f32.cu, sweep_f16.cu).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace lbm {

// Unsigned 32-bit division by an invariant divisor with one multiply-high, after
// Granlund & Montgomery, "Division by invariant integers using multiplication"
// (PLDI 1994), Fig. 4.1: q = (t + ((n - t) >> s1)) >> s2 with t = mulhi(m, n).
struct FastDiv {
  uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;  // l = ceil(log2 d)
  FastDiv f;
  f.d = d;
  f.m = uint32_t(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fdiv(const FastDiv& f, uint32_t n) {
  uint32_t t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}
#endif

// One boundary-face node as the sweep reads it. Velocity face: the prescribed velocity
// in double and float, and 1 / (1 - u.n) for the density relation (n = inward normal),
// formed in double on the host. Pressure face: the tangential velocity (normal part
// zero) in double and float, and the prescribed density in `inv`.
struct __align__(16) FaceNode {
  double u[3];
  double inv;
  float uf[3];
  float pad;
};

// Boundary data of one face for the sweep.
struct FaceBC {
  const FaceNode* tab;  // device [n2][n1] or nullptr (uniform: `uni`)
  FaceNode uni;
};

// Everything one sweep launch needs, passed by value.
struct SweepArgs {
  const void* src;   // storage [19][N], post-collision state of the previous step
  void* dst;         // storage [19][N], post-collision state after this step
  const void* src_pop[19];  // src + k N: the start of population k (set with src / dst
  void* dst_pop[19];        // so that each access is one add and one wide multiply-add)
  uint32_t nx, ny, nz, N;
  FastDiv div_nx, div_ny;
  FastDiv div_nxh;    // nx / 2 (the paired binary16 sweep, even nx)
  uint32_t periodic;  // bit a set: axis a is periodic
  uint32_t pressure;  // bit f set: face f is a pressure face
  double rho0;
  double omega;       // 1 / tau
  float rho0f, omegaf;
  float mom_coef[2][2];  // omegaf / 6 and omegaf / 12 as hi + lo float pairs
  FaceBC face[6];
  void* snap;         // residual steps: [3][N] velocity snapshot in the compute type
  double* partials;   // residual steps: [blocks][4] per-block sums
  const uint32_t* links;  // optional [N] geometry words (nullptr: no geometry), see below
  uint32_t forced;        // nonzero: a body force acts (eq. gravity)
  double force[3];        // F: momentum the collision adds per step
  double tforce[3];       // tau F: the equilibrium velocity shift times rho
  float forcef[3], tforcef[3];
  // Device word a sweep sets (bit 0) when it gave up waiting for its staged loads (a
  // bounded wait ran out); the host reads and clears it at its synchronisation points.
  uint32_t* err;
  // Failure injection for tests of the bounded waits: nonzero makes the row-staged
  // sweep's first CTA announce the copies of its first row group but not issue them,
  // so its waits run out (no fault, no unbounded wait).
  uint32_t drop_copies;
};

// Error bits of SweepArgs::err.
constexpr uint32_t ERR_STAGE_WAIT = 1u;

// Geometry word of a node: bits 0..18 (nodes without a rule): the pull source of
// population k is solid (mid-grid bounce-back); bits 24..29: the node's on-site rule
// (0: none; 1..50: the C ABI codes of planes, concave edges, corners and junctions;
// 51..62: the convex edges -7..-18 as 44 - code); bit 31: the node is solid.
constexpr uint32_t SOLID_NODE = 1u << 31;
constexpr int RULE_SHIFT = 24;
constexpr uint32_t RULE_BITS = 0x3fu;

// One lattice of a batch, as the batched sweep reads it from device memory.
struct BatchEntry {
  SweepArgs a;           // src/dst are taken from buf[] and the step parity
  const void* buf[2];    // the lattice's two population buffers
  uint32_t cur;          // index into buf[] of the current state at step parity 0
  uint32_t block_begin;  // first global block of this lattice in the batch
  uint32_t nblocks;      // 256-node blocks of this lattice
  uint32_t slot;         // row of the batch's result table
};

struct BatchHeader {
  uint32_t nentries;      // entries in use, ordered by block_begin
  uint32_t total_blocks;  // sum of nblocks
  uint32_t nchunks;       // work units of the batched sweep (chunk table rows - 1)
  uint32_t pad;
};

// One work unit of the batched sweep: the global blocks from `start` up to the next
// chunk's start, the first of them in entry `entry`. The table ends with a sentinel
// row {total_blocks, nentries}. CTAs take chunks in order from a device counter, so
// a CTA that met expensive blocks (boundary-heavy lattices) takes fewer chunks.
struct BatchChunk {
  uint32_t start;
  uint32_t entry;
};

constexpr int SWEEP_THREADS = 256;
constexpr int REDUCE_THREADS = 1024;

inline uint32_t sweep_blocks(uint32_t N) { return (N + SWEEP_THREADS - 1) / SWEEP_THREADS; }

// mode: 0 A/B pull, 1 AA gather-scatter step, 2 AA in-place step (see kernels.cuh)
template <typename S> cudaError_t launch_sweep(const SweepArgs& a, bool resid, int mode, cudaStream_t s);
template <typename S> cudaError_t launch_init(void* dst, uint32_t N, double rho0, cudaStream_t s);
// swapped: the state holds f_k in slot -k (an AA lattice between step pairs)
template <typename S> cudaError_t launch_macros(const void* src, uint32_t N, double rho0, void* rho,
                                                void* u, bool swapped, cudaStream_t s);
template <typename S> cudaError_t launch_state_reduce(const void* src, uint32_t N, double rho0,
                                                      void* snap, double* partials, bool swapped, cudaStream_t s);
cudaError_t launch_final_reduce(const double* partials, uint32_t nblocks, double* out, cudaStream_t s);
// next_chunk: a device counter that is zero when the launch starts (the caller clears
// it in stream order before every launch); each CTA draws chunks from it until the
// table is exhausted
template <typename S> cudaError_t launch_sweep_batched(const BatchHeader* hdr, const BatchEntry* ents,
                                                       const BatchChunk* chunks, uint32_t* next_chunk, uint32_t parity,
                                                       bool resid, int mode, int grid, cudaStream_t s);
// persistent grid of a batched variant: SMs x its resident blocks per SM (0 on error)
template <typename S> int batched_grid(bool resid, int mode);
template <typename S> uint32_t bounds_errors();  // debug build: indices out of range (read resets)
cudaError_t launch_batch_final_reduce(const BatchHeader* hdr, const BatchEntry* ents, int capacity, double* results,
                                      cudaStream_t s);

// Sets the calling thread's context-free error message (lbm_last_error(NULL)).
void record_error(const char* msg);

}  // namespace lbm
