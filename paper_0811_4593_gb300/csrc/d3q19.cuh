// d3q19.cuh -- compile-time D3Q19 lattice for the CUDA sweep.
//
// c_1..c_19 are the columns of the paper's matrix M (eq. deffs); population i lives
// at index k = i-1. Each component is packed two bits per population (value + 1) so
// that every query folds to a constant inside fully unrolled loops.
#pragma once
#include <cstdint>

namespace lbm {

constexpr int Q = 19;

__host__ __device__ constexpr int cx(int k) { return int((0x15500aa552ull >> (2 * k)) & 3ull) - 1; }
__host__ __device__ constexpr int cy(int k) { return int((0x10a5252525ull >> (2 * k)) & 3ull) - 1; }
__host__ __device__ constexpr int cz(int k) { return int((0x1222525255ull >> (2 * k)) & 3ull) - 1; }
__host__ __device__ constexpr int ca(int k, int a) { return a == 0 ? cx(k) : (a == 1 ? cy(k) : cz(k)); }

// index of the population with c = -c_k
__host__ __device__ constexpr int opp(int k) {
  int r = -1;
  for (int m = 0; m < Q; ++m)
    if (cx(m) == -cx(k) && cy(m) == -cy(k) && cz(m) == -cz(k)) r = m;
  return r;
}

// index of the population with c = (x, y, z), or -1
__host__ __device__ constexpr int vel_index(int x, int y, int z) {
  int r = -1;
  for (int m = 0; m < Q; ++m)
    if (cx(m) == x && cy(m) == y && cz(m) == z) r = m;
  return r;
}

// lattice weights (eq. weights) as multiples of 1/36
__host__ __device__ constexpr int w36(int k) { return k < 6 ? 2 : (k < 18 ? 1 : 12); }

template <typename T>
__host__ __device__ constexpr T wgt(int k) { return T(w36(k)) / T(36); }

// Axis (0, 1, 2) and sign of the axis vector c_k (k < 6).
__host__ __device__ constexpr int axis_of(int k) { return cx(k) != 0 ? 0 : (cy(k) != 0 ? 1 : 2); }
__host__ __device__ constexpr int sign_of(int k) { return cx(k) + cy(k) + cz(k); }

// The diagonal with index j (0..3, in increasing population index) among the twelve
// diagonals perpendicular to the axis vector c_p: the bulk normal of junction codes.
__host__ __device__ constexpr int junction_diagonal(int p, int j) {
  int seen = 0, r = -1;
  for (int k = 6; k < 18; ++k)
    if (cx(k) * cx(p) + cy(k) * cy(p) + cz(k) * cz(p) == 0) {
      if (seen == j) r = k;
      ++seen;
    }
  return r;
}

}  // namespace lbm
