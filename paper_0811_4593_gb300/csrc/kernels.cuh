// kernels.cuh -- fused D3Q19 sweep and its companion kernels, templated on the
// storage type S (double, float, __half). Included by one translation unit per S.
//
// In registers every population is carried shifted, h_i = f_i - w_i rho0. The
// closure and collision rules are linear in f with weights that sum to one where a
// density is formed, so they hold unchanged for h (sum_i w_i c_i = 0 and the density
// relation's weights sum to 1); the shift keeps the small deviations from rest at
// full precision in float arithmetic. FP64 storage holds f_i; FP32 and binary16
// storage hold h_i, so their rounding is relative to the small deviation from rest
// rather than to f_i itself.
#pragma once
#include <cuda_fp16.h>
#include <type_traits>
#include <utility>

#include "d3q19.cuh"
#include "lbm_internal.h"

namespace lbm {

template <int K, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (K < N) {
    f(std::integral_constant<int, K>{});
    static_for<K + 1, N>(f);
  }
}

template <typename S> struct ComputeOf { using T = float; };
template <> struct ComputeOf<double> { using T = double; };

// Storage codec: stored value <-> shifted population h in the compute type.
template <typename S> struct Codec;
template <> struct Codec<double> {
  __device__ static double load(const double* p, double shift) { return __ldg(p) - shift; }
  __device__ static double store(double h, double shift) { return h + shift; }
};
template <> struct Codec<float> {
  __device__ static float load(const float* p, float) { return __ldg(p); }
  __device__ static float store(float h, float) { return h; }
};
template <> struct Codec<__half> {
  __device__ static float load(const __half* p, float) { return __half2float(__ldg(p)); }
  __device__ static __half store(float h, float) { return __float2half_rn(h); }
};

// shift_k = w_k rho0 in the compute type, for the three weight classes
template <typename T>
struct Shifts {
  T axis, diag, rest;
  __device__ explicit Shifts(double rho0)
      : axis(T(wgt<double>(0) * rho0)), diag(T(wgt<double>(6) * rho0)), rest(T(wgt<double>(18) * rho0)) {}
  template <int k> __device__ T get() const { return k < 6 ? axis : (k < 18 ? diag : rest); }
};

// ---------------------------------------------------------------------------------
// Boundary closures on the shifted populations h (readings identical to the FP64
// oracle; see the header of each rule).
// ---------------------------------------------------------------------------------

// On-site velocity closure of a plane with inward normal SG * e_A: density from the
// in-plane populations and twice the outgoing ones (eq. uin and the appendix
// relations, formed in double), transverse corrections N on the two tangential axes
// (eqs. Nx, Ny and analogues), and for every unknown population i (c_i.n > 0)
//   h_i = h_-i + 6 w_i rho c_i.u - t_i.N     (eq. f5, eqs. f9-f17, appendix).
template <int A, int SG, typename T>
__device__ __forceinline__ void close_face(T (&h)[Q], const double (&u)[3], double rho0) {
  double s = 0.0;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int cn = SG * ca(k, A);
    if constexpr (cn == 0) s += double(h[k]);
    else if constexpr (cn < 0) s += 2.0 * double(h[k]);
  });
  // sum over the relation's weights is 1, so sum f = rho0 + sum h
  const double rho_d = (rho0 + s) / (1.0 - double(SG) * u[A]);
  const T rho = T(rho_d);
  constexpr int B = (A == 0) ? 1 : 0;
  constexpr int C = (A == 2) ? 1 : 2;
  T sb = T(0), sc = T(0);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (ca(k, A) == 0) {
      if constexpr (ca(k, B) != 0) sb += T(ca(k, B)) * h[k];
      if constexpr (ca(k, C) != 0) sc += T(ca(k, C)) * h[k];
    }
  });
  const T third = T(1) / T(3);
  const T NB = T(0.5) * sb - rho * T(u[B]) * third;
  const T NC = T(0.5) * sc - rho * T(u[C]) * third;
  const T ux = T(u[0]), uy = T(u[1]), uz = T(u[2]);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (SG * ca(k, A) > 0) {
      constexpr int m = opp(k);
      const T cu = T(cx(k)) * ux + T(cy(k)) * uy + T(cz(k)) * uz;
      const T coef = T(6 * w36(k)) / T(36);
      T t = T(0);
      if constexpr (ca(k, B) != 0) t += T(ca(k, B)) * NB;
      if constexpr (ca(k, C) != 0) t += T(ca(k, C)) * NC;
      h[k] = h[m] + coef * rho * cu - t;
    }
  });
}

// Concave no-slip edge of the planes with inward normals n1 = S1 e_A1 and
// n2 = S2 e_A2 (Sec. "On-site no-slip boundary condition"): bounce-back of every
// unknown population except the two buried links c = +-(n1 - n2); removal of the
// momentum left along e = n1 x n2, h_i -= (c_i.e) (h_{+e} - h_{-e}) / 4 (eq. edge with
// the sign that cancels the slip); buried links = (sum of the 16 other moving
// populations) / 22 and rest population = 12 times that (eq. buried).
template <int A1, int S1, int A2, int S2>
struct EdgeRule {
  static constexpr int n1x = A1 == 0 ? S1 : 0, n1y = A1 == 1 ? S1 : 0, n1z = A1 == 2 ? S1 : 0;
  static constexpr int n2x = A2 == 0 ? S2 : 0, n2y = A2 == 1 ? S2 : 0, n2z = A2 == 2 ? S2 : 0;
  static constexpr int ex = n1y * n2z - n1z * n2y, ey = n1z * n2x - n1x * n2z, ez = n1x * n2y - n1y * n2x;
  static constexpr int PE = vel_index(ex, ey, ez), ME = vel_index(-ex, -ey, -ez);
  __host__ __device__ static constexpr bool buried(int k) {
    return (cx(k) == n1x - n2x && cy(k) == n1y - n2y && cz(k) == n1z - n2z) ||
           (cx(k) == n2x - n1x && cy(k) == n2y - n1y && cz(k) == n2z - n1z);
  }
  __host__ __device__ static constexpr bool unknown(int k) { return S1 * ca(k, A1) > 0 || S2 * ca(k, A2) > 0; }
  __host__ __device__ static constexpr int along(int k) { return cx(k) * ex + cy(k) * ey + cz(k) * ez; }
};

template <int A1, int S1, int A2, int S2, typename T>
__device__ __forceinline__ void close_edge(T (&h)[Q]) {
  using R = EdgeRule<A1, S1, A2, S2>;
  static_assert(R::PE >= 0 && R::ME >= 0, "edge direction must be a lattice vector");
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int m = opp(k);
    if constexpr (R::unknown(k) && !R::buried(k)) h[k] = h[m];
  });
  const T Ne = T(0.25) * (h[R::PE] - h[R::ME]);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int ce = R::along(k);
    if constexpr (R::unknown(k) && !R::buried(k) && ce != 0) h[k] -= T(ce) * Ne;
  });
  T s = T(0);
  static_for<0, Q - 1>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (!R::buried(k)) s += h[k];
  });
  const T fb = s / T(22);
  static_for<0, Q - 1>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (R::buried(k)) h[k] = fb;
  });
  h[Q - 1] = T(12) * fb;
}

// No-slip corner with inward normals SX e_x, SY e_y, SZ e_z (eq. corner): bounce-back
// of the unknown populations that are not buried, the six buried ones
// (c.(n1+n2+n3) = 0) = (sum of the 12 other moving populations) / 18, rest
// population = 12 times that.
template <int SX, int SY, int SZ>
struct CornerRule {
  __host__ __device__ static constexpr bool buried(int k) {
    return k < Q - 1 && SX * cx(k) + SY * cy(k) + SZ * cz(k) == 0;
  }
  __host__ __device__ static constexpr bool unknown(int k) {
    return SX * cx(k) > 0 || SY * cy(k) > 0 || SZ * cz(k) > 0;
  }
};

template <int SX, int SY, int SZ, typename T>
__device__ __forceinline__ void close_corner(T (&h)[Q]) {
  using R = CornerRule<SX, SY, SZ>;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int m = opp(k);
    if constexpr (R::unknown(k) && !R::buried(k)) h[k] = h[m];
  });
  T s = T(0);
  static_for<0, Q - 1>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (!R::buried(k)) s += h[k];
  });
  const T fb = s / T(18);
  static_for<0, Q - 1>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (R::buried(k)) h[k] = fb;
  });
  h[Q - 1] = T(12) * fb;
}

// Prescribed velocity of face (A, SG) at node (x, y, z).
template <int A, int SG>
__device__ __forceinline__ void face_velocity(const SweepArgs& a, uint32_t x, uint32_t y, uint32_t z,
                                              double (&u)[3]) {
  constexpr int f = 2 * A + (SG > 0 ? 0 : 1);
  const double* tab = a.face[f].tab;
  if (tab) {
    const uint32_t t1 = (A == 0) ? y : x;
    const uint32_t t2 = (A == 2) ? y : z;
    const uint32_t n1 = (A == 0) ? a.ny : a.nx;
    const double* p = tab + 3ull * (size_t(t2) * n1 + t1);
    u[0] = __ldg(p);
    u[1] = __ldg(p + 1);
    u[2] = __ldg(p + 2);
  } else {
    u[0] = a.face[f].u[0];
    u[1] = a.face[f].u[1];
    u[2] = a.face[f].u[2];
  }
}

template <int A, int SG, typename T>
__device__ __forceinline__ void face_case(const SweepArgs& a, uint32_t x, uint32_t y, uint32_t z, T (&h)[Q]) {
  double u[3];
  face_velocity<A, SG>(a, x, y, z, u);
  close_face<A, SG>(h, u, a.rho0);
}

// code = fx + 3 fy + 9 fz with f = 0 (interior or periodic), 1 (low face), 2 (high face)
template <typename T>
__device__ __forceinline__ void apply_boundary(int code, const SweepArgs& a, uint32_t x, uint32_t y,
                                               uint32_t z, T (&h)[Q]) {
  switch (code) {
    // faces
    case 1: face_case<0, +1>(a, x, y, z, h); break;
    case 2: face_case<0, -1>(a, x, y, z, h); break;
    case 3: face_case<1, +1>(a, x, y, z, h); break;
    case 6: face_case<1, -1>(a, x, y, z, h); break;
    case 9: face_case<2, +1>(a, x, y, z, h); break;
    case 18: face_case<2, -1>(a, x, y, z, h); break;
    // x-y edges
    case 4: close_edge<0, +1, 1, +1>(h); break;
    case 5: close_edge<0, -1, 1, +1>(h); break;
    case 7: close_edge<0, +1, 1, -1>(h); break;
    case 8: close_edge<0, -1, 1, -1>(h); break;
    // x-z edges
    case 10: close_edge<0, +1, 2, +1>(h); break;
    case 11: close_edge<0, -1, 2, +1>(h); break;
    case 19: close_edge<0, +1, 2, -1>(h); break;
    case 20: close_edge<0, -1, 2, -1>(h); break;
    // y-z edges
    case 12: close_edge<1, +1, 2, +1>(h); break;
    case 15: close_edge<1, -1, 2, +1>(h); break;
    case 21: close_edge<1, +1, 2, -1>(h); break;
    case 24: close_edge<1, -1, 2, -1>(h); break;
    // corners
    case 13: close_corner<+1, +1, +1>(h); break;
    case 14: close_corner<-1, +1, +1>(h); break;
    case 16: close_corner<+1, -1, +1>(h); break;
    case 17: close_corner<-1, -1, +1>(h); break;
    case 22: close_corner<+1, +1, -1>(h); break;
    case 23: close_corner<-1, +1, -1>(h); break;
    case 25: close_corner<+1, -1, -1>(h); break;
    case 26: close_corner<-1, -1, -1>(h); break;
    default: break;
  }
}

// Density deviation, velocity, and BGK relaxation toward the second-order
// equilibrium (eq. rho, eq. vel, eq. feq, eq. bgk) on shifted populations:
//   h_i^eq = w_i (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u^2)).
template <typename T>
struct Moments {
  T drho, rho, ux, uy, uz;
};

template <typename T>
__device__ __forceinline__ Moments<T> moments(const T (&h)[Q], double rho0) {
  T d = T(0), jx = T(0), jy = T(0), jz = T(0);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    d += h[k];
    if constexpr (cx(k) != 0) jx += T(cx(k)) * h[k];
    if constexpr (cy(k) != 0) jy += T(cy(k)) * h[k];
    if constexpr (cz(k) != 0) jz += T(cz(k)) * h[k];
  });
  Moments<T> m;
  m.drho = d;
  m.rho = T(rho0) + d;
  const T inv = T(1) / m.rho;
  m.ux = jx * inv;
  m.uy = jy * inv;
  m.uz = jz * inv;
  return m;
}

template <typename T>
__device__ __forceinline__ void collide(T (&h)[Q], const Moments<T>& m, T omega) {
  const T usq15 = T(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    T cu = T(0);
    if constexpr (cx(k) != 0) cu += T(cx(k)) * m.ux;
    if constexpr (cy(k) != 0) cu += T(cy(k)) * m.uy;
    if constexpr (cz(k) != 0) cu += T(cz(k)) * m.uz;
    const T heq = wgt<T>(k) * (m.drho + m.rho * (T(3) * cu + T(4.5) * cu * cu - usq15));
    h[k] = h[k] - omega * (h[k] - heq);
  });
}

// Deterministic block sum of four doubles; thread 0 of the block gets the totals.
__device__ __forceinline__ void block_sum4(double (&v)[4], double* out) {
  __shared__ double red[SWEEP_THREADS / 32][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) red[warp][j] = v[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int w = 0; w < SWEEP_THREADS / 32; ++w)
#pragma unroll
      for (int j = 0; j < 4; ++j) t[j] += red[w][j];
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = t[j];
  }
}

// Per-node contributions to the residual reductions: mass, |u - u_snap|^2, |u|^2 and
// a bad-node flag; replaces the snapshot by the current velocity.
template <typename T>
__device__ __forceinline__ void residual_terms(const Moments<T>& m, double rho0, T* snap, uint32_t N,
                                               uint32_t cell, double (&v)[4]) {
  const double rho = rho0 + double(m.drho);
  const double u[3] = {double(m.ux), double(m.uy), double(m.uz)};
  const double p[3] = {double(snap[cell]), double(snap[N + cell]), double(snap[2ull * N + cell])};
  snap[cell] = m.ux;
  snap[N + cell] = m.uy;
  snap[2ull * N + cell] = m.uz;
  v[0] = rho;
  v[1] = (u[0] - p[0]) * (u[0] - p[0]) + (u[1] - p[1]) * (u[1] - p[1]) + (u[2] - p[2]) * (u[2] - p[2]);
  v[2] = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const bool ok = isfinite(rho) && rho > 0.0 && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
  v[3] = ok ? 0.0 : 1.0;
}

// ---------------------------------------------------------------------------------
// The fused time step: pull stream, classify, close, collide, store.
// ---------------------------------------------------------------------------------
template <typename S, bool RESID>
__global__ void __launch_bounds__(SWEEP_THREADS) sweep_kernel(const SweepArgs a) {
  using T = typename ComputeOf<S>::T;
  const uint32_t cell = blockIdx.x * SWEEP_THREADS + threadIdx.x;
  const bool active = cell < a.N;
  double red[4] = {0.0, 0.0, 0.0, 0.0};
  if (active) {
    const uint32_t q1 = fdiv(a.div_nx, cell);
    const uint32_t x = cell - q1 * a.nx;
    const uint32_t z = fdiv(a.div_ny, q1);
    const uint32_t y = q1 - z * a.ny;
    const bool px = a.periodic & 1u, py = a.periodic & 2u, pz = a.periodic & 4u;
    // pull sources: population with c_a = +1 comes from coordinate - 1, c_a = -1 from + 1;
    // outside a walled axis the index is clamped (that population is unknown and is
    // overwritten by the closure)
    const uint32_t xm = x ? x - 1 : (px ? a.nx - 1 : 0);
    const uint32_t xp = (x + 1 < a.nx) ? x + 1 : (px ? 0 : a.nx - 1);
    const uint32_t ym = y ? y - 1 : (py ? a.ny - 1 : 0);
    const uint32_t yp = (y + 1 < a.ny) ? y + 1 : (py ? 0 : a.ny - 1);
    const uint32_t zm = z ? z - 1 : (pz ? a.nz - 1 : 0);
    const uint32_t zp = (z + 1 < a.nz) ? z + 1 : (pz ? 0 : a.nz - 1);
    const S* __restrict__ src = static_cast<const S*>(a.src);
    S* __restrict__ dst = static_cast<S*>(a.dst);
    const Shifts<T> sh(a.rho0);
    T h[Q];
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const uint32_t sx = cx(k) > 0 ? xm : (cx(k) < 0 ? xp : x);
      const uint32_t sy = cy(k) > 0 ? ym : (cy(k) < 0 ? yp : y);
      const uint32_t sz = cz(k) > 0 ? zm : (cz(k) < 0 ? zp : z);
      const uint32_t idx = (sz * a.ny + sy) * a.nx + sx;
      h[k] = Codec<S>::load(src + size_t(k) * a.N + idx, sh.template get<k>());
    });
    const int fx = px ? 0 : (x == 0 ? 1 : (x == a.nx - 1 ? 2 : 0));
    const int fy = py ? 0 : (y == 0 ? 1 : (y == a.ny - 1 ? 2 : 0));
    const int fz = pz ? 0 : (z == 0 ? 1 : (z == a.nz - 1 ? 2 : 0));
    const int code = fx + 3 * fy + 9 * fz;
    if (code != 0) apply_boundary(code, a, x, y, z, h);
    const Moments<T> m = moments(h, a.rho0);
    if constexpr (RESID) residual_terms(m, a.rho0, static_cast<T*>(a.snap), a.N, cell, red);
    collide(h, m, T(a.omega));
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      dst[size_t(k) * a.N + cell] = Codec<S>::store(h[k], sh.template get<k>());
    });
  }
  if constexpr (RESID) block_sum4(red, a.partials + 4ull * blockIdx.x);
}

// Stored state -> residual terms (no streaming, no update).
template <typename S>
__global__ void __launch_bounds__(SWEEP_THREADS)
    state_reduce_kernel(const S* __restrict__ src, uint32_t N, double rho0, void* snap, double* partials) {
  using T = typename ComputeOf<S>::T;
  const uint32_t cell = blockIdx.x * SWEEP_THREADS + threadIdx.x;
  double red[4] = {0.0, 0.0, 0.0, 0.0};
  if (cell < N) {
    const Shifts<T> sh(rho0);
    T h[Q];
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      h[k] = Codec<S>::load(src + size_t(k) * N + cell, sh.template get<k>());
    });
    const Moments<T> m = moments(h, rho0);
    residual_terms(m, rho0, static_cast<T*>(snap), N, cell, red);
  }
  block_sum4(red, partials + 4ull * blockIdx.x);
}

template <typename S>
__global__ void __launch_bounds__(SWEEP_THREADS) init_kernel(S* __restrict__ dst, uint32_t N, double rho0) {
  using T = typename ComputeOf<S>::T;
  const uint32_t cell = blockIdx.x * SWEEP_THREADS + threadIdx.x;
  if (cell >= N) return;
  const Shifts<T> sh(rho0);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    dst[size_t(k) * N + cell] = Codec<S>::store(T(0), sh.template get<k>());
  });
}

template <typename S>
__global__ void __launch_bounds__(SWEEP_THREADS)
    macros_kernel(const S* __restrict__ src, uint32_t N, double rho0, typename ComputeOf<S>::T* rho,
                  typename ComputeOf<S>::T* u) {
  using T = typename ComputeOf<S>::T;
  const uint32_t cell = blockIdx.x * SWEEP_THREADS + threadIdx.x;
  if (cell >= N) return;
  const Shifts<T> sh(rho0);
  T h[Q];
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    h[k] = Codec<S>::load(src + size_t(k) * N + cell, sh.template get<k>());
  });
  const Moments<T> m = moments(h, rho0);
  if (rho) rho[cell] = m.rho;
  if (u) {
    u[cell] = m.ux;
    u[N + cell] = m.uy;
    u[2ull * N + cell] = m.uz;
  }
}

// ---------------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------------
template <typename S>
cudaError_t launch_sweep_impl(const SweepArgs& a, bool resid, cudaStream_t s) {
  const uint32_t blocks = sweep_blocks(a.N);
  if (resid) sweep_kernel<S, true><<<blocks, SWEEP_THREADS, 0, s>>>(a);
  else sweep_kernel<S, false><<<blocks, SWEEP_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_init_impl(void* dst, uint32_t N, double rho0, cudaStream_t s) {
  init_kernel<S><<<sweep_blocks(N), SWEEP_THREADS, 0, s>>>(static_cast<S*>(dst), N, rho0);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macros_impl(const void* src, uint32_t N, double rho0, void* rho, void* u, cudaStream_t s) {
  using T = typename ComputeOf<S>::T;
  macros_kernel<S><<<sweep_blocks(N), SWEEP_THREADS, 0, s>>>(static_cast<const S*>(src), N, rho0,
                                                             static_cast<T*>(rho), static_cast<T*>(u));
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_state_reduce_impl(const void* src, uint32_t N, double rho0, void* snap, double* partials,
                                     cudaStream_t s) {
  state_reduce_kernel<S><<<sweep_blocks(N), SWEEP_THREADS, 0, s>>>(static_cast<const S*>(src), N, rho0, snap,
                                                                   partials);
  return cudaGetLastError();
}

#define LBM_INSTANTIATE(S)                                                                              \
  template <> cudaError_t launch_sweep<S>(const SweepArgs& a, bool resid, cudaStream_t s) {             \
    return launch_sweep_impl<S>(a, resid, s);                                                           \
  }                                                                                                     \
  template <> cudaError_t launch_init<S>(void* dst, uint32_t N, double rho0, cudaStream_t s) {          \
    return launch_init_impl<S>(dst, N, rho0, s);                                                        \
  }                                                                                                     \
  template <> cudaError_t launch_macros<S>(const void* src, uint32_t N, double rho0, void* rho, void* u, \
                                           cudaStream_t s) {                                            \
    return launch_macros_impl<S>(src, N, rho0, rho, u, s);                                              \
  }                                                                                                     \
  template <> cudaError_t launch_state_reduce<S>(const void* src, uint32_t N, double rho0, void* snap,  \
                                                 double* partials, cudaStream_t s) {                   \
    return launch_state_reduce_impl<S>(src, N, rho0, snap, partials, s);                                \
  }

}  // namespace lbm
