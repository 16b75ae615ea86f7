// kernels.cuh -- fused D3Q19 sweep and its companion kernels, templated on the
// storage type S (double, float, __half). Included by one translation unit per S.
//
// FP32 and binary16 storage hold the shifted populations h_i = f_i - w_i rho0 and the
// sweep carries them shifted in registers, so float rounding is relative to the small
// deviation from rest rather than to f_i. The closure and collision rules hold
// unchanged for h (sum_i w_i c_i = 0, and the weights of the density relation sum to
// one), with every density written as rho0 + (sum of h). FP64 storage holds f_i itself;
// the same code runs on it with the reference density 0 (then "sum of h" is rho), which
// spares the FP64 pipe the 38 shift additions per node.
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

// Arithmetic with one explicit rounding per operation. The compiler may neither fuse
// nor reorder these, so every sweep variant (single node, paired, residual, batched,
// AA, geometry) computes the same bits for a node; a plain a * b + c may be fused in one
// kernel and not in another.
__device__ __forceinline__ float op_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double op_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float op_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double op_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float op_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double op_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float op_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double op_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Two FP32 values as one operand of the packed FP32 instructions (PTX add, sub, mul and
// fma with the .rn.f32x2 type, sm_100 and later): lane x belongs to node A of a pair,
// lane y to node B. Every lane is one IEEE single-precision operation rounded to
// nearest, exactly as the scalar op_* functions round, so code written once over T
// gives the same bits per node for T = float and T = f32x2 with half the arithmetic
// instructions for the pair.
struct f32x2 {
  float x, y;
  f32x2() = default;
  __host__ __device__ constexpr f32x2(float v) : x(v), y(v) {}
  __host__ __device__ constexpr f32x2(double v) : x(float(v)), y(float(v)) {}
  __host__ __device__ constexpr f32x2(int v) : x(float(v)), y(float(v)) {}
  __host__ __device__ constexpr f32x2(float a, float b) : x(a), y(b) {}
};
__device__ __forceinline__ unsigned long long pk(f32x2 v) {
  return static_cast<unsigned long long>(__float_as_uint(v.x)) |
         (static_cast<unsigned long long>(__float_as_uint(v.y)) << 32);
}
__device__ __forceinline__ f32x2 upk(unsigned long long d) {
  return f32x2(__uint_as_float(static_cast<unsigned>(d)), __uint_as_float(static_cast<unsigned>(d >> 32)));
}
__device__ __forceinline__ f32x2 op_add(f32x2 a, f32x2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
__device__ __forceinline__ f32x2 op_sub(f32x2 a, f32x2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
__device__ __forceinline__ f32x2 op_mul(f32x2 a, f32x2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
__device__ __forceinline__ f32x2 op_fma(f32x2 a, f32x2 b, f32x2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
  return upk(d);
}
__device__ __forceinline__ f32x2 operator-(f32x2 a) { return f32x2(-a.x, -a.y); }
// per-lane IEEE division, as the scalar a / b
__device__ __forceinline__ f32x2 operator/(f32x2 a, f32x2 b) { return f32x2(a.x / b.x, a.y / b.y); }

// The scalar type of one lane (float for f32x2).
template <typename T> struct LaneOf { using type = T; };
template <> struct LaneOf<f32x2> { using type = float; };

// Index checks of the debug build (LBM_DEBUG_BOUNDS): an index at or beyond its limit
// is counted in this translation unit's error word and replaced by 0, so the access
// stays inside the buffer; lbm_debug_bounds_errors reads the count. The release build
// compiles the check away.
#ifdef LBM_DEBUG_BOUNDS
static __device__ unsigned int g_bounds_errors;
__device__ __forceinline__ uint32_t chk(uint32_t i, uint32_t limit) {
  if (i < limit) return i;
  atomicAdd(&g_bounds_errors, 1u);
  return 0u;
}
#else
__device__ __forceinline__ uint32_t chk(uint32_t i, uint32_t) { return i; }
#endif

// Signed sums whose first term is taken as it is (negation is exact), so that no
// rounded addition of zero is ever issued.
template <int SGN, typename T>
__device__ __forceinline__ T sgn(T v) { return SGN > 0 ? v : -v; }
template <int SGN, typename T>
__device__ __forceinline__ void acc(T& s, T v, bool first) {
  if (first) s = sgn<SGN>(v);
  else s = SGN > 0 ? op_add(s, v) : op_sub(s, v);
}
// c_k . (x, y, z) for a moving population k
template <int k, typename T>
__device__ __forceinline__ T dot_c(T x, T y, T z) {
  constexpr int X = cx(k), Y = cy(k), Z = cz(k);
  T s = T(0);
  if constexpr (X != 0) acc<X>(s, x, true);
  if constexpr (Y != 0) acc<Y>(s, y, X == 0);
  if constexpr (Z != 0) acc<Z>(s, z, X == 0 && Y == 0);
  return s;
}
// first population index lying in the plane normal to axis A with component X != 0
template <int A>
__host__ __device__ constexpr int first_in_plane(int X) {
  for (int k = 0; k < Q; ++k)
    if (ca(k, A) == 0 && ca(k, X) != 0) return k;
  return -1;
}
// first population index with component a of sign `sg` (0: component zero)
__host__ __device__ constexpr int first_with(int a, int sg) {
  for (int k = 0; k < Q; ++k) {
    const int c = ca(k, a);
    if ((sg > 0 && c > 0) || (sg < 0 && c < 0) || (sg == 0 && c == 0)) return k;
  }
  return -1;
}
__host__ __device__ constexpr int first_nonzero(int a) {
  for (int k = 0; k < Q; ++k)
    if (ca(k, a) != 0) return k;
  return -1;
}

// Storage codec: stored value <-> register value v (h_i for shifted storage, f_i for
// FP64) in the compute type.
template <typename S> struct Storage;
template <> struct Storage<double> {
  static constexpr bool shifted = false;
  __device__ static double load(const double* p) { return __ldg(p); }
  __device__ static double store(double v) { return v; }
};
// FP32 loads are read-only loads that also ask L2 to fetch the enclosing 256-byte block
// (PTX ld.global.nc with the .L2::256B prefetch-size qualifier): consecutive warps read
// consecutive 128-byte pieces of each population row. Measured: the single-lattice
// sweep unchanged, the batched sweep on a serving mix 1 - 2 % faster.
template <> struct Storage<float> {
  static constexpr bool shifted = true;
  __device__ static float load(const float* p) {
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
  }
  __device__ static float store(float v) { return v; }
};
template <> struct Storage<__half> {
  static constexpr bool shifted = true;
  __device__ static float load(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static __half store(float v) { return __float2half_rn(v); }
};

// Population load of a sweep step: the A/B step reads through the storage codec (for
// FP32 with the L2 prefetch hint); the AA steps read plain read-only loads (with the
// hint the FP32 AA steps, which write the array they read, measured 2.6 % slower).
template <typename S, int MODE>
__device__ __forceinline__ typename std::conditional<std::is_same<S, double>::value, double, float>::type
load_pop(const S* p) {
  if constexpr (MODE != 0 && std::is_same<S, float>::value) return __ldg(p);
  else return Storage<S>::load(p);
}

// The reference density the register values are shifted by: rho0, or 0 for FP64.
template <typename S>
__device__ __forceinline__ double ref_rho(double rho0) { return Storage<S>::shifted ? rho0 : 0.0; }

// ---------------------------------------------------------------------------------
// Boundary closures on the shifted populations h (readings identical to the FP64
// oracle; see the header of each rule).
// ---------------------------------------------------------------------------------

// Error-free accumulation of a float sum as hi + lo (Knuth's TwoSum); the rounded
// intrinsics keep the compiler from contracting or reassociating the steps.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float t) {
  const float s = __fadd_rn(hi, t);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// Velocity of a face node in the compute type, and 1 / (1 - u.n) in double.
template <typename T>
struct FaceVals {
  T u[3];
  double inv;
};

// The relation's sum over the shifted populations of a plane with inward normal
// SG * e_A: in-plane populations once, outgoing ones twice (its weights sum to 1, so
// the plane's density relation reads rho (1 - u.n) = ref + S). FP64: accumulated in
// double. Float sweeps: accumulated as a float pair hi + lo with TwoSum, which is
// exact except for the float rounding of lo's own sum of the 14 error terms; that
// leaves an error below about 14^2 2^-48 (~7e-13) of the largest partial sum, against
// 14 2^-53 (~2e-15) for accumulation in double -- both far below the float rounding of
// the populations, and the pair costs no FP64 work on the face nodes until the final
// conversion.
template <int A, int SG, typename T>
__device__ __forceinline__ double relation_sum(const T (&h)[Q]) {
  if constexpr (std::is_same<T, double>::value) {
    double S = 0.0;
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int cn = SG * ca(k, A);
      if constexpr (cn == 0) S += h[k];
      else if constexpr (cn < 0) S += 2.0 * h[k];
    });
    return S;
  } else {
    float hi = 0.0f, lo = 0.0f;
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      constexpr int cn = SG * ca(k, A);
      if constexpr (cn == 0) two_sum_acc(hi, lo, h[k]);
      else if constexpr (cn < 0) two_sum_acc(hi, lo, __fmul_rn(2.0f, h[k]));
    });
    return double(hi) + double(lo);
  }
}

// Unknown populations of a plane with inward normal SG * e_A, given the node's density
// rho and velocity u: transverse corrections N on the two tangential axes (eqs. Nx, Ny
// and analogues) and, for every unknown i (c_i.n > 0),
//   h_i = h_-i + 6 w_i rho c_i.u - t_i.N     (eq. f5, eqs. f9-f17, appendix).
template <int A, int SG, typename T>
__device__ __forceinline__ void fill_unknowns(T (&h)[Q], T rho, const T (&u)[3]) {
  constexpr int B = (A == 0) ? 1 : 0;
  constexpr int C = (A == 2) ? 1 : 2;
  T sb = T(0), sc = T(0);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (ca(k, A) == 0) {
      if constexpr (ca(k, B) != 0) acc<ca(k, B)>(sb, h[k], k == first_in_plane<A>(B));
      if constexpr (ca(k, C) != 0) acc<ca(k, C)>(sc, h[k], k == first_in_plane<A>(C));
    }
  });
  const T third = T(1) / T(3);
  const T NB = op_sub(op_mul(T(0.5), sb), op_mul(op_mul(rho, u[B]), third));
  const T NC = op_sub(op_mul(T(0.5), sc), op_mul(op_mul(rho, u[C]), third));
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (SG * ca(k, A) > 0) {
      constexpr int m = opp(k);
      const T cu = dot_c<k>(u[0], u[1], u[2]);
      const T coef = T(6 * w36(k)) / T(36);
      const T hk = op_fma(op_mul(coef, rho), cu, h[m]);
      // minus the transverse correction t_i.N
      if constexpr (ca(k, B) != 0 && ca(k, C) != 0) {
        T t = T(0);
        acc<ca(k, B)>(t, NB, true);
        acc<ca(k, C)>(t, NC, false);
        h[k] = op_sub(hk, t);
      } else if constexpr (ca(k, B) != 0) {
        h[k] = ca(k, B) > 0 ? op_sub(hk, NB) : op_add(hk, NB);
      } else if constexpr (ca(k, C) != 0) {
        h[k] = ca(k, C) > 0 ? op_sub(hk, NC) : op_add(hk, NC);
      } else {
        h[k] = hk;
      }
    }
  });
}

// On-site velocity closure (eq. uin and the appendix relations): the density
// rho = (ref + S) / (1 - u.n), formed in double (fv.inv = 1 / (1 - u.n) from the host),
// then the unknown populations.
template <int A, int SG, typename T>
__device__ __forceinline__ void close_face(T (&h)[Q], const FaceVals<T>& fv, double ref) {
  const T rho = T((ref + relation_sum<A, SG>(h)) * fv.inv);
  fill_unknowns<A, SG>(h, rho, fv.u);
}

// Pressure variant (eq. rhoin and the appendix relations): the density rho_p
// (fv.inv) and the tangential velocity are prescribed; the normal velocity
// u.n = 1 - (ref + S) / rho_p, formed in double; then the unknown populations.
template <int A, int SG, typename T>
__device__ __forceinline__ void close_face_pressure(T (&h)[Q], const FaceVals<T>& fv, double ref) {
  const double rho_p = fv.inv;
  const double un = 1.0 - (ref + relation_sum<A, SG>(h)) / rho_p;
  T u[3] = {fv.u[0], fv.u[1], fv.u[2]};
  u[A] = T(double(SG) * un);
  fill_unknowns<A, SG>(h, T(rho_p), u);
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

// Next to a pressure plane (pressure = true) the buried links and the rest population
// instead make the node density the prescribed one (eq. buried_rho): with drho_p the
// prescribed density minus the reference, buried = (drho_p - sum of the 16) / 14.
template <int A1, int S1, int A2, int S2, typename T>
__device__ __forceinline__ void close_edge(T (&h)[Q], bool pressure, T drho_p) {
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
  const T fb = pressure ? (drho_p - s) / T(14) : s / T(22);
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

// Next to a pressure plane: buried = (drho_p - sum of the 12) / 18 (the corner variant,
// prescribed density rho_p, drho_p = rho_p - reference).
template <int SX, int SY, int SZ, typename T>
__device__ __forceinline__ void close_corner(T (&h)[Q], bool pressure, T drho_p) {
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
  const T fb = pressure ? (drho_p - s) / T(18) : s / T(18);
  static_for<0, Q - 1>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (R::buried(k)) h[k] = fb;
  });
  h[Q - 1] = T(12) * fb;
}

// Prescribed velocity of face (A, SG) at node (x, y, z): from the face's node table
// when it has one, else the face's uniform value.
template <int A, int SG, typename T>
__device__ __forceinline__ FaceVals<T> face_values(const SweepArgs& a, uint32_t x, uint32_t y, uint32_t z) {
  constexpr int f = 2 * A + (SG > 0 ? 0 : 1);
  const FaceBC& fb = a.face[f];
  FaceVals<T> v;
  if (fb.tab) {
    const uint32_t t1 = (A == 0) ? y : x;
    const uint32_t t2 = (A == 2) ? y : z;
    const uint32_t n1 = (A == 0) ? a.ny : a.nx;
    const uint32_t n2 = (A == 2) ? a.ny : a.nz;
    const FaceNode* p = fb.tab + chk(t2 * n1 + t1, n1 * n2);
    if constexpr (std::is_same<T, double>::value) {
      const double2 a0 = __ldg(reinterpret_cast<const double2*>(p));
      const double2 a1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
      v.u[0] = a0.x;
      v.u[1] = a0.y;
      v.u[2] = a1.x;
      v.inv = a1.y;
    } else {
      const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 2);
      v.u[0] = b.x;
      v.u[1] = b.y;
      v.u[2] = b.z;
      v.inv = __ldg(&p->inv);
    }
  } else {
    if constexpr (std::is_same<T, double>::value) {
      v.u[0] = fb.uni.u[0];
      v.u[1] = fb.uni.u[1];
      v.u[2] = fb.uni.u[2];
    } else {
      v.u[0] = fb.uni.uf[0];
      v.u[1] = fb.uni.uf[1];
      v.u[2] = fb.uni.uf[2];
    }
    v.inv = fb.uni.inv;
  }
  return v;
}

// Reference density of the register values: 0 for FP64 (unshifted), rho0 otherwise.
template <typename T>
__device__ __forceinline__ double ref_density(const SweepArgs& a) {
  return std::is_same<T, double>::value ? 0.0 : a.rho0;
}

template <int A, int SG>
constexpr int face_id() { return 2 * A + (SG > 0 ? 0 : 1); }

template <int A, int SG, typename T>
__device__ __forceinline__ void face_case(const SweepArgs& a, uint32_t x, uint32_t y, uint32_t z, T (&h)[Q]) {
  const FaceVals<T> fv = face_values<A, SG, T>(a, x, y, z);
  if (a.pressure & (1u << face_id<A, SG>())) close_face_pressure<A, SG>(h, fv, ref_density<T>(a));
  else close_face<A, SG>(h, fv, ref_density<T>(a));
}

// Edge of faces (A1, S1) and (A2, S2); when one of them is a pressure face its density
// at the node fixes the node's density.
template <int A1, int S1, int A2, int S2, typename T>
__device__ __forceinline__ void edge_case(const SweepArgs& a, uint32_t x, uint32_t y, uint32_t z, T (&h)[Q]) {
  constexpr uint32_t b1 = 1u << face_id<A1, S1>(), b2 = 1u << face_id<A2, S2>();
  if (a.pressure & (b1 | b2)) {
    const double rp = (a.pressure & b1) ? face_values<A1, S1, T>(a, x, y, z).inv : face_values<A2, S2, T>(a, x, y, z).inv;
    close_edge<A1, S1, A2, S2>(h, true, T(rp - ref_density<T>(a)));
  } else {
    close_edge<A1, S1, A2, S2>(h, false, T(0));
  }
}

template <int SX, int SY, int SZ, typename T>
__device__ __forceinline__ void corner_case(const SweepArgs& a, uint32_t x, uint32_t y, uint32_t z, T (&h)[Q]) {
  constexpr uint32_t bx = 1u << face_id<0, SX>(), by = 1u << face_id<1, SY>(), bz = 1u << face_id<2, SZ>();
  if (a.pressure & (bx | by | bz)) {
    const double rp = (a.pressure & bx)   ? face_values<0, SX, T>(a, x, y, z).inv
                      : (a.pressure & by) ? face_values<1, SY, T>(a, x, y, z).inv
                                          : face_values<2, SZ, T>(a, x, y, z).inv;
    close_corner<SX, SY, SZ>(h, true, T(rp - ref_density<T>(a)));
  } else {
    close_corner<SX, SY, SZ>(h, false, T(0));
  }
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
    case 4: edge_case<0, +1, 1, +1>(a, x, y, z, h); break;
    case 5: edge_case<0, -1, 1, +1>(a, x, y, z, h); break;
    case 7: edge_case<0, +1, 1, -1>(a, x, y, z, h); break;
    case 8: edge_case<0, -1, 1, -1>(a, x, y, z, h); break;
    // x-z edges
    case 10: edge_case<0, +1, 2, +1>(a, x, y, z, h); break;
    case 11: edge_case<0, -1, 2, +1>(a, x, y, z, h); break;
    case 19: edge_case<0, +1, 2, -1>(a, x, y, z, h); break;
    case 20: edge_case<0, -1, 2, -1>(a, x, y, z, h); break;
    // y-z edges
    case 12: edge_case<1, +1, 2, +1>(a, x, y, z, h); break;
    case 15: edge_case<1, -1, 2, +1>(a, x, y, z, h); break;
    case 21: edge_case<1, +1, 2, -1>(a, x, y, z, h); break;
    case 24: edge_case<1, -1, 2, -1>(a, x, y, z, h); break;
    // corners
    case 13: corner_case<+1, +1, +1>(a, x, y, z, h); break;
    case 14: corner_case<-1, +1, +1>(a, x, y, z, h); break;
    case 16: corner_case<+1, -1, +1>(a, x, y, z, h); break;
    case 17: corner_case<-1, -1, +1>(a, x, y, z, h); break;
    case 22: corner_case<+1, +1, -1>(a, x, y, z, h); break;
    case 23: corner_case<-1, +1, -1>(a, x, y, z, h); break;
    case 25: corner_case<+1, -1, -1>(a, x, y, z, h); break;
    case 26: corner_case<-1, -1, -1>(a, x, y, z, h); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------------
// On-site rules of a general geometry (Sec. "On-site no-slip boundary condition",
// complex geometries): every wall is at rest.
// ---------------------------------------------------------------------------------

// Convex edge with bulk normal d = (DX, DY, DZ) (a diagonal: the sum of the two plane
// normals) and edge direction e = n1 x n2 (eq. edge2): the population coming from the
// solid side, c = d, is bounced back; then 1/4 (c_i.e) sum_j h_j (c_j.e) is subtracted
// from every population travelling into the bulk (c_i.d > 0), which removes all
// momentum along the edge (four of them have c_i.e = +-1).
template <int DX, int DY, int DZ>
struct ConvexRule {
  static constexpr int n1x = DX != 0 ? DX : 0, n1y = DX == 0 ? DY : 0, n1z = 0;
  static constexpr int n2x = 0, n2y = DX != 0 ? DY : 0, n2z = DZ;
  static constexpr int ex = n1y * n2z - n1z * n2y, ey = n1z * n2x - n1x * n2z, ez = n1x * n2y - n1y * n2x;
  static constexpr int KD = vel_index(DX, DY, DZ);
  __host__ __device__ static constexpr int along(int k) { return cx(k) * ex + cy(k) * ey + cz(k) * ez; }
  __host__ __device__ static constexpr int into_bulk(int k) { return cx(k) * DX + cy(k) * DY + cz(k) * DZ > 0; }
};

template <int DX, int DY, int DZ, typename T>
__device__ __forceinline__ void close_convex(T (&h)[Q]) {
  using R = ConvexRule<DX, DY, DZ>;
  static_assert(R::KD >= 0 && R::ex * R::ex + R::ey * R::ey + R::ez * R::ez == 1, "diagonal bulk normal");
  h[R::KD] = h[opp(R::KD)];
  T P = T(0);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (R::along(k) != 0) P += T(R::along(k)) * h[k];
  });
  const T q = T(0.25) * P;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (R::into_bulk(k) && R::along(k) != 0) h[k] -= T(R::along(k)) * q;
  });
}

// Convex edge with bulk normal d = (DX, DY, DZ) meeting the plane with inward normal
// SG e_A: bounce-back of the populations coming through the plane (SG c_A > 0) or from
// the edge's solid side (c = d); rest population = 12/36 of the node density, i.e. one
// half of the moving populations (the sum of shifted populations obeys the same
// relation, since the weights of the moving populations add up to 24/36).
template <int A, int SG, int DX, int DY, int DZ, typename T>
__device__ __forceinline__ void close_junction(T (&h)[Q]) {
  constexpr int KD = vel_index(DX, DY, DZ);
  static_assert(KD >= 0, "diagonal bulk normal");
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (SG * ca(k, A) > 0 || k == KD) h[k] = h[opp(k)];
  });
  T s = T(0);
  static_for<0, Q - 1>([&](auto kc) { s += h[decltype(kc)::value]; });
  h[Q - 1] = T(0.5) * s;
}


// Rule R of the geometry word (see SOLID_NODE): R = 1..6 planes c_R, 7..18 concave
// edges with bulk normal c_R, 19..26 corners, 27..50 junctions, 51..62 convex edges
// with bulk normal c_(R-44).
template <int R, typename T>
__device__ __forceinline__ void rule_case(T (&h)[Q], double ref) {
  if constexpr (R >= 1 && R <= 6) {
    constexpr int k = R - 1;
    const FaceVals<T> rest = {{T(0), T(0), T(0)}, 1.0};
    close_face<axis_of(k), sign_of(k)>(h, rest, ref);
  } else if constexpr (R >= 7 && R <= 18) {
    constexpr int k = R - 1;
    constexpr int A1 = cx(k) != 0 ? 0 : 1;
    constexpr int S1 = A1 == 0 ? cx(k) : cy(k);
    constexpr int A2 = cz(k) != 0 ? 2 : 1;
    constexpr int S2 = A2 == 2 ? cz(k) : cy(k);
    close_edge<A1, S1, A2, S2>(h, false, T(0));
  } else if constexpr (R >= 19 && R <= 26) {
    constexpr int b = R - 19;
    close_corner<(b & 1) ? -1 : 1, (b & 2) ? -1 : 1, (b & 4) ? -1 : 1>(h, false, T(0));
  } else if constexpr (R >= 27 && R <= 50) {
    constexpr int p = (R - 27) / 4;
    constexpr int d = junction_diagonal(p, (R - 27) % 4);
    close_junction<axis_of(p), sign_of(p), cx(d), cy(d), cz(d)>(h);
  } else if constexpr (R >= 51 && R <= 62) {
    constexpr int k = R - 45;
    close_convex<cx(k), cy(k), cz(k)>(h);
  }
}

template <int LO, int HI, typename T>
__device__ __forceinline__ void apply_rule(uint32_t r, T (&h)[Q], double ref) {
  if constexpr (LO == HI) {
    rule_case<LO>(h, ref);
  } else {
    constexpr int MID = (LO + HI) / 2;
    if (r <= uint32_t(MID)) apply_rule<LO, MID>(r, h, ref);
    else apply_rule<MID + 1, HI>(r, h, ref);
  }
}

// Density deviation, velocity, and BGK relaxation toward the second-order
// equilibrium (eq. rho, eq. vel, eq. feq, eq. bgk) on shifted populations:
//   h_i^eq = w_i (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u^2)).
template <typename T>
struct Moments {
  T drho, rho, jx, jy, jz, ux, uy, uz;  // drho = sum of v; rho = ref + drho; j = rho u
  T inv;                                // 1 / rho
};

template <typename T>
__device__ __forceinline__ Moments<T> moments(const T (&h)[Q], T rho0) {
  // the populations with c_x = +1, -1 and 0 are summed apart, so that the density and
  // the x momentum share the three partial sums (37 additions instead of 45)
  T sp = T(0), sm = T(0), s0 = T(0), jy = T(0), jz = T(0);
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (cx(k) > 0) acc<1>(sp, h[k], k == first_with(0, 1));
    else if constexpr (cx(k) < 0) acc<1>(sm, h[k], k == first_with(0, -1));
    else acc<1>(s0, h[k], k == first_with(0, 0));
    if constexpr (cy(k) != 0) acc<cy(k)>(jy, h[k], k == first_nonzero(1));
    if constexpr (cz(k) != 0) acc<cz(k)>(jz, h[k], k == first_nonzero(2));
  });
  Moments<T> m;
  m.drho = op_add(op_add(sp, sm), s0);
  m.rho = op_add(rho0, m.drho);
  m.jx = op_sub(sp, sm);
  m.jy = jy;
  m.jz = jz;
  const T inv = T(1) / m.rho;
  m.inv = inv;
  m.ux = op_mul(m.jx, inv);
  m.uy = op_mul(jy, inv);
  m.uz = op_mul(jz, inv);
  return m;
}

// Moments with compensated sums (FP32 storage with a geometry or a body force): each
// of the five partial sums runs as a TwoSum float pair, and density and momenta are
// rounded to float once, from the pairs, so they carry about half an ulp of error
// instead of up to one per term. In a steady flow these roundings repeat every step
// and integrate over the relaxation time (a 32^3 body-force Poiseuille at tau = 2
// relaxes over ~190 steps), so the exact sums reduce the float error of such flows.
__device__ __forceinline__ Moments<float> moments_compensated(const float (&h)[Q], float rho0) {
  float sp = 0.0f, spl = 0.0f, sm = 0.0f, sml = 0.0f, s0 = 0.0f, s0l = 0.0f;
  float jy = 0.0f, jyl = 0.0f, jz = 0.0f, jzl = 0.0f;
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (cx(k) > 0) two_sum_acc(sp, spl, h[k]);
    else if constexpr (cx(k) < 0) two_sum_acc(sm, sml, h[k]);
    else two_sum_acc(s0, s0l, h[k]);
    if constexpr (cy(k) != 0) two_sum_acc(jy, jyl, cy(k) > 0 ? h[k] : -h[k]);
    if constexpr (cz(k) != 0) two_sum_acc(jz, jzl, cz(k) > 0 ? h[k] : -h[k]);
  });
  Moments<float> m;
  float d = sp, dl = __fadd_rn(__fadd_rn(spl, sml), s0l);
  two_sum_acc(d, dl, sm);
  two_sum_acc(d, dl, s0);
  m.drho = __fadd_rn(d, dl);
  float x = sp, xl = __fsub_rn(spl, sml);
  two_sum_acc(x, xl, -sm);
  m.jx = __fadd_rn(x, xl);
  m.jy = __fadd_rn(jy, jyl);
  m.jz = __fadd_rn(jz, jzl);
  m.rho = __fadd_rn(rho0, m.drho);
  const float inv = 1.0f / m.rho;
  m.inv = inv;
  m.ux = __fmul_rn(m.jx, inv);
  m.uy = __fmul_rn(m.jy, inv);
  m.uz = __fmul_rn(m.jz, inv);
  return m;
}

// EXACT_MOMENTUM: the momentum term 3 omega w_i (c_i.j) takes its coefficient as an
// unevaluated pair hi + lo (coef, from the host), so the collision conserves momentum
// to float rounding of each product instead of biasing it by the rounding of one
// constant -- a bias that acts like a small body force and dominated the FP32 error at
// low viscosity (4.6e-5 of u_max on a 256 x 64 x 64 duct at tau = 0.6, 7.6e-6 with
// the pair). Used for FP32 storage; binary16 storage error is set by its 11-bit
// mantissa.
//
// BGK relaxation v_i <- (1 - omega) v_i + omega v_i^eq with the second-order
// equilibrium written for the pair (i, -i), whose c.u only changes sign:
//   v^eq_{+-i} = w_i (b + s_i +- a_i),  b = drho - 3/2 j.u,  s_i = 9/2 (c_i.j)(c_i.u),
//   a_i = 3 c_i.j
// (j = rho u), which equals w_i (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u^2)) (eq. feq)
// term by term and shares the symmetric part between the two populations. omega w_i is
// folded into the per-class factors. The FP64 sweep, bound by the FP64 pipe, writes the
// quadratic term as the momentum term A_i = 3 omega w_i (c_i.j) times c_i.u' with
// u' = 3/2 u (omega w_i s_i = A_i (c_i.u'), b = drho - j.u'), one multiply fewer per
// pair; the float sweeps, bound by memory, keep g_i (c_i.j)(c_i.u) with
// g_i = 9/2 omega w_i, which measured marginally faster there.
// The binary16 sweeps (no coefficient pair) also run on packed pairs of nodes (f32x2),
// whose multiplies the assembler was measured to fuse with a following add or subtract
// although both are written with round-to-nearest; so there no product feeds an add:
// c_i.u is formed as (c_i.j) / rho, and the momentum term enters the populations through
// fused multiply-adds, v^eq_{+-i} part = fma(+-3 omega w_i, c_i.j, t_i).
template <bool EXACT_MOMENTUM = false, typename T>
__device__ __forceinline__ void collide(T (&h)[Q], const Moments<T>& m, T omega,
                                        const float (*coef)[2] = nullptr) {
  constexpr bool VFORM = std::is_same<T, double>::value;
  T vx = m.ux, vy = m.uy, vz = m.uz;
  if constexpr (VFORM) {
    vx = op_mul(T(1.5), m.ux);
    vy = op_mul(T(1.5), m.uy);
    vz = op_mul(T(1.5), m.uz);
  }
  const T jv = op_fma(m.jz, vz, op_fma(m.jy, vy, op_mul(m.jx, vx)));
  T b;
  if constexpr (VFORM) b = op_sub(m.drho, jv);
  else b = op_fma(T(-1.5), jv, m.drho);
  const T keep = op_sub(T(1), omega);
  using L = typename LaneOf<T>::type;
  const T ow_axis = op_mul(omega, T(wgt<L>(0))), ow_diag = op_mul(omega, T(wgt<L>(6)));
  const T ob_axis = op_mul(ow_axis, b), ob_diag = op_mul(ow_diag, b);
  const T g_axis = op_mul(T(4.5), ow_axis), g_diag = op_mul(T(4.5), ow_diag);
  const T a_axis = op_mul(T(3), ow_axis), a_diag = op_mul(T(3), ow_diag);
  const T na_axis = -a_axis, na_diag = -a_diag;  // exact
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int o = opp(k);
    if constexpr (k == Q - 1) {
      h[k] = op_fma(keep, h[k], op_mul(op_mul(omega, T(wgt<L>(k))), b));
    } else if constexpr (k < o) {
      constexpr bool axis = w36(k) == 2;
      const T cj = dot_c<k>(m.jx, m.jy, m.jz);
      if constexpr (VFORM || EXACT_MOMENTUM) {
        const T cv = dot_c<k>(vx, vy, vz);
        T a;
        if constexpr (EXACT_MOMENTUM) {
          const float* ab = coef[axis ? 0 : 1];
          a = op_fma(T(ab[0]), cj, op_mul(T(ab[1]), cj));
        } else {
          a = op_mul(axis ? a_axis : a_diag, cj);
        }
        T t;
        if constexpr (VFORM) t = op_fma(a, cv, axis ? ob_axis : ob_diag);
        else t = op_fma(op_mul(axis ? g_axis : g_diag, cj), cv, axis ? ob_axis : ob_diag);
        h[k] = op_fma(keep, h[k], op_add(t, a));
        h[o] = op_fma(keep, h[o], op_sub(t, a));
      } else {
        const T cv = op_mul(cj, m.inv);
        const T t = op_fma(op_mul(axis ? g_axis : g_diag, cj), cv, axis ? ob_axis : ob_diag);
        h[k] = op_fma(keep, h[k], op_fma(axis ? a_axis : a_diag, cj, t));
        h[o] = op_fma(keep, h[o], op_fma(axis ? na_axis : na_diag, cj, t));
      }
    }
  });
}

// Launch parameters in the compute type (no per-node double-to-float conversion);
// rho0_of is the reference density of the register values (0 for FP64 storage).
template <typename T> __device__ __forceinline__ T rho0_of(const SweepArgs& a);
template <> __device__ __forceinline__ double rho0_of<double>(const SweepArgs&) { return 0.0; }
template <> __device__ __forceinline__ float rho0_of<float>(const SweepArgs& a) { return a.rho0f; }
template <typename T> __device__ __forceinline__ T omega_of(const SweepArgs& a);
template <> __device__ __forceinline__ double omega_of<double>(const SweepArgs& a) { return a.omega; }
template <> __device__ __forceinline__ float omega_of<float>(const SweepArgs& a) { return a.omegaf; }
template <typename T> __device__ __forceinline__ T force_of(const SweepArgs& a, int i);
template <> __device__ __forceinline__ double force_of<double>(const SweepArgs& a, int i) { return a.force[i]; }
template <> __device__ __forceinline__ float force_of<float>(const SweepArgs& a, int i) { return a.forcef[i]; }
template <typename T> __device__ __forceinline__ T tforce_of(const SweepArgs& a, int i);
template <> __device__ __forceinline__ double tforce_of<double>(const SweepArgs& a, int i) { return a.tforce[i]; }
template <> __device__ __forceinline__ float tforce_of<float>(const SweepArgs& a, int i) { return a.tforcef[i]; }

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
  const double d0 = op_sub(u[0], p[0]), d1 = op_sub(u[1], p[1]), d2 = op_sub(u[2], p[2]);
  v[1] = op_fma(d2, d2, op_fma(d1, d1, op_mul(d0, d0)));
  v[2] = op_fma(u[2], u[2], op_fma(u[1], u[1], op_mul(u[0], u[0])));
  const bool ok = isfinite(rho) && rho > 0.0 && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
  v[3] = ok ? 0.0 : 1.0;
}

// ---------------------------------------------------------------------------------
// The fused time step: pull stream, classify, close, collide, store.
// ---------------------------------------------------------------------------------
enum StreamMode : int { STREAM_AB = 0, STREAM_AA_GATHER = 1, STREAM_AA_LOCAL = 2 };
// Block `blk` (nodes blk*256 .. blk*256+255) of the lattice described by `a`, with the
// streaming scheme MODE:
//   STREAM_AB         pull f_i(x) = src_i(x - c_i), store dst_i(x)          (two arrays)
//   STREAM_AA_GATHER  read slot -i of node x - c_i, write f*_i back to slot i of node
//                     x + c_i -- the location the read of -i came from   (one array)
//   STREAM_AA_LOCAL   read slot i of node x, write f*_i to slot -i of node x (one array)
// The two AA steps alternate starting from a state that holds f*_i(x) in slot -i of
// node x (the "swapped" state); after the gather step the array holds the streamed
// populations in natural slots, after the local step the swapped post-collision state
// again. Each node reads and writes the same 19 locations, so one array suffices.
// GEOM: the lattice may have a geometry (solid nodes, on-site rules) and a body force;
// the plain variant reads neither.
template <typename S, bool RESID, int MODE, bool GEOM = false>
__device__ __forceinline__ void sweep_block(const SweepArgs& a, uint32_t blk) {
  using T = typename ComputeOf<S>::T;
  const uint32_t cell = blk * SWEEP_THREADS + threadIdx.x;
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
    // node the population k is pulled from (x - c_k); for STREAM_AA_GATHER also the node
    // f*_{-k} is pushed to
    auto pull_idx = [&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const uint32_t sx = cx(k) > 0 ? xm : (cx(k) < 0 ? xp : x);
      const uint32_t sy = cy(k) > 0 ? ym : (cy(k) < 0 ? yp : y);
      const uint32_t sz = cz(k) > 0 ? zm : (cz(k) < 0 ? zp : z);
      return chk((sz * a.ny + sy) * a.nx + sx, a.N);
    };
    // geometry word (A/B lattices with a geometry only; 0 everywhere else)
    uint32_t lm = 0u;
    if constexpr (GEOM) lm = a.links ? __ldg(a.links + chk(cell, a.N)) : 0u;
    T h[Q];
    if (!GEOM || (lm & ~(RULE_BITS << RULE_SHIFT)) == 0u) {
      static_for<0, Q>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (MODE == STREAM_AB) {
          h[k] = Storage<S>::load(static_cast<const S*>(a.src_pop[k]) + pull_idx(kc));
        } else if constexpr (MODE == STREAM_AA_GATHER) {
          h[k] = load_pop<S, MODE>(static_cast<const S*>(a.src_pop[opp(k)]) + pull_idx(kc));
        } else {
          h[k] = load_pop<S, MODE>(static_cast<const S*>(a.src_pop[k]) + cell);
        }
      });
    } else {
      // a solid node keeps its populations; next to a solid node the population that
      // would come from it is the node's own population -k reversed (mid-grid
      // bounce-back, Sec. "Boundary conditions")
      static_for<0, Q>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const bool own = (lm & SOLID_NODE) != 0u;
        const bool back = (lm >> k) & 1u;
        const S* p = own ? static_cast<const S*>(a.src_pop[k]) + cell
                         : (back ? static_cast<const S*>(a.src_pop[opp(k)]) + cell
                                 : static_cast<const S*>(a.src_pop[k]) + pull_idx(kc));
        h[k] = Storage<S>::load(p);
      });
    }
    const bool solid = (lm & SOLID_NODE) != 0u;
    const uint32_t rule = (lm >> RULE_SHIFT) & RULE_BITS;
    const int fx = px ? 0 : (x == 0 ? 1 : (x == a.nx - 1 ? 2 : 0));
    const int fy = py ? 0 : (y == 0 ? 1 : (y == a.ny - 1 ? 2 : 0));
    const int fz = pz ? 0 : (z == 0 ? 1 : (z == a.nz - 1 ? 2 : 0));
    const int code = fx + 3 * fy + 9 * fz;
    if constexpr (GEOM) {
      if (rule != 0u) apply_rule<1, 62>(rule, h, ref_density<T>(a));
      else if (code != 0 && !solid) apply_boundary(code, a, x, y, z, h);
    } else {
      if (code != 0) apply_boundary(code, a, x, y, z, h);
    }
    Moments<T> m;
    if constexpr (GEOM && std::is_same<S, float>::value) m = moments_compensated(h, rho0_of<T>(a));
    else m = moments(h, rho0_of<T>(a));
    if constexpr (GEOM) {
      if (a.forced && !solid) {
        // eq. gravity: the collision relaxes toward the equilibrium at u + tau F / rho
        // and so adds F to the momentum; the residual sees the stored velocity
        const T inv = T(1) / m.rho;
        if constexpr (RESID) {
          Moments<T> mp = m;
          mp.jx += force_of<T>(a, 0);
          mp.jy += force_of<T>(a, 1);
          mp.jz += force_of<T>(a, 2);
          mp.ux = mp.jx * inv;
          mp.uy = mp.jy * inv;
          mp.uz = mp.jz * inv;
          residual_terms(mp, ref_rho<S>(a.rho0), static_cast<T*>(a.snap), a.N, cell, red);
        }
        m.jx += tforce_of<T>(a, 0);
        m.jy += tforce_of<T>(a, 1);
        m.jz += tforce_of<T>(a, 2);
        m.ux = m.jx * inv;
        m.uy = m.jy * inv;
        m.uz = m.jz * inv;
      } else if constexpr (RESID) {
        residual_terms(m, ref_rho<S>(a.rho0), static_cast<T*>(a.snap), a.N, cell, red);
      }
    } else if constexpr (RESID) {
      residual_terms(m, ref_rho<S>(a.rho0), static_cast<T*>(a.snap), a.N, cell, red);
    }
    if (!solid) collide<std::is_same<S, float>::value>(h, m, omega_of<T>(a), a.mom_coef);
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (MODE == STREAM_AB) {
        static_cast<S*>(a.dst_pop[k])[cell] = Storage<S>::store(h[k]);
      } else if constexpr (MODE == STREAM_AA_LOCAL) {
        static_cast<S*>(a.dst_pop[opp(k)])[cell] = Storage<S>::store(h[k]);
      } else {
        // push f*_k to node x + c_k = the pull source of -k; a target outside a walled
        // axis does not exist (the population leaves the domain)
        constexpr int o = opp(k);
        const bool inside = code == 0 || !((fx == 1 && cx(o) > 0) || (fx == 2 && cx(o) < 0) ||
                                           (fy == 1 && cy(o) > 0) || (fy == 2 && cy(o) < 0) ||
                                           (fz == 1 && cz(o) > 0) || (fz == 2 && cz(o) < 0));
        if (inside) static_cast<S*>(a.dst_pop[k])[pull_idx(std::integral_constant<int, o>{})] = Storage<S>::store(h[k]);
      }
    });
  }
  if constexpr (RESID) block_sum4(red, a.partials + 4ull * blk);
}

// Resident 256-thread blocks per SM each sweep variant is compiled for (the register
// budget is 65536 / (256 * blocks)). The float sweeps are memory-bound and need many
// warps in flight to hide DRAM latency: 6 blocks (<= 42 registers) for the plain step,
// single-lattice or batched (the batched kernel at 4 blocks served 14 % fewer jobs per
// second; its spills are in the geometry path, which serving lattices do not take); the
// residual variant carries the reduction and gets 5. The FP64 sweeps are bound by the
// FP64 pipe and get room for their double registers.
// The AA gather-scatter step also keeps its push targets and takes 2 blocks fewer, the
// AA in-place step one fewer.
// The general-geometry variant (GEOM) carries the rule dispatch and the force and is
// compiled for 4 blocks (2 for FP64).
template <typename S, bool RESID, bool BATCHED, int MODE, bool GEOM = false>
struct SweepOccupancy {
  static constexpr int base = RESID ? 5 : 6;
  static constexpr int blocks = GEOM ? 4 : (MODE == 1 ? (base > 4 ? 4 : base - 1) : (MODE == 2 ? (base > 5 ? 5 : base) : base));
};
template <bool RESID, bool BATCHED, int MODE, bool GEOM>
struct SweepOccupancy<double, RESID, BATCHED, MODE, GEOM> {
  static constexpr int blocks = (RESID && BATCHED) || MODE == 1 || GEOM ? 2 : 3;
};

template <typename S, bool RESID, int MODE, bool GEOM>
__global__ void __launch_bounds__(SWEEP_THREADS, (SweepOccupancy<S, RESID, false, MODE, GEOM>::blocks))
    sweep_kernel(const __grid_constant__ SweepArgs a) {
  sweep_block<S, RESID, MODE, GEOM>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------------
// Paired binary16 sweep: the plain A/B step (no residual, no geometry, no force) of a
// binary16 lattice with even nx, two neighbouring nodes (x0, x0 + 1), x0 even, per
// thread. The binary16 sweep moves half the bytes of the float one for the same
// arithmetic and is bound by instruction issue; pairing halves the index and address
// work per node: a population with c_x = 0 is read as one aligned half2 for both
// nodes, one with c_x != 0 as two halves, and the two results of a population are
// stored as one half2. Each node runs the single-node sweep's closure,
// moment and collision code, so both sweeps give the same bits.
// ---------------------------------------------------------------------------------
// Read-only loads that also ask L2 to fetch the enclosing 256-byte block (PTX
// ld.global.nc with the .L2::256B prefetch-size qualifier): consecutive warps stream
// consecutive 128-byte pieces of each population row, so the next warp's data is
// already on its way when it asks.
__device__ __forceinline__ float ld_half_l2(const __half* p) {
  unsigned short v;
  asm("ld.global.nc.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return __half2float(__ushort_as_half(v));
}
__device__ __forceinline__ void ld_half2_l2(const __half* p, float& lo, float& hi) {
  unsigned int v;
  asm("ld.global.nc.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(p));
  lo = __half2float(__ushort_as_half(static_cast<unsigned short>(v & 0xffffu)));
  hi = __half2float(__ushort_as_half(static_cast<unsigned short>(v >> 16)));
}

// Populations of both nodes of a pair. Node A = x0 pulls c_x = +1 populations from
// xam (x0 - 1, or the wrap / clamp at the row start), node B = x0 + 1 pulls c_x = -1
// populations from xbp (x0 + 2, or the wrap / clamp at the row end). One code path for
// every pair: splitting off the row ends as a separate branch cost 9 % (both branches
// ran in the warps holding a row end, and the larger body took registers).
// MODE STREAM_AA_GATHER reads slot -k of the source node instead of slot k.
template <int MODE>
__device__ __forceinline__ void load_pair(const SweepArgs& a, uint32_t x0, uint32_t xam, uint32_t xbp,
                                          const uint32_t (&rows)[3][3], f32x2 (&h)[Q]) {
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    constexpr int slot = MODE == STREAM_AA_GATHER ? opp(k) : k;
    const __half* base = static_cast<const __half*>(a.src_pop[slot]);
    const uint32_t row = rows[1 - cz(k)][1 - cy(k)];
    if constexpr (cx(k) == 0) {
      ld_half2_l2(base + chk(row + x0, a.N - 1), h[k].x, h[k].y);
    } else if constexpr (cx(k) > 0) {  // pulled from x - 1
      h[k].y = ld_half_l2(base + chk(row + x0, a.N));
      h[k].x = ld_half_l2(base + chk(row + xam, a.N));
    } else {  // pulled from x + 1
      h[k].x = ld_half_l2(base + chk(row + x0 + 1, a.N));
      h[k].y = ld_half_l2(base + chk(row + xbp, a.N));
    }
  });
}

// Boundary closure of one node of a pair (LANE 0: node A, 1: node B) on its scalar
// populations.
template <int LANE>
__device__ __forceinline__ void close_lane(int code, const SweepArgs& a, uint32_t x, uint32_t y, uint32_t z,
                                           f32x2 (&h)[Q]) {
  float t[Q];
  static_for<0, Q>([&](auto kc) { t[decltype(kc)::value] = LANE ? h[decltype(kc)::value].y : h[decltype(kc)::value].x; });
  apply_boundary(code, a, x, y, z, t);
  static_for<0, Q>([&](auto kc) {
    if (LANE) h[decltype(kc)::value].y = t[decltype(kc)::value];
    else h[decltype(kc)::value].x = t[decltype(kc)::value];
  });
}

// MODE: STREAM_AB (pull from the other array), STREAM_AA_GATHER (read slot -k of node
// x - c_k, write f*_k to slot k of node x + c_k) or STREAM_AA_LOCAL (read and write the
// pair's own slots, k and -k exchanged), as in the single-node sweep.
template <typename S, int MODE>
__global__ void __launch_bounds__(SWEEP_THREADS, 4) sweep_pair_kernel(const __grid_constant__ SweepArgs a) {
  static_assert(std::is_same<S, __half>::value, "the paired sweep is for binary16 storage");
  const uint32_t pair = blockIdx.x * SWEEP_THREADS + threadIdx.x;
  if (pair >= (a.N >> 1)) return;
  const uint32_t q1 = fdiv(a.div_nxh, pair);
  const uint32_t x0 = 2u * (pair - q1 * (a.nx >> 1));
  const uint32_t z = fdiv(a.div_ny, q1);
  const uint32_t y = q1 - z * a.ny;
  const uint32_t cell = q1 * a.nx + x0;
  const bool px = a.periodic & 1u, py = a.periodic & 2u, pz = a.periodic & 4u;
  const uint32_t ym = y ? y - 1 : (py ? a.ny - 1 : 0);
  const uint32_t yp = (y + 1 < a.ny) ? y + 1 : (py ? 0 : a.ny - 1);
  const uint32_t zm = z ? z - 1 : (pz ? a.nz - 1 : 0);
  const uint32_t zp = (z + 1 < a.nz) ? z + 1 : (pz ? 0 : a.nz - 1);
  // rows[1 - c_z][1 - c_y]: start of the row a population is pulled from;
  // rows[1 + c_z][1 + c_y]: the row the AA gather step pushes it to
  const uint32_t zs[3] = {zm, z, zp}, ys[3] = {ym, y, yp};
  uint32_t rows[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) rows[i][j] = (zs[i] * a.ny + ys[j]) * a.nx;
  // source x of node A for c_x = +1 and of node B for c_x = -1 (clamped outside a
  // walled axis: those populations are unknown and overwritten by the closure)
  const uint32_t xam = x0 ? x0 - 1 : (px ? a.nx - 1 : 0);
  const uint32_t xbp = (x0 + 2 < a.nx) ? x0 + 2 : (px ? 0 : a.nx - 1);
  f32x2 h[Q];
  if constexpr (MODE == STREAM_AA_LOCAL) {
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      ld_half2_l2(static_cast<const __half*>(a.src_pop[k]) + chk(cell, a.N - 1), h[k].x, h[k].y);
    });
  } else {
    load_pair<MODE>(a, x0, xam, xbp, rows, h);
  }
  const int fxA = px ? 0 : (x0 == 0 ? 1 : 0);
  const int fxB = px ? 0 : (x0 + 1 == a.nx - 1 ? 2 : 0);
  const int fy = py ? 0 : (y == 0 ? 1 : (y == a.ny - 1 ? 2 : 0));
  const int fz = pz ? 0 : (z == 0 ? 1 : (z == a.nz - 1 ? 2 : 0));
  const int codeA = fxA + 3 * fy + 9 * fz;
  const int codeB = fxB + 3 * fy + 9 * fz;
  if (codeA != 0) close_lane<0>(codeA, a, x0, y, z, h);
  if (codeB != 0) close_lane<1>(codeB, a, x0 + 1, y, z, h);
  // moments and collision of both nodes at once, in packed FP32
  const Moments<f32x2> m = moments(h, f32x2(a.rho0f));
  collide(h, m, f32x2(a.omegaf));
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if constexpr (MODE == STREAM_AB) {
      *reinterpret_cast<__half2*>(static_cast<__half*>(a.dst_pop[k]) + chk(cell, a.N - 1)) =
          __floats2half2_rn(h[k].x, h[k].y);
    } else if constexpr (MODE == STREAM_AA_LOCAL) {
      *reinterpret_cast<__half2*>(static_cast<__half*>(a.dst_pop[opp(k)]) + chk(cell, a.N - 1)) =
          __floats2half2_rn(h[k].x, h[k].y);
    } else {
      // push f*_k to slot k of node x + c_k; a target beyond a walled face does not exist
      const bool in_yz = !((fy == 1 && cy(k) < 0) || (fy == 2 && cy(k) > 0) || (fz == 1 && cz(k) < 0) ||
                           (fz == 2 && cz(k) > 0));
      if (in_yz) {
        __half* pop = static_cast<__half*>(a.dst_pop[k]);
        const uint32_t row = rows[1 + cz(k)][1 + cy(k)];
        if constexpr (cx(k) == 0) {
          *reinterpret_cast<__half2*>(pop + chk(row + x0, a.N - 1)) = __floats2half2_rn(h[k].x, h[k].y);
        } else if constexpr (cx(k) > 0) {  // A -> x0 + 1, B -> x0 + 2
          pop[chk(row + x0 + 1, a.N)] = __float2half_rn(h[k].x);
          if (fxB != 2) pop[chk(row + xbp, a.N)] = __float2half_rn(h[k].y);
        } else {  // A -> x0 - 1, B -> x0
          if (fxA != 1) pop[chk(row + xam, a.N)] = __float2half_rn(h[k].x);
          pop[chk(row + x0, a.N)] = __float2half_rn(h[k].y);
        }
      }
    }
  });
}

// ---------------------------------------------------------------------------------
// Row-staged binary16 sweep: the plain A/B step of a binary16 lattice whose rows are
// whole 16-byte multiples (nx % 8 == 0) and at least ROWS_MIN_NX long. A CTA walks
// destination rows (y, z). One producer warp issues, per row, the 19 bulk copies
// (cp.async.bulk, global -> shared, completing on the stage's "full" mbarrier) of the
// source rows the pull reads -- population k of row (y - c_ky, z - c_kz) -- into a ring
// of ROWS_STAGES shared-memory stages; eight consumer warps wait on a stage, read
// their pairs' populations from it and release it at once on its "empty" mbarrier (one
// arrival per consumer thread), then compute and store while the producer refills it:
// the two sides run decoupled, without block-wide barriers. The x shift of the pull is
// an index into the staged row. Whole rows in flight in shared memory replace loads held in registers,
// which bounded the register-staged paired sweep (64 registers, 32 warps per SM,
// latency-bound). Consumers compute node pairs (x0, x0 + 1) with the paired sweep's
// per-node code (same closure, packed moments and collision), so the bits are those
// of the single-node sweep; results go to global memory as half2 stores.
// Every wait is bounded (STAGE_WAIT_LIMIT_NS); a warp that gives up sets
// ERR_STAGE_WAIT in the lattice's error word and leaves, and the producer, before it
// leaves, waits (bounded again) for the copies it has in flight.
// ---------------------------------------------------------------------------------
constexpr uint32_t ROWS_MIN_NX = 256;
// nodes a stage holds at least (R = ceil(ROWS_STAGE_NODES / nx) rows)
constexpr uint32_t ROWS_STAGE_NODES = 512;
constexpr int ROWS_CONSUMER_WARPS = 8;
constexpr int ROWS_THREADS = 32 * (ROWS_CONSUMER_WARPS + 1);
constexpr uint64_t STAGE_WAIT_LIMIT_NS = 1000000000ull;  // 1 s: far beyond any copy's latency

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// One potentially blocking test of the phase: the thread may be suspended until the
// phase completes or about `hint_ns` have passed, so waiting warps do not spin on the
// issue slots the computing warps need.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity, uint32_t hint_ns = 1000000u) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of `parity` to complete; false once `limit_ns` have passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global
// to shared memory, counted on the mbarrier `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Loads from shared memory through 32-bit shared-window addresses (ld.shared: the
// compiler cannot lose the state space the way it can for a generic pointer), and
// half2 stores through st.global.
__device__ __forceinline__ float lds_half(uint32_t addr) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr) : "memory");
  return __half2float(__ushort_as_half(v));
}
__device__ __forceinline__ void lds_half2(uint32_t addr, float& lo, float& hi) {
  unsigned int v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  lo = __half2float(__ushort_as_half(static_cast<unsigned short>(v & 0xffffu)));
  hi = __half2float(__ushort_as_half(static_cast<unsigned short>(v >> 16)));
}
__device__ __forceinline__ void stg_half2(__half* p, float lo, float hi) {
  const __half2 v = __floats2half2_rn(lo, hi);
  asm volatile("st.global.b32 [%0], %1;" ::"l"(p), "r"(*reinterpret_cast<const unsigned int*>(&v)) : "memory");
}

// MODE: STREAM_AB (pull from the other array, store in place), or the AA steps of an
// even-nx binary16 lattice as in the single-node sweep: STREAM_AA_GATHER stages slot -k
// of the pull sources and pushes f*_k to slot k of node x + c_k, STREAM_AA_LOCAL
// stages the row's own slots and writes slot -k of the same node. In both AA steps
// every node reads and writes only locations it alone owns, so staging a row before
// other rows' nodes write theirs changes nothing.
// Push of the AA gather step for the pair (x0, x0 + 1) of the row-staged sweep: f*_k of
// each node to slot k of node x + c_k, whose row starts zoff[1 + c_z] + yoff[1 + c_y] - x0
// cells into the array (yoff carries x0). CHECK: the pair lies on a walled y or z face
// (fy, fz != 0), where a target beyond the face does not exist; a target beyond a
// walled x face (node A of the first pair for c_x = -1, node B of the last for c_x = +1)
// does not exist either. (Aligned half2 stores of the c_x != 0 populations, with the
// neighbouring pair's value taken by a warp shuffle, measured slower: 2.02 against 1.85
// ms per 512^3 AA step, for the extra shuffles and edge stores.)
template <bool CHECK>
__device__ __forceinline__ void push_gather_rows(const SweepArgs& a, const f32x2 (&h)[Q], const uint32_t (&zoff)[3],
                                                 const uint32_t (&yoff)[3], uint32_t x0, uint32_t xam, uint32_t xbp,
                                                 int fxA, int fxB, int fy, int fz) {
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    if (CHECK && ((fy == 1 && cy(k) < 0) || (fy == 2 && cy(k) > 0) || (fz == 1 && cz(k) < 0) || (fz == 2 && cz(k) > 0)))
      return;
    const uint32_t at = zoff[1 + cz(k)] + yoff[1 + cy(k)];  // target row start + x0
    __half* pop = static_cast<__half*>(a.dst_pop[k]);
    if constexpr (cx(k) == 0) {
      stg_half2(pop + chk(at, a.N - 1), h[k].x, h[k].y);
    } else if constexpr (cx(k) > 0) {  // A -> x0 + 1, B -> x0 + 2
      pop[chk(at + 1, a.N)] = __float2half_rn(h[k].x);
      if (fxB != 2) pop[chk(at - x0 + xbp, a.N)] = __float2half_rn(h[k].y);
    } else {  // A -> x0 - 1, B -> x0
      if (fxA != 1) pop[chk(at - x0 + xam, a.N)] = __float2half_rn(h[k].x);
      pop[chk(at, a.N)] = __float2half_rn(h[k].y);
    }
  });
}

// FIXED: R * nx equals ROWS_STAGE_NODES (nx 256 or 512), so the distance between the
// population rows of a stage is a constant folded into the shared-memory load offsets
// (measured 1.65 against 1.71 ms per 512^3 step with the distance in a register).
template <int STAGES, int MODE, bool FIXED>
__global__ void __launch_bounds__(ROWS_THREADS, 3) sweep_rows_kernel(const __grid_constant__ SweepArgs a) {
  extern __shared__ __align__(128) unsigned char rows_smem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
  const uint32_t nx = a.nx, nrows = a.ny * a.nz;
  const bool px = a.periodic & 1u, py = a.periodic & 2u, pz = a.periodic & 4u;
  const __half* stage0 = reinterpret_cast<const __half*>(rows_smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1u);
      mbar_init(smem_u32(&empty[s]), uint32_t(32 * ROWS_CONSUMER_WARPS));  // every consumer thread
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  // a stage holds R consecutive rows, R * nx / 2 >= the consumer threads when nx allows
  const uint32_t R = (ROWS_STAGE_NODES + nx - 1) / nx;
  const uint32_t ngroups = (nrows + R - 1) / R;
  if (warp == ROWS_CONSUMER_WARPS) {
    // producer: one lane issues every copy of this CTA's row groups (measured faster
    // than spreading the 19 populations over the warp's lanes: 1.77 against 1.85 ms per
    // 512^3 step; issuing faster only sharpened the read bursts)
    if (lane != 0) return;
    const uint32_t row_bytes = nx * uint32_t(sizeof(__half));
    uint32_t i = 0;
    for (;; ++i) {
      const uint32_t g = blockIdx.x + i * gridDim.x;
      if (g >= ngroups) break;
      const int s = int(i % STAGES);
      if (i >= uint32_t(STAGES) &&
          !mbar_wait_bounded(smem_u32(&empty[s]), ((i / STAGES) - 1u) & 1u, STAGE_WAIT_LIMIT_NS)) {
        if (a.err) atomicOr(a.err, ERR_STAGE_WAIT);
        break;
      }
      const uint32_t r0 = g * R;
      const uint32_t rows_here = nrows - r0 < R ? nrows - r0 : R;
      const uint32_t bar = smem_u32(&full[s]);
      mbar_expect_tx(bar, Q * row_bytes * rows_here);
      if (a.drop_copies && blockIdx.x == 0 && i == 0) continue;  // test hook: the wait runs out
      for (uint32_t j = 0; j < rows_here; ++j) {
        const uint32_t r = r0 + j;
        const uint32_t z = fdiv(a.div_ny, r);
        const uint32_t y = r - z * a.ny;
        const uint32_t ym = y ? y - 1 : (py ? a.ny - 1 : 0);
        const uint32_t yp = (y + 1 < a.ny) ? y + 1 : (py ? 0 : a.ny - 1);
        const uint32_t zm = z ? z - 1 : (pz ? a.nz - 1 : 0);
        const uint32_t zp = (z + 1 < a.nz) ? z + 1 : (pz ? 0 : a.nz - 1);
        static_for<0, Q>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          constexpr bool local = MODE == STREAM_AA_LOCAL;
          const uint32_t sy = (local || cy(k) == 0) ? y : (cy(k) > 0 ? ym : yp);
          const uint32_t sz = (local || cz(k) == 0) ? z : (cz(k) > 0 ? zm : zp);
          const uint32_t srow = chk(sz * a.ny + sy, nrows);
          constexpr int slot = MODE == STREAM_AA_GATHER ? opp(k) : k;
          const __half* src = static_cast<const __half*>(a.src_pop[slot]) + size_t(srow) * nx;
          bulk_g2s(smem_u32(stage0 + ((size_t(s) * Q + k) * R + j) * nx), src, row_bytes, bar);
        });
      }
    }
    // the copies of the last (up to STAGES) groups issued may still be in flight: the
    // consumers wait for them; if the loop ended early, wait for them here (bounded)
    if (blockIdx.x + i * gridDim.x < ngroups) {
      for (uint32_t j = (i > uint32_t(STAGES) ? i - STAGES : 0); j < i; ++j)
        (void)mbar_wait_bounded(smem_u32(&full[j % STAGES]), (j / STAGES) & 1u, STAGE_WAIT_LIMIT_NS);
    }
    return;
  }
  // consumers: 256 threads over the node pairs of the group's rows
  const uint32_t npairs = nx >> 1;
  for (uint32_t i = 0;; ++i) {
    const uint32_t g = blockIdx.x + i * gridDim.x;
    if (g >= ngroups) break;
    const int s = int(i % STAGES);
    if (!mbar_wait_bounded(smem_u32(&full[s]), (i / STAGES) & 1u, STAGE_WAIT_LIMIT_NS)) {
      if (a.err) atomicOr(a.err, ERR_STAGE_WAIT);
      return;
    }
    const uint32_t r0 = g * R;
    const uint32_t rows_here = nrows - r0 < R ? nrows - r0 : R;
    const uint32_t empty_bar = smem_u32(&empty[s]);
    const uint32_t total = rows_here * npairs;  // node pairs of the group
    uint32_t q = threadIdx.x;                   // this thread's slot
    if (q >= total) mbar_arrive(empty_bar);     // no pair here: done with stage s
    for (; q < total; q += 32u * ROWS_CONSUMER_WARPS) {
      uint32_t pc = q, jc = 0;  // pair of the row and row of the group
      while (pc >= npairs) {
        pc -= npairs;
        ++jc;
      }
      const bool last = q + 32u * ROWS_CONSUMER_WARPS >= total;  // the thread's last slot of the group
      const uint32_t r = r0 + jc;
      // shared address of row jc of population 0 in stage s
      const uint32_t st = smem_u32(stage0) + uint32_t(((size_t(s) * Q * R + jc) * nx) * sizeof(__half));
      const uint32_t z = fdiv(a.div_ny, r);
      const uint32_t y = r - z * a.ny;
      const int fy = py ? 0 : (y == 0 ? 1 : (y == a.ny - 1 ? 2 : 0));
      const int fz = pz ? 0 : (z == 0 ? 1 : (z == a.nz - 1 ? 2 : 0));
      const uint32_t x0 = 2u * pc;
      const uint32_t xam = x0 ? x0 - 1 : (px ? nx - 1 : 0);
      const uint32_t xbp = (x0 + 2 < nx) ? x0 + 2 : (px ? 0 : nx - 1);
      f32x2 h[Q];
      // population k -> k + 1
      const uint32_t row_stride = (FIXED ? ROWS_STAGE_NODES : R * nx) * uint32_t(sizeof(__half));
      static_for<0, Q>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const uint32_t row = st + uint32_t(k) * row_stride;
        if constexpr (cx(k) == 0 || MODE == STREAM_AA_LOCAL) {
          lds_half2(row + 2u * x0, h[k].x, h[k].y);
        } else if constexpr (cx(k) > 0) {  // pulled from x - 1
          h[k].x = lds_half(row + 2u * xam);
          h[k].y = lds_half(row + 2u * x0);
        } else {  // pulled from x + 1
          h[k].x = lds_half(row + 2u * (x0 + 1));
          h[k].y = lds_half(row + 2u * xbp);
        }
      });
      // the thread's last reads of stage s: the producer refills the stage once every
      // consumer thread has passed here, while the group is still computed and stored
      // (releasing it only after the stores measured 1.77 against 1.65 ms per 512^3 step)
      if (last) mbar_arrive(empty_bar);
      const int fxA = px ? 0 : (x0 == 0 ? 1 : 0);
      const int fxB = px ? 0 : (x0 + 1 == nx - 1 ? 2 : 0);
      const int codeA = fxA + 3 * fy + 9 * fz;
      const int codeB = fxB + 3 * fy + 9 * fz;
      if (codeA != 0) close_lane<0>(codeA, a, x0, y, z, h);
      if (codeB != 0) close_lane<1>(codeB, a, x0 + 1, y, z, h);
      const Moments<f32x2> m = moments(h, f32x2(a.rho0f));
      collide(h, m, f32x2(a.omegaf));
      const uint32_t cell = r * nx + x0;
      if constexpr (MODE == STREAM_AA_GATHER) {
        // push f*_k to slot k of node x + c_k: the target row starts at
        // zoff[1 + c_z] + yoff[1 + c_y]; only a pair on a walled y or z face has targets
        // that do not exist, so only those rows test each population
        const uint32_t ym = y ? y - 1 : (py ? a.ny - 1 : 0);
        const uint32_t yp = (y + 1 < a.ny) ? y + 1 : (py ? 0 : a.ny - 1);
        const uint32_t zm = z ? z - 1 : (pz ? a.nz - 1 : 0);
        const uint32_t zp = (z + 1 < a.nz) ? z + 1 : (pz ? 0 : a.nz - 1);
        const uint32_t plane = a.ny * nx;
        const uint32_t zoff[3] = {zm * plane, z * plane, zp * plane};
        const uint32_t yoff[3] = {ym * nx + x0, y * nx + x0, yp * nx + x0};
        if ((fy | fz) == 0) push_gather_rows<false>(a, h, zoff, yoff, x0, xam, xbp, fxA, fxB, 0, 0);
        else push_gather_rows<true>(a, h, zoff, yoff, x0, xam, xbp, fxA, fxB, fy, fz);
      } else {
        static_for<0, Q>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          constexpr int slot = MODE == STREAM_AA_LOCAL ? opp(k) : k;
          stg_half2(static_cast<__half*>(a.dst_pop[slot]) + chk(cell, a.N - 1), h[k].x, h[k].y);
        });
      }
    }
  }
}

// One time step of every lattice of a batch. A persistent grid draws chunks of the
// batch's global block range from a device counter (the chunk sizes shrink toward the
// end of the range, so the CTAs finish together however unequal the cost of the blocks
// is); a CTA keeps the descriptor of the lattice it is in (in shared memory) while
// consecutive blocks stay in that lattice, and runs the same per-block code as the
// single-lattice sweep, so every lattice computes the same bits alone or in a batch,
// whichever CTA takes which block.
// AB lattices: `parity` picks the direction buf[cur ^ parity] -> buf[cur ^ parity ^ 1].
// AA lattices (MODE != STREAM_AB): both slots of buf[] are the one array.
template <typename S, bool RESID, int MODE>
__global__ void __launch_bounds__(SWEEP_THREADS, (SweepOccupancy<S, RESID, true, MODE>::blocks))
    sweep_batched_kernel(const BatchHeader* __restrict__ hdr, const BatchEntry* __restrict__ ents,
                         const BatchChunk* __restrict__ chunks, uint32_t* __restrict__ next_chunk, uint32_t parity) {
  __shared__ SweepArgs sa;
  __shared__ uint32_t s_chunk;
  const uint32_t nchunks = hdr->nchunks;
  uint32_t cur = 0xffffffffu, lat_begin = 0, lat_end = 0;
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(next_chunk, 1u);
    __syncthreads();
    const uint32_t c = s_chunk;
    __syncthreads();  // s_chunk is rewritten by the next draw
    if (c >= nchunks) break;
    uint32_t b = __ldg(&chunks[c].start);
    const uint32_t bend = __ldg(&chunks[c + 1].start);
    uint32_t e = __ldg(&chunks[c].entry);
    while (b < bend) {
      if (e != cur) {
        __syncthreads();  // every thread is done with the previous descriptor
        const BatchEntry* ent = ents + chk(e, hdr->nentries);
        const uint32_t* from = reinterpret_cast<const uint32_t*>(&ent->a);
        uint32_t* to = reinterpret_cast<uint32_t*>(&sa);
        for (uint32_t w = threadIdx.x; w < sizeof(SweepArgs) / 4; w += SWEEP_THREADS) to[w] = from[w];
        __syncthreads();
        if (threadIdx.x < Q) {
          const uint32_t cb = (ent->cur ^ parity) & 1u;
          const S* src = static_cast<const S*>(ent->buf[cb]);
          S* dst = static_cast<S*>(const_cast<void*>(ent->buf[cb ^ 1u]));
          sa.src_pop[threadIdx.x] = src + size_t(threadIdx.x) * ent->a.N;
          sa.dst_pop[threadIdx.x] = dst + size_t(threadIdx.x) * ent->a.N;
          if (threadIdx.x == 0) {
            sa.src = src;
            sa.dst = dst;
          }
        }
        lat_begin = ent->block_begin;
        lat_end = ent->block_begin + ent->nblocks;
        cur = e;
        __syncthreads();
      }
      if constexpr (MODE == STREAM_AB) {
        if (sa.links || sa.forced) sweep_block<S, RESID, MODE, true>(sa, b - lat_begin);
        else sweep_block<S, RESID, MODE, false>(sa, b - lat_begin);
      } else {
        sweep_block<S, RESID, MODE, false>(sa, b - lat_begin);
      }
      if constexpr (RESID) __syncthreads();  // the block-sum buffer is reused by the next block
      ++b;
      if (b >= lat_end) ++e;
    }
  }
}

// Stored state -> residual terms (no streaming, no update).
// SWAPPED: the state holds f_k in slot -k (an AA lattice after a local step).
template <typename S, bool SWAPPED = false>
__global__ void __launch_bounds__(SWEEP_THREADS)
    state_reduce_kernel(const S* __restrict__ src, uint32_t N, double rho0, void* snap, double* partials) {
  using T = typename ComputeOf<S>::T;
  const uint32_t cell = blockIdx.x * SWEEP_THREADS + threadIdx.x;
  double red[4] = {0.0, 0.0, 0.0, 0.0};
  if (cell < N) {
    T h[Q];
    static_for<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      h[k] = Storage<S>::load(src + size_t(SWAPPED ? opp(k) : k) * N + cell);
    });
    const double ref = ref_rho<S>(rho0);
    const Moments<T> m = moments(h, T(ref));
    residual_terms(m, ref, static_cast<T*>(snap), N, cell, red);
  }
  block_sum4(red, partials + 4ull * blockIdx.x);
}

template <typename S>
__global__ void __launch_bounds__(SWEEP_THREADS) init_kernel(S* __restrict__ dst, uint32_t N, double rho0) {
  using T = typename ComputeOf<S>::T;
  const uint32_t cell = blockIdx.x * SWEEP_THREADS + threadIdx.x;
  if (cell >= N) return;
  // f = f_eq(rho0, 0) = w_i rho0; shifted storage holds 0
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const T v = Storage<S>::shifted ? T(0) : T(wgt<double>(k) * rho0);
    dst[size_t(k) * N + cell] = Storage<S>::store(v);
  });
}

template <typename S, bool SWAPPED>
__global__ void __launch_bounds__(SWEEP_THREADS)
    macros_kernel(const S* __restrict__ src, uint32_t N, double rho0, typename ComputeOf<S>::T* rho,
                  typename ComputeOf<S>::T* u) {
  using T = typename ComputeOf<S>::T;
  const uint32_t cell = blockIdx.x * SWEEP_THREADS + threadIdx.x;
  if (cell >= N) return;
  T h[Q];
  static_for<0, Q>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    h[k] = Storage<S>::load(src + size_t(SWAPPED ? opp(k) : k) * N + cell);
  });
  const Moments<T> m = moments(h, T(ref_rho<S>(rho0)));
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
template <typename S, int MODE, bool GEOM>
void launch_sweep_mode(const SweepArgs& a, bool resid, cudaStream_t s) {
  const uint32_t blocks = sweep_blocks(a.N);
  if (resid) sweep_kernel<S, true, MODE, GEOM><<<blocks, SWEEP_THREADS, 0, s>>>(a);
  else sweep_kernel<S, false, MODE, GEOM><<<blocks, SWEEP_THREADS, 0, s>>>(a);
}

// Stages of the row-staged sweep's shared-memory ring.
constexpr int ROWS_STAGES = 2;

// The row-staged binary16 sweep over every row of the lattice: a persistent grid of
// SMs x the CTAs that fit per SM with the ring's shared memory. Returns
// cudaErrorNotSupported when the ring does not fit (the caller then takes the paired
// sweep).
template <typename S, int MODE>
cudaError_t launch_rows(const SweepArgs& a, cudaStream_t s) {
  static_assert(std::is_same<S, __half>::value, "the row-staged sweep is for binary16 storage");
  const uint32_t R = (ROWS_STAGE_NODES + a.nx - 1) / a.nx;  // rows per stage (as the kernel)
  const size_t smem = size_t(ROWS_STAGES) * Q * R * a.nx * sizeof(__half);
  const bool fixed = R * a.nx == ROWS_STAGE_NODES;
  const void* fn = fixed ? reinterpret_cast<const void*>(sweep_rows_kernel<ROWS_STAGES, MODE, true>)
                         : reinterpret_cast<const void*>(sweep_rows_kernel<ROWS_STAGES, MODE, false>);
  int dev = 0, sms = 0, per = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem + ROWS_STAGES * sizeof(uint64_t) > size_t(optin)) return cudaErrorNotSupported;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, ROWS_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorNotSupported;
  const uint32_t ngroups = (a.ny * a.nz + R - 1) / R;
  const uint32_t grid = uint32_t(sms * per) < ngroups ? uint32_t(sms * per) : ngroups;
  if (fixed) sweep_rows_kernel<ROWS_STAGES, MODE, true><<<grid, ROWS_THREADS, smem, s>>>(a);
  else sweep_rows_kernel<ROWS_STAGES, MODE, false><<<grid, ROWS_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_sweep_impl(const SweepArgs& a, bool resid, int mode, cudaStream_t s) {
  if constexpr (std::is_same<S, __half>::value) {
    if (!resid && !a.links && !a.forced && a.nx % 8 == 0 && a.nx >= ROWS_MIN_NX) {
      const cudaError_t e = mode == STREAM_AA_GATHER ? launch_rows<S, STREAM_AA_GATHER>(a, s)
                            : mode == STREAM_AA_LOCAL ? launch_rows<S, STREAM_AA_LOCAL>(a, s)
                                                      : launch_rows<S, STREAM_AB>(a, s);
      if (e != cudaErrorNotSupported) return e;
    }
    if (!resid && !a.links && !a.forced && (a.nx & 1u) == 0) {
      const uint32_t blocks = sweep_blocks(a.N >> 1);
      if (mode == STREAM_AA_GATHER) sweep_pair_kernel<S, STREAM_AA_GATHER><<<blocks, SWEEP_THREADS, 0, s>>>(a);
      else if (mode == STREAM_AA_LOCAL) sweep_pair_kernel<S, STREAM_AA_LOCAL><<<blocks, SWEEP_THREADS, 0, s>>>(a);
      else sweep_pair_kernel<S, STREAM_AB><<<blocks, SWEEP_THREADS, 0, s>>>(a);
      return cudaGetLastError();
    }
  }
  if (mode == STREAM_AA_GATHER) launch_sweep_mode<S, STREAM_AA_GATHER, false>(a, resid, s);
  else if (mode == STREAM_AA_LOCAL) launch_sweep_mode<S, STREAM_AA_LOCAL, false>(a, resid, s);
  else if (a.links || a.forced) launch_sweep_mode<S, STREAM_AB, true>(a, resid, s);
  else launch_sweep_mode<S, STREAM_AB, false>(a, resid, s);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_init_impl(void* dst, uint32_t N, double rho0, cudaStream_t s) {
  init_kernel<S><<<sweep_blocks(N), SWEEP_THREADS, 0, s>>>(static_cast<S*>(dst), N, rho0);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macros_impl(const void* src, uint32_t N, double rho0, void* rho, void* u, bool swapped,
                               cudaStream_t s) {
  using T = typename ComputeOf<S>::T;
  if (swapped)
    macros_kernel<S, true><<<sweep_blocks(N), SWEEP_THREADS, 0, s>>>(static_cast<const S*>(src), N, rho0,
                                                                     static_cast<T*>(rho), static_cast<T*>(u));
  else
    macros_kernel<S, false><<<sweep_blocks(N), SWEEP_THREADS, 0, s>>>(static_cast<const S*>(src), N, rho0,
                                                                      static_cast<T*>(rho), static_cast<T*>(u));
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_state_reduce_impl(const void* src, uint32_t N, double rho0, void* snap, double* partials,
                                     bool swapped, cudaStream_t s) {
  if (swapped)
    state_reduce_kernel<S, true><<<sweep_blocks(N), SWEEP_THREADS, 0, s>>>(static_cast<const S*>(src), N, rho0,
                                                                           snap, partials);
  else
    state_reduce_kernel<S, false><<<sweep_blocks(N), SWEEP_THREADS, 0, s>>>(static_cast<const S*>(src), N, rho0,
                                                                            snap, partials);
  return cudaGetLastError();
}

template <typename S, int MODE>
void launch_batched_mode(const BatchHeader* hdr, const BatchEntry* ents, const BatchChunk* chunks, uint32_t* next,
                         uint32_t parity, bool resid, int grid, cudaStream_t s) {
  if (resid) sweep_batched_kernel<S, true, MODE><<<grid, SWEEP_THREADS, 0, s>>>(hdr, ents, chunks, next, parity);
  else sweep_batched_kernel<S, false, MODE><<<grid, SWEEP_THREADS, 0, s>>>(hdr, ents, chunks, next, parity);
}

template <typename S>
cudaError_t launch_sweep_batched_impl(const BatchHeader* hdr, const BatchEntry* ents, const BatchChunk* chunks,
                                      uint32_t* next, uint32_t parity, bool resid, int mode, int grid,
                                      cudaStream_t s) {
  if (mode == STREAM_AA_GATHER) launch_batched_mode<S, STREAM_AA_GATHER>(hdr, ents, chunks, next, parity, resid, grid, s);
  else if (mode == STREAM_AA_LOCAL) launch_batched_mode<S, STREAM_AA_LOCAL>(hdr, ents, chunks, next, parity, resid, grid, s);
  else launch_batched_mode<S, STREAM_AB>(hdr, ents, chunks, next, parity, resid, grid, s);
  return cudaGetLastError();
}

// Persistent grid of each batched variant: SMs x the residency the occupancy query
// gives for that variant (the chunk counter balances any grid size).
template <typename S>
int batched_grid_impl(bool resid, int mode) {
  int dev = 0, sms = 0, r = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const void* fn = nullptr;
  if (mode == STREAM_AA_GATHER)
    fn = resid ? reinterpret_cast<const void*>(sweep_batched_kernel<S, true, STREAM_AA_GATHER>)
               : reinterpret_cast<const void*>(sweep_batched_kernel<S, false, STREAM_AA_GATHER>);
  else if (mode == STREAM_AA_LOCAL)
    fn = resid ? reinterpret_cast<const void*>(sweep_batched_kernel<S, true, STREAM_AA_LOCAL>)
               : reinterpret_cast<const void*>(sweep_batched_kernel<S, false, STREAM_AA_LOCAL>);
  else
    fn = resid ? reinterpret_cast<const void*>(sweep_batched_kernel<S, true, STREAM_AB>)
               : reinterpret_cast<const void*>(sweep_batched_kernel<S, false, STREAM_AB>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, fn, SWEEP_THREADS, 0) != cudaSuccess) return 0;
  return sms * r;
}

// Count of out-of-range indices this translation unit's kernels met (debug build; the
// count is reset by the read), or 0 in the release build.
static inline uint32_t bounds_errors_impl() {
#ifdef LBM_DEBUG_BOUNDS
  unsigned int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_errors, sizeof v) != cudaSuccess) return ~0u;
  if (cudaMemcpyToSymbol(g_bounds_errors, &zero, sizeof zero) != cudaSuccess) return ~0u;
  return v;
#else
  return 0u;
#endif
}

#define LBM_INSTANTIATE(S)                                                                              \
  template <> cudaError_t launch_sweep<S>(const SweepArgs& a, bool resid, int mode, cudaStream_t s) {   \
    return launch_sweep_impl<S>(a, resid, mode, s);                                                     \
  }                                                                                                     \
  template <> cudaError_t launch_init<S>(void* dst, uint32_t N, double rho0, cudaStream_t s) {          \
    return launch_init_impl<S>(dst, N, rho0, s);                                                        \
  }                                                                                                     \
  template <> cudaError_t launch_macros<S>(const void* src, uint32_t N, double rho0, void* rho, void* u, \
                                           bool swapped, cudaStream_t s) {                              \
    return launch_macros_impl<S>(src, N, rho0, rho, u, swapped, s);                                     \
  }                                                                                                     \
  template <> cudaError_t launch_state_reduce<S>(const void* src, uint32_t N, double rho0, void* snap,  \
                                                 double* partials, bool swapped, cudaStream_t s) {     \
    return launch_state_reduce_impl<S>(src, N, rho0, snap, partials, swapped, s);                       \
  }                                                                                                     \
  template <> cudaError_t launch_sweep_batched<S>(const BatchHeader* hdr, const BatchEntry* ents,       \
                                                  const BatchChunk* chunks, uint32_t* next,             \
                                                  uint32_t parity, bool resid, int mode, int grid,      \
                                                  cudaStream_t s) {                                     \
    return launch_sweep_batched_impl<S>(hdr, ents, chunks, next, parity, resid, mode, grid, s);        \
  }                                                                                                     \
  template <> int batched_grid<S>(bool resid, int mode) { return batched_grid_impl<S>(resid, mode); }   \
  template <> uint32_t bounds_errors<S>() { return bounds_errors_impl(); }

}  // namespace lbm
