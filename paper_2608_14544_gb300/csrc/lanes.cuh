// lanes.cuh -- one or two walkers per thread: FP32 values of type float (one
// walker) or float2 (two walkers, walker l in lane l), the arithmetic that
// maps to Blackwell's packed FP32x2 instructions, and lane access.  Shared by
// the two-state and the N_s-state FP32-bulk kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qcl_common.cuh"

namespace qcl {

// ------------------------------------------------ walker lanes (1 or 2) --
// A thread advances one walker (values of type float) or two (float2: walker
// l in lane l).  All FP32 arithmetic of a step goes through vfma / vmul / vadd
// / vsub: for float2 these are the packed FP32x2 instructions (one issue slot
// for both walkers), and every form rounds each lane exactly as the scalar
// operation does (IEEE round to nearest, never contracted), so a walker's bits
// do not depend on the lane count.  Work without a packed form (MUFU,
// conversions, comparisons, selects, integer work) runs lane by lane.
template <typename V>
struct Lanes;
template <>
struct Lanes<float> {
  static constexpr int W = 1;
  using I = int;
  using U = uint32_t;
};
template <>
struct Lanes<float2> {
  static constexpr int W = 2;
  using I = int2;
  using U = uint2;
};

__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <typename V>
__device__ __forceinline__ V splat(float c);
template <>
__device__ __forceinline__ float splat<float>(float c) { return c; }
template <>
__device__ __forceinline__ float2 splat<float2>(float c) { return make_float2(c, c); }
// a - b = fma(b, -1, a) exactly (one rounding, as a subtraction)
template <typename V>
__device__ __forceinline__ V vsub(V a, V b) { return vfma(b, splat<V>(-1.0f), a); }

// lane l of a value (l a compile-time constant after unrolling)
__device__ __forceinline__ float& ln(float& v, int) { return v; }
__device__ __forceinline__ const float& ln(const float& v, int) { return v; }
__device__ __forceinline__ float& ln(float2& v, int l) { return l ? v.y : v.x; }
__device__ __forceinline__ const float& ln(const float2& v, int l) { return l ? v.y : v.x; }
__device__ __forceinline__ int& ln(int& v, int) { return v; }
__device__ __forceinline__ const int& ln(const int& v, int) { return v; }
__device__ __forceinline__ int& ln(int2& v, int l) { return l ? v.y : v.x; }
__device__ __forceinline__ const int& ln(const int2& v, int l) { return l ? v.y : v.x; }
__device__ __forceinline__ uint32_t& ln(uint32_t& v, int) { return v; }
__device__ __forceinline__ const uint32_t& ln(const uint32_t& v, int) { return v; }
__device__ __forceinline__ uint32_t& ln(uint2& v, int l) { return l ? v.y : v.x; }
__device__ __forceinline__ const uint32_t& ln(const uint2& v, int l) { return l ? v.y : v.x; }

template <typename V>
__device__ __forceinline__ PairV<V> two_sum_v(V a, V b) {
  const V s = vadd(a, b);
  const V bb = vsub(s, a);
  return {s, vadd(vsub(a, vsub(s, bb)), vsub(b, bb))};
}
template <typename V>
__device__ __forceinline__ PairV<V> fast_two_sum_v(V a, V b) {  // |a| >= |b|
  const V s = vadd(a, b);
  return {s, vsub(b, vsub(s, a))};
}

// (hi, lo) += b  (as df_add)
template <typename V>
__device__ __forceinline__ PairV<V> df_add_v(PairV<V> a, V b) {
  const PairV<V> s = two_sum_v(a.hi, b);
  return fast_two_sum_v(s.hi, vadd(s.lo, a.lo));
}

// (hi, lo) *= (q0 + q1)  (as df_mul)
template <typename V>
__device__ __forceinline__ PairV<V> df_mul_v(PairV<V> a, V q0, V q1) {
  const V p = vmul(a.hi, q0);
  V e = vfma(a.hi, q0, vmul(p, splat<V>(-1.0f)));
  e = vfma(a.hi, q1, e);
  e = vfma(a.lo, q0, e);
  return fast_two_sum_v(p, e);
}

}  // namespace qcl
