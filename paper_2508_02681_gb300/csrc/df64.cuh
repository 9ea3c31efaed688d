// Float-pair ("double-float") arithmetic on the FP32 pipes, for the FP64-accurate residual
// replacement of the mixed-precision path (FP64 instructions run at 1/64 of the FP32 rate on
// this GPU).  A value is hi + lo with |lo| <= ulp(hi)/2.  The error-free transformations are the
// textbook ones (Knuth's TwoSum, Dekker's fast TwoSum for |a| >= |b|, the FMA-based exact
// product); the intrinsics keep the compiler from contracting or reordering them.
#pragma once
#include <cuda_runtime.h>

namespace unocg {

struct df32 {
  float hi, lo;
};

__device__ __forceinline__ df32 df_make(float v) { return {v, 0.0f}; }

__device__ __forceinline__ df32 df_from_double(double v) {
  const float hi = __double2float_rn(v);
  return {hi, __double2float_rn(v - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df32 x) { return (double)x.hi + (double)x.lo; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly, for |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df32 r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.hi, -a.lo}; }

// a * b (both pairs)
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  df32 r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// x += m * w for a small integer m (exact in FP32) and a pair w
__device__ __forceinline__ void df_add_mul(df32& x, float m, df32 w) {
  const float p = __fmul_rn(m, w.hi);
  float pe = __fmaf_rn(m, w.hi, -p);
  pe = __fmaf_rn(m, w.lo, pe);
  float s, e;
  two_sum(x.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(pe, x.lo));
  fast_two_sum(s, e, x.hi, x.lo);
}

// u + a * d for FP32 u, d and a pair a
__device__ __forceinline__ df32 df_axpy(df32 a, float d, float u) {
  const float p = __fmul_rn(a.hi, d);
  float pe = __fmaf_rn(a.hi, d, -p);
  pe = __fmaf_rn(a.lo, d, pe);
  float s, e;
  two_sum(u, p, s, e);
  e = __fadd_rn(e, pe);
  df32 r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

}  // namespace unocg
