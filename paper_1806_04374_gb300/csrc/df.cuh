// df.cuh -- double-float ("float-float") arithmetic for the exact re-scoring
// and least-squares inputs of the rotational OMP kernels.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the error-free
// transformations of Knuth (TwoSum) and of Dekker with a fused multiply-add
// (TwoProd), as used by Ogita, Rump and Oishi, "Accurate Sum and Dot
// Product" (SIAM J. Sci. Comput. 26(6), 2005).  GB300 runs FP32 at 64 times
// its FP64 rate, so these few FP32 operations per multiply-add are far
// cheaper than FP64.  The file must be compiled without fast-math: the
// transformations rely on IEEE round-to-nearest and on no reassociation.
#pragma once

#include <cuda_runtime.h>

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi) { return {hi, 0.0f}; }

// a + b = s + e exactly (Knuth's TwoSum).
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// a + b = s + e exactly when |a| >= |b| (Dekker's FastTwoSum).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

// a * b = p + e exactly (TwoProd with FMA).
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// (hi + lo) * f for a float f.
__device__ __forceinline__ df df_mul_f(df a, float f) {
  df p = two_prod(a.hi, f);
  float e = __fmaf_rn(a.lo, f, p.lo);
  return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, e);
}

// acc + a * b (a, b double-float).
__device__ __forceinline__ df df_fma(df acc, df a, df b) { return df_add(acc, df_mul(a, b)); }

__device__ __forceinline__ double df_to_d(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_from_d(double v) {
  float hi = __double2float_rn(v);
  float lo = __double2float_rn(v - (double)hi);
  return {hi, lo};
}

__device__ __forceinline__ df df_shfl_xor(df a, int mask) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, mask), __shfl_xor_sync(0xffffffffu, a.lo, mask)};
}

// Sum over the 32 lanes of a warp; every lane receives the same value.
__device__ __forceinline__ df df_warp_sum(df a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
  return {__shfl_sync(0xffffffffu, a.hi, 0), __shfl_sync(0xffffffffu, a.lo, 0)};
}
