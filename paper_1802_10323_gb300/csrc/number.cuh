// number.cuh — the number types the RK3 predictor is written in.
//
// The predictor's body is written once for a number type N: float for FP32 fields and
// ddf, a double-float pair (~48-bit significand on the FP32 pipe, built on the df
// helpers of common.cuh), for FP64 fields. Kept out of common.cuh so that only the
// predictor's translation unit depends on it.
#pragma once
#include <type_traits>

#include "common.cuh"

// ddf: the same hi + lo representation as df, with +, −, × overloaded, so that a
// kernel body can be written once for a number type N: float for FP32 fields, ddf
// for FP64 fields (NumOf<T>). Num<N> converts: in() from the field type (FP64 split
// on its bit pattern), out() to it (one FP64 add for ddf), zero(), and scale() by a
// power of two (exact).
struct ddf {
  float h, l;
};
// Addition without the final renormalisation of df_add: (s.h, s.l + a.l + b.l) with
// s = TwoSum(a.h, b.h), three FP32 operations fewer. The low word may then exceed half an
// ulp of the high one; the pair still holds the sum to about 2^−47 of the larger operand,
// the product takes both words of each operand in its cross terms, and out() adds the two
// words in FP64, so nothing downstream assumes the pair is normalised.
__device__ __forceinline__ ddf operator+(ddf a, ddf b) {
  const df s = two_sum(a.h, b.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ ddf operator-(ddf a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ddf operator-(ddf a, ddf b) { return a + (-b); }
__device__ __forceinline__ ddf operator*(ddf a, ddf b) {
  const df r = df_mul(df{a.h, a.l}, df{b.h, b.l});
  return {r.h, r.l};
}
template <class N>
struct Num;
template <>
struct Num<float> {
  static __device__ __forceinline__ float in(float x) { return x; }
  static __device__ __forceinline__ float out(float x) { return x; }
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ float scale(float x, float pow2) { return x * pow2; }
};
template <>
struct Num<ddf> {
  static __device__ __forceinline__ ddf in(double x) {
    ddf r;
    split_f64(x, r.h, r.l);
    return r;
  }
  static __device__ __forceinline__ double out(ddf x) { return widen_f32(x.h) + widen_f32(x.l); }
  static __device__ __forceinline__ ddf zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ ddf scale(ddf x, float pow2) { return {x.h * pow2, x.l * pow2}; }
};
template <class T>
using NumOf = typename std::conditional<sizeof(T) == 8, ddf, float>::type;
