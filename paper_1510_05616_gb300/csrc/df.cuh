// df.cuh -- double-float arithmetic on the FP32 pipes: a real number is an unevaluated pair of
// floats (h, l), |l| at most a few ulp of h, ~48 significant bits.  Sums use the error-free
// TwoSum / Fast2Sum transformations and products the FMA-based exact product (Dekker / Knuth,
// as in double-double libraries).  The _rn intrinsics keep the compiler from contracting or
// reassociating the transformations.
#pragma once
#include <cuda_runtime.h>

namespace stokes {

struct df {
  float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Exact when |a| >= |b| (or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// acc += a * b, acc a double-float accumulator (the l * l term dropped).
__device__ __forceinline__ void df_mul_acc(df &acc, df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const df s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}

// Renormalise an accumulator so |l| <= ulp(h)/2: without it the low word collects every
// rounding error of a long sum, grows like sqrt(n) ulp(h), and its own rounding then costs
// ~2^-24 of that per addition.
__device__ __forceinline__ void df_renorm(df &a) { a = fast_two_sum(a.h, a.l); }

__device__ __forceinline__ df split_df(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - double(h))};
}

}  // namespace stokes
