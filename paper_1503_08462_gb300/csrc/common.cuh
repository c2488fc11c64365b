// Shared device helpers: error plumbing, launch geometry and float-float
// ("double-float") arithmetic.
//
// Float-float numbers are unevaluated sums hi + lo of two float32 values with
// |lo| <= ulp(hi)/2, giving a 48-bit significand.  The error-free
// transformations are Knuth's TwoSum, Dekker's Fast-TwoSum and the FMA form of
// Dekker's TwoProduct (Dekker 1971, "A floating-point technique for extending
// the available precision"; Knuth, TAOCP vol. 2, 4.2.2); the accumulation in
// dot products follows the compensated scheme of Ogita, Rump and Oishi (2005,
// "Accurate sum and dot product").  On this GPU float32 FMA issues ~59x faster
// than float64 FMA and its dependent latency is ~14x lower, so the
// latency-bound dense eigensolver runs in float-float.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "amgeig.h"

namespace amgeig {

constexpr int kNumSms = 152;

// ---------------------------------------------------------------- float-float

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l = 0.f) { return df{h, l}; }

__device__ __forceinline__ df df_from_double(double d) {
  float h = static_cast<float>(d);
  float l = static_cast<float>(d - static_cast<double>(h));
  return df{h, l};
}

__device__ __forceinline__ double df_to_double(df x) {
  return static_cast<double>(x.hi) + static_cast<double>(x.lo);
}

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // requires |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df{s, e};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return df{p, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// a / b: float quotient refined by two Newton-type corrections on the remainder
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = df_sub(a, df_mul_f(b, q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = df_sub(r, df_mul_f(b, q2));
  float q3 = __fdiv_rn(r.hi, b.hi);
  df q = fast_two_sum(q1, q2);
  return df_add(q, df{q3, 0.f});
}

// 1 / b: the float32 reciprocal refined by one Newton step in float-float,
// r <- r + r (1 - b r); the relative error squares (2^-24 -> ~2^-48).  Cheaper
// than df_div's three corrections, for the latency-bound pivots and shifts.
__device__ __forceinline__ df df_recip(df b) {
  const float r = __frcp_rn(b.hi);
  const df e = df_sub(df{1.f, 0.f}, df_mul_f(b, r));
  return df_add(df{r, 0.f}, df_mul_f(e, r));
}

__device__ __forceinline__ df df_sqrt(df a) {
  if (a.hi <= 0.f) return df{0.f, 0.f};
  float s = __fsqrt_rn(a.hi);
  df s2 = two_prod(s, s);
  df r = df_sub(a, s2);
  float c = __fdiv_rn(r.hi, 2.f * s);
  return fast_two_sum(s, c);
}

__device__ __forceinline__ float df_float(df a) { return a.hi + a.lo; }
__device__ __forceinline__ bool df_lt0(df a) { return a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f); }
__device__ __forceinline__ df df_abs(df a) { return df_lt0(a) ? df_neg(a) : a; }

// Compensated accumulator for sum_i x_i*y_i (x_i, y_i float-float).  Plain
// aggregate (usable in shared memory); start from acc_zero().
struct df_acc {
  float s, c;  // running sum s (float) and compensation c (float)
  __device__ __forceinline__ void fma(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    df t = two_sum(s, p.hi);
    s = t.hi;
    float cross = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
    c = __fadd_rn(c, __fadd_rn(t.lo, __fadd_rn(p.lo, cross)));
  }
  __device__ __forceinline__ void add(df x) {
    df t = two_sum(s, x.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, x.lo));
  }
  __device__ __forceinline__ void merge(const df_acc& o) {
    df t = two_sum(s, o.s);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, o.c));
  }
  __device__ __forceinline__ df value() const { return fast_two_sum(s, c); }
};

__device__ __forceinline__ df_acc acc_zero() {
  df_acc a;
  a.s = 0.f;
  a.c = 0.f;
  return a;
}

__device__ __forceinline__ df_acc shfl_xor_acc(df_acc a, int mask) {
  df_acc o;
  o.s = __shfl_xor_sync(0xffffffffu, a.s, mask);
  o.c = __shfl_xor_sync(0xffffffffu, a.c, mask);
  return o;
}

// ---------------------------------------------------------------- reductions

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

inline int ceil_div(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace amgeig
