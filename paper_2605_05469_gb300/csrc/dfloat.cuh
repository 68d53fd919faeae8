// Double-float arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2: a ~48-bit significand (relative precision ~2^-47),
// against 53 bits for FP64, at FP32 throughput (GB300 issues FP64 at 1/58 of
// its FP32 rate). Built from the error-free transformations
//   TwoSum   (Knuth, TAOCP vol. 2): s + e = a + b exactly, 6 operations;
//   FastTwoSum (Dekker 1971): the same when |a| >= |b| (or a = 0), 3;
//   TwoProd  p + e = a b exactly with one FMA (e = fma(a, b, -p)), 2;
// and the double-word sum and product of Joldes, Muller & Popescu (ACM TOMS
// 2017: "AccurateDWPlusDW", relative error <= 3 u^2; "DWTimesDW", <= 5 u^2 with
// u = 2^-24). Every addition and product here uses the _rn intrinsics, which
// the compiler never contracts into an FMA, so the transformations stay exact.
#pragma once
#include <cuda_runtime.h>

namespace pic {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) { return {hi, lo}; }
__device__ __forceinline__ df df_from(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 df_pack(df a) { return make_float2(a.hi, a.lo); }

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| or a == 0
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}

// a + b (AccurateDWPlusDW)
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  const df v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a b (DWTimesDW)
__device__ __forceinline__ df df_mul(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  float t = __fmul_rn(a.hi, b.lo);
  t = fmaf(a.lo, b.hi, t);
  return fast_two_sum(p.hi, __fadd_rn(p.lo, t));
}

// A running sum of double-float terms whose hi parts are added exactly
// (TwoSum) and whose low parts and rounding errors gather in one FP32 word;
// the result is renormalised once at the end. For k terms of magnitude <= M
// its absolute error is about k 2^-24 max|lo| + 2^-48 |sum| <= ~k 2^-48 M.
struct DfAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(df a) {
    const df s = two_sum(hi, a.hi);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, a.lo));
  }
  // += w * a (w, a double-float)
  __device__ __forceinline__ void add_mul(df w, df a) {
    const df p = two_prod(w.hi, a.hi);
    float t = __fmul_rn(w.hi, a.lo);
    t = fmaf(w.lo, a.hi, t);
    const df s = two_sum(hi, p.hi);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, __fadd_rn(p.lo, t)));
  }
  __device__ __forceinline__ df value() const {
    // |lo| may exceed |hi| after cancellation: normalise with TwoSum
    return two_sum(hi, lo);
  }
};

// ---------------------------------------------------------------------------
// Two double-float values at once on Blackwell's packed FP32 instructions
// (FADD2 / FMUL2 / FFMA2 on float2): lane i of every operation rounds exactly
// as the scalar _rn operation on lane i would, so a pair computes bit for bit
// what two scalar double-float computations give, in half the instructions.
// ---------------------------------------------------------------------------
struct df2 {
  float2 hi, lo;  // lane x: first value, lane y: second
};

__device__ __forceinline__ float2 bcast(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ df2 df2_pair(df a, df b) { return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ df2 df2_bcast(df a) { return {bcast(a.hi), bcast(a.lo)}; }
__device__ __forceinline__ df df2_x(const df2& a) { return {a.hi.x, a.lo.x}; }
__device__ __forceinline__ df df2_y(const df2& a) { return {a.hi.y, a.lo.y}; }

__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ df2 two_prod2(float2 a, float2 b) {
  const float2 p = mul2(a, b);
  return {p, fma2(a, b, neg2(p))};
}

// a + b lane by lane (AccurateDWPlusDW)
__device__ __forceinline__ df2 df2_add(const df2& a, const df2& b) {
  const df2 s = two_sum2(a.hi, b.hi);
  const df2 t = two_sum2(a.lo, b.lo);
  const df2 v = fast_two_sum2(s.hi, add2(s.lo, t.hi));
  return fast_two_sum2(v.hi, add2(t.lo, v.lo));
}

// a b lane by lane (DWTimesDW)
__device__ __forceinline__ df2 df2_mul(const df2& a, const df2& b) {
  const df2 p = two_prod2(a.hi, b.hi);
  float2 t = mul2(a.hi, b.lo);
  t = fma2(a.lo, b.hi, t);
  return fast_two_sum2(p.hi, add2(p.lo, t));
}

// DfAcc on a pair of running sums.
struct DfAcc2 {
  float2 hi = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
  // += w * a (w, a double-float pairs)
  __device__ __forceinline__ void add_mul(const df2& w, const df2& a) {
    const df2 p = two_prod2(w.hi, a.hi);
    float2 t = mul2(w.hi, a.lo);
    t = fma2(w.lo, a.hi, t);
    const df2 s = two_sum2(hi, p.hi);
    hi = s.hi;
    lo = add2(lo, add2(s.lo, add2(p.lo, t)));
  }
  __device__ __forceinline__ df2 value() const { return two_sum2(hi, lo); }
};

// Double-float of an FP64 value (FP64 operations: for inputs and outputs only).
__device__ __forceinline__ df df_of_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}
__device__ __forceinline__ double double_of_df(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace pic
