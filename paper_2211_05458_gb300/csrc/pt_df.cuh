// pt_df.cuh -- double-float arithmetic: a value is an unevaluated sum hi + lo
// of two FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  Built
// from the error-free transformations TwoSum (Knuth, TAOCP vol. 2) and the
// FMA form of TwoProduct (Ogita, Rump & Oishi, SIAM J. Sci. Comput. 2005),
// with dot products accumulated as in their Dot2 algorithm.  Used for the
// final Newton residuals of the FP32 mode, which need ~1e-14 relative
// accuracy and would otherwise run on GB300's narrow FP64 pipe.
#pragma once
#include <cuda_runtime.h>

namespace pt {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_from(float a) { return {a, 0.f}; }

// split a double into hi + lo
__device__ __forceinline__ df df_from_double(double a) {
  float h = (float)a;
  return {h, (float)(a - (double)h)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, valid for |a| >= |b|
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// p + e = a * b exactly
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ df df_mul(df a, df b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}

// running dot product: (s, c) accumulates sum x_i y_i (Dot2 with the cross
// terms of the double-float operands added to the compensation)
struct df_acc {
  float s, c;
};
__device__ __forceinline__ void dacc_init(df_acc& a) { a.s = a.c = 0.f; }
__device__ __forceinline__ void dacc_fma(df_acc& a, df x, df y) {
  float p, pe, s, se;
  two_prod(x.hi, y.hi, p, pe);
  two_sum(a.s, p, s, se);
  a.s = s;
  float c = __fadd_rn(a.c, __fadd_rn(pe, se));
  c = __fmaf_rn(x.hi, y.lo, c);
  a.c = __fmaf_rn(x.lo, y.hi, c);
}
__device__ __forceinline__ df dacc_result(const df_acc& a) {
  df r;
  two_sum(a.s, a.c, r.hi, r.lo);
  return r;
}

}  // namespace pt
