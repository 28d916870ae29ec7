// Double-float arithmetic on pairs of float32 values for the outer Krylov
// iteration of the float32-cycle solve.
//
// The float64 pipe of this GPU runs at about 1/60 of the float32 rate
// (measured: 1.1 against 69.9 TFLOP/s), so float64 vector work over the finest grid
// (Gram-Schmidt dots and updates, the outer operator, the combination
// x += Z y) is bound by arithmetic, not by memory.  A value v is kept as an
// unevaluated sum hi + lo of two float32 numbers (|lo| <= ulp(hi)/2 after
// normalisation: 48 significant bits against float64's 53), and every step
// uses error-free transformations on float32 numbers only:
//
//   Knuth's two-sum:       s = fl(a + b), e = (a - (s - bb)) + (b - bb) with
//                          bb = s - a gives s + e = a + b exactly;
//   the FMA two-product:   p = fl(a b), e = fma(a, b, -p) gives p + e = a b
//                          exactly (Dekker's product, with the FMA in place
//                          of his splitting).
//
// A running sum keeps its large terms exactly as (s, u) by two-sum, and the
// small terms (two-sum errors, product errors, cross products hi*lo) in a
// float32 tail t; the value is s + t.  The cross product lo*lo is below 2^-48
// of the product and is dropped.  The explicit float64 residual at every
// restart of the outer iteration removes the drift this leaves.
#pragma once

#include <cuda_runtime.h>
#ifndef __CUDA_ARCH__
#include <cmath>
#endif

namespace adr {

struct DfSum { float s, t; };   // value s + t

// Round-to-nearest float32 operations: the device intrinsics (never
// contracted into an FMA), or plain IEEE operations when this header is
// compiled for the host (the host-side checks of the transformations).
#ifdef __CUDA_ARCH__
#define ADR_DF_ADD(a, b) __fadd_rn(a, b)
#define ADR_DF_SUB(a, b) __fsub_rn(a, b)
#define ADR_DF_MUL(a, b) __fmul_rn(a, b)
#define ADR_DF_FMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define ADR_DF_ADD(a, b) ((a) + (b))
#define ADR_DF_SUB(a, b) ((a) - (b))
#define ADR_DF_MUL(a, b) ((a) * (b))
#define ADR_DF_FMA(a, b, c) std::fmaf(a, b, c)
#endif

__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = ADR_DF_ADD(a, b);
  const float bb = ADR_DF_SUB(s, a);
  e = ADR_DF_ADD(ADR_DF_SUB(a, ADR_DF_SUB(s, bb)), ADR_DF_SUB(b, bb));
}

// a += p + q, p added exactly, q (small) into the tail.
__host__ __device__ __forceinline__ void df_acc(DfSum& a, float p, float q) {
  float s, u;
  two_sum(a.s, p, s, u);
  a.s = s;
  a.t = ADR_DF_ADD(a.t, ADR_DF_ADD(u, q));
}

// a += (c_hi + c_lo) x for a float32 x.
__host__ __device__ __forceinline__ void df_add_prod(DfSum& a, float c_hi, float c_lo, float x) {
  const float p = ADR_DF_MUL(c_hi, x);
  float e = ADR_DF_FMA(c_hi, x, -p);
  e = ADR_DF_FMA(c_lo, x, e);
  df_acc(a, p, e);
}

// a += (x_hi + x_lo)(y_hi + y_lo).
__host__ __device__ __forceinline__ void df_add_prod2(DfSum& a, float xh, float xl, float yh, float yl) {
  const float p = ADR_DF_MUL(xh, yh);
  float e = ADR_DF_FMA(xh, yh, -p);
  e = ADR_DF_FMA(xh, yl, e);
  e = ADR_DF_FMA(xl, yh, e);
  df_acc(a, p, e);
}

// a += b
__host__ __device__ __forceinline__ void df_add(DfSum& a, const DfSum& b) { df_acc(a, b.s, b.t); }

// The normalised pair (hi, lo) of s + t: hi = fl(s + t).  Two-sum, not the
// fast form: after cancellation the tail can exceed s.
__host__ __device__ __forceinline__ float2 df_pair(const DfSum& a) {
  float h, l;
  two_sum(a.s, a.t, h, l);
  return make_float2(h, l);
}

// Widened to float64 (two conversions and an add: per thread once, not per
// element).
__host__ __device__ __forceinline__ double df_double(const DfSum& a) { return (double)a.s + (double)a.t; }

// The float32 pair of a float64 value (|v - hi - lo| <= 2^-48 |v|).
__host__ __device__ __forceinline__ float2 df_split(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ DfSum df_shfl_down(const DfSum& a, int o) {
  return DfSum{__shfl_down_sync(0xffffffffu, a.s, o), __shfl_down_sync(0xffffffffu, a.t, o)};
}

}  // namespace adr
