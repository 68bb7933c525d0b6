// Double-float arithmetic for the FP32-bulk flux: a value is the unevaluated
// sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48
// significant bits, computed on the FP32 pipes (this part's FP64 rate is a
// small fraction of its FP32 rate).  Built from error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2): s = fl(a + b) and the exact
//     error e with a + b = s + e, for any a, b;
//   FastTwoSum (Dekker 1971): the same when |a| >= |b|, used to renormalise;
//   TwoProd with a fused multiply-add: p = fl(a b), e = fma(a, b, -p) exactly.
// The addition keeps both the high and the low parts exact through TwoSum
// before renormalising, so a sum with cancellation between its operands keeps
// a relative error of a few 2^-48.  Every operation is spelled with the
// round-to-nearest intrinsics so the compiler cannot contract or reorder it.
#pragma once

#include <cuda_runtime.h>

namespace wlseno {

struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfloat df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfloat df_neg(dfloat x) { return {-x.hi, -x.lo}; }

// x + y
__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
  dfloat s = df_two_sum(x.hi, y.hi);
  const dfloat t = df_two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

// x * y
__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
  dfloat p = df_two_prod(x.hi, y.hi);
  p.lo = __fmaf_rn(x.hi, y.lo, p.lo);
  p.lo = __fmaf_rn(x.lo, y.hi, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}

// The pair nearest an FP64 value (hi = fl32(v), lo = fl32(v - hi)); host and
// device.
__host__ __device__ __forceinline__ dfloat df_from_double(double v) {
  const float hi = static_cast<float>(v);
  return {hi, static_cast<float>(v - static_cast<double>(hi))};
}

}  // namespace wlseno
