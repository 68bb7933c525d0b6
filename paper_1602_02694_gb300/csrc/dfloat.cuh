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

#include <cstdint>
#include <cstring>

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

// The same pair from the bits of v by integer arithmetic alone (no FP64
// instruction: on this part the FP64 pipe is the narrow one), where hi and
// lo are normal FP32 numbers (binary exponent of v in [-73, 117]) and for
// zeros; other values take df_from_double.  With v = (-1)^s (2^52 + m) 2^(e - 52): hi
// keeps the top 23 bits of m rounded to nearest, ties to even (a carry out
// of the mantissa moves into the exponent field, as it should); the
// remainder r = (m mod 2^29) - 2^29 [rounded up] is v - hi in units of
// 2^(e - 52), an integer of at most 29 bits, so fl32(v - hi) is the
// round-to-nearest conversion of r times an exact power of two.  The
// result equals df_from_double(v) bit for bit.
__host__ __device__ __forceinline__ dfloat df_from_double_bits(double v) {
  uint64_t b;
  std::memcpy(&b, &v, sizeof b);
  const uint32_t hw = static_cast<uint32_t>(b >> 32);
  const int E = static_cast<int>((hw >> 20) & 0x7ffu);
  if ((b << 1) == 0) {  // +-0: (+-0, +0)
    const uint32_t zb = hw & 0x80000000u;
    float z;
    std::memcpy(&z, &zb, sizeof z);
    return {z, 0.0f};
  }
  if (E < 950 || E > 1140) return df_from_double(v);
  const uint32_t top = static_cast<uint32_t>(b >> 29) & 0x7fffffu;
  const uint32_t rem = static_cast<uint32_t>(b) & 0x1fffffffu;
  const uint32_t up = (rem > 0x10000000u || (rem == 0x10000000u && (top & 1u))) ? 1u : 0u;
  const uint32_t sign = hw & 0x80000000u;
  const uint32_t hb = (sign | (static_cast<uint32_t>(E - 896) << 23) | top) + up;
  const int32_t r = static_cast<int32_t>(rem) - static_cast<int32_t>(up << 29);
  const uint32_t sb = static_cast<uint32_t>(E - 948) << 23;  // 2^(e - 52)
  float hi, scale;
  std::memcpy(&hi, &hb, sizeof hi);
  std::memcpy(&scale, &sb, sizeof scale);
  return {hi, static_cast<float>(sign ? -r : r) * scale};
}

// The bits of the FP64 value of a non-negative FP32 number s (a maximum
// taken on FP64 bit patterns), by integer arithmetic for zero, infinity and
// normal s (exponent rebiased by 1023 - 127, mantissa moved up 29 bits);
// subnormal s and NaN take the conversion.
__host__ __device__ __forceinline__ uint64_t df_f64_bits_nonneg(float s) {
  uint32_t fb;
  std::memcpy(&fb, &s, sizeof fb);
  if (fb == 0u) return 0ull;
  if (fb == 0x7f800000u) return 0x7ff0000000000000ull;
  if (fb >= 0x00800000u && fb < 0x7f800000u) return (static_cast<uint64_t>(fb) + (896ull << 23)) << 29;
  const double d = static_cast<double>(s);
  uint64_t db;
  std::memcpy(&db, &d, sizeof db);
  return db;
}

}  // namespace wlseno
