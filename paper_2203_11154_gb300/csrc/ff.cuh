// Float-float (pairs of FP32) and fixed-point helpers of the residual kernels that avoid
// FP64 instructions (GB300 issues FP64 at 1/58 of its FP32 rate): the error-free
// transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the FMA product split, exact
// power-of-two scaling, FP64 bits -> float-float, FP64 bits -> three FP32 limbs of a
// fixed-point value, and packed (FP32x2) forms of the float-float operations.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace pd {
namespace ff {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// exact when a = 0 or exponent(a) >= exponent(b)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
// a * b as an unnormalised pair (p, e), p + e = a b to about 2^-47 |a b|
__device__ __forceinline__ DF df_mul_un(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return {p, __fadd_rn(__fmaf_rn(a.hi, b.hi, -p), __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi)))};
}

// 2^e as FP32 for e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// x * 2^-s for s in [-126, 252] (two exact power-of-two products; flushes below 2^-149)
__device__ __forceinline__ float scale_down(float x, int s) {
  const int a = s >> 1;
  return __fmul_rn(__fmul_rn(x, pow2f(-a)), pow2f(a - s));
}
__device__ __forceinline__ DF df_scale_down(DF x, int s) { return {scale_down(x.hi, s), scale_down(x.lo, s)}; }

// Integer -> FP32 without a conversion instruction (conversions issue on GB300's slow
// FP64 pipe): for 0 <= x < 2^23, the FP32 number with x in the mantissa of 2^23 is
// 2^23 + x exactly; subtracting 2^23 leaves x.
__device__ __forceinline__ float u23_to_float(unsigned x) {
  return __fsub_rn(__uint_as_float(0x4B000000u | x), 8388608.f);
}

// FP64 bits -> float-float: |x| >= 2^-100 kept (hi truncated to 24 bits, lo the rest,
// rounded to 24 bits), smaller values are 0; Inf/NaN give NaN
__device__ __forceinline__ DF split_bits(uint32_t hw, uint32_t lw) {
  const int e = (int)((hw >> 20) & 0x7FFu);
  if (e == 0x7FF || e > 1023 + 127) return {__int_as_float(0x7FC00000), 0.f};
  if (e < 1023 - 100) return {0.f, 0.f};
  const uint32_t sign = hw & 0x80000000u;
  const float hi = __uint_as_float(sign | ((uint32_t)(e - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  // remaining 29 bits, weight 2^(e - 1075), e - 1075 in [-152, 52]
  const int ex = e - 1075;
  const int a = ex >> 1;
  const unsigned rem = lw & 0x1FFFFFFFu;  // 29 bits = 23 high + 6 low
  const float remf = __fmaf_rn(u23_to_float(rem >> 6), 64.f, u23_to_float(rem & 63u));
  float lo = __fmul_rn(__fmul_rn(remf, pow2f(a)), pow2f(ex - a));
  if (sign) lo = -lo;
  return {hi, lo};
}

__device__ __forceinline__ DF split(double x) {
  return split_bits((uint32_t)__double2hiint(x), (uint32_t)__double2loint(x));
}

// 64-bit logical right shift; amounts of 64 and more give 0 (PTX shr clamps the amount)
__device__ __forceinline__ unsigned long long shr64(unsigned long long x, unsigned s) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}

// FP64 bits -> the three limbs of its fixed-point value in units 2^-S, S = 1081 - emax:
// v = m 2^(e - 1075 + S) = (m << 6) >> (emax - e) (m < 2^53, so m << 6 < 2^59; truncated
// below a unit), cut into 21-bit pieces t_j and made FP32 by the mantissa trick at the
// limb's own exponent: the FP32 number X_j with t_j in the mantissa of 2^(23 + 21 j) is
// 2^(23 + 21 j) + t_j 2^(21 j), and sg (X_j - 2^(23 + 21 j)) is exact (sg = +-1, the sign;
// one FMA, see limbs2 below).  Zero and subnormal inputs (e = 0) are taken with the
// implicit bit: below 2^-1022 they only matter in a tile with emax < 64, where every scaled
// coefficient is 0.  limb_bits is the integer part: the words X_j and sg.
struct LimbBits {
  uint32_t x2, x1, x0;
  float sg;
};
__device__ __forceinline__ LimbBits limb_bits(unsigned long long bits, unsigned emax) {
  const uint32_t hw = (uint32_t)(bits >> 32), lw = (uint32_t)bits;
  const unsigned e = (hw >> 20) & 0x7FFu;
  const unsigned long long m = ((unsigned long long)((hw & 0xFFFFFu) | 0x100000u) << 32) | lw;
  const unsigned long long v = shr64(m << 6, emax - e);
  const uint32_t vl = (uint32_t)v, vh = (uint32_t)(v >> 32);
  LimbBits b;
  b.x0 = (150u << 23) | (vl & 0x1FFFFFu);
  b.x1 = (171u << 23) | (__funnelshift_r(vl, vh, 21) & 0x1FFFFFu);
  b.x2 = (192u << 23) | (vh >> 10);
  b.sg = __uint_as_float((hw & 0x80000000u) | 0x3F800000u);
  return b;
}

// Packed FP32x2 arithmetic (sm_100 and later: one FADD2 / FMUL2 / FFMA2 instruction does
// the operation on both components, each rounded as its scalar form), for kernels that
// carry two independent points (or the two components of a complex value) side by side.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
struct DF2 {  // two float-float values: (hi.x, lo.x) and (hi.y, lo.y)
  float2 hi, lo;
};
__device__ __forceinline__ DF2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b), bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ DF2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ DF2 mul_un2(DF2 c, DF2 x) {
  const float2 p = mul2(c.hi, x.hi);
  return {p, add2(fma2(c.hi, x.hi, neg2(p)), fma2(c.hi, x.lo, mul2(c.lo, x.hi)))};
}
// the three limbs of two values (components x and y) from their LimbBits: sg (X_j - 2^(23 + 21 j))
struct Limbs2 {
  float2 l2, l1, l0;
};
__device__ __forceinline__ Limbs2 limbs2(const LimbBits &a, const LimbBits &b) {
  const float2 sg = make_float2(a.sg, b.sg);
  Limbs2 l;
  l.l2 = fma2(sg, make_float2(__uint_as_float(a.x2), __uint_as_float(b.x2)), mul2(sg, bc2(-0x1p65f)));
  l.l1 = fma2(sg, make_float2(__uint_as_float(a.x1), __uint_as_float(b.x1)), mul2(sg, bc2(-0x1p44f)));
  l.l0 = fma2(sg, make_float2(__uint_as_float(a.x0), __uint_as_float(b.x0)), mul2(sg, bc2(-0x1p23f)));
  return l;
}

__device__ __forceinline__ DF df_shfl_down(DF a, int o) {
  return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

}  // namespace ff
}  // namespace pd
