// FP32 <-> FP64 conversions by bit operations.  On GB300 the conversion instructions
// (F2F) issue on the FP64 pipe, a few operations per clock per SM: a kernel that converts
// every element it streams would be bound by them, not by HBM.
#pragma once

#include <cstdint>

namespace pd {

// exact FP32 -> FP64; zero and subnormal inputs give 0, Inf/NaN give NaN
__device__ __forceinline__ double f32_to_f64(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  if (e == 0xFFu) return __longlong_as_double(0x7FF8000000000000ll);
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xFFFFFu);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// x 2^s -> FP32, truncated to 24 significant bits (relative error below 2^-23): results
// below 2^-126 in magnitude (and zero or subnormal x) give 0; results of 2^128 or more,
// Inf and NaN give NaN
__device__ __forceinline__ float f64_to_f32(double x, int s = 0) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  int e = (int)((hw >> 20) & 0x7FFu);
  if (e == 0) return 0.f;
  if (e == 0x7FF) return __int_as_float(0x7FC00000);
  e += s;
  if (e < 1023 - 126) return 0.f;
  if (e > 1023 + 127) return __int_as_float(0x7FC00000);
  return __uint_as_float((hw & 0x80000000u) | ((unsigned)(e - 896) << 23) | ((hw & 0xFFFFFu) << 3) |
                         (lw >> 29));
}

// the exponent s of a power of two 2^s given as a double
__host__ __device__ __forceinline__ int pow2_exponent(double p) {
  union {
    double d;
    unsigned long long u;
  } v;
  v.d = p;
  return (int)((v.u >> 52) & 0x7FFu) - 1023;
}

}  // namespace pd
