// Complex helpers on interleaved (re, im) pairs: double2 for FP64, float2 for FP32.
#pragma once

#include <cuda_runtime.h>

namespace pd {

__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename C> __device__ __forceinline__ C cx(decltype(C::x) re, decltype(C::x) im) {
  C r;
  r.x = re;
  r.y = im;
  return r;
}
template <typename C> __device__ __forceinline__ C czero() { return cx<C>(0, 0); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cx<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cx<C>(a.x - b.x, a.y - b.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) {
  return cx<C>(a.x * s, a.y * s);
}
// a * b
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cx<C>(fmadd(a.x, b.x, -a.y * b.y), fmadd(a.x, b.y, a.y * b.x));
}
// a * b + c
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c) {
  return cx<C>(fmadd(a.x, b.x, fmadd(-a.y, b.y, c.x)), fmadd(a.x, b.y, fmadd(a.y, b.x, c.y)));
}
// FP32 complex: element-wise operations as paired FP32 instructions (one instruction for
// both components on sm_100 and later); products keep the scalar FMA form, whose operands
// would need swapped or broadcast register pairs
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return __fadd2_rn(a, __fmul2_rn(b, make_float2(-1.f, -1.f)));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
#endif
template <typename C> __device__ __forceinline__ double cabs2(C a) {
  return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

}  // namespace pd
