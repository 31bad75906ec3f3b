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
template <typename C> __device__ __forceinline__ double cabs2(C a) {
  return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

}  // namespace pd
