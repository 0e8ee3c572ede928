// Complex helpers for float2 / double2 (interleaved re, im).
#pragma once
#include <cuda_runtime.h>

namespace chi0 {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename C> __host__ __device__ __forceinline__ C cmk(double re, double im);
template <> __host__ __device__ __forceinline__ float2 cmk<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __host__ __device__ __forceinline__ double2 cmk<double2>(double re, double im) {
  return make_double2(re, im);
}

__device__ __forceinline__ float2 cz(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 cz(double2) { return make_double2(0.0, 0.0); }

// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// conj(a) * b
template <typename C> __device__ __forceinline__ C cconjmul(C a, C b) {
  C r;
  r.x = fma(a.x, b.x, a.y * b.y);
  r.y = fma(a.x, b.y, -(a.y * b.x));
  return r;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = fma(a.x, b.x, -(a.y * b.y));
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

__device__ __forceinline__ float2 to_c(double2 v, float2) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_c(double2 v, double2) { return v; }

}  // namespace chi0
