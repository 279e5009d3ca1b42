// Small complex / colour-matrix helpers for the device code.
#pragma once
#include <cuda_runtime.h>

namespace mglma {

template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cx(R a, R b) {
  Cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return cx(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return cx(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a) { return cx(-a.re, -a.im); }
template <typename R>
__device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return cx(s * a.re, s * a.im); }
template <typename R>
__device__ __forceinline__ Cx<R> conj(Cx<R> a) { return cx(a.re, -a.im); }
// i * a
template <typename R>
__device__ __forceinline__ Cx<R> mul_i(Cx<R> a) { return cx(-a.im, a.re); }
// acc += a * b
template <typename R>
__device__ __forceinline__ void cfma(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cfma_conj(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

template <typename R>
struct M3 {
  Cx<R> e[3][3];
};

template <typename R>
__device__ __forceinline__ M3<R> mul(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> s = cx<R>(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma(s, a.e[i][k], b.e[k][j]);
      c.e[i][j] = s;
    }
  return c;
}
template <typename R>
__device__ __forceinline__ M3<R> dagger(const M3<R>& a) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c.e[i][j] = conj(a.e[j][i]);
  return c;
}
template <typename R>
__device__ __forceinline__ M3<R> add(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c.e[i][j] = a.e[i][j] + b.e[i][j];
  return c;
}

}  // namespace mglma
