// Double-float ("double-word") arithmetic: a real as an unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant
// bits.  GB300 runs FP32 at many times its FP64 rate, so a stencil that must
// reach FP64-level accuracy on FP32 inputs runs faster in this form.
//
// Building blocks (exact error-free transformations of IEEE binary32):
//   two_sum(a, b)      = (s, e), s = fl(a + b), a + b = s + e exactly
//                        (Knuth's branch-free form, six operations)
//   fast_two_sum(a, b) = the same for |a| >= |b| (Dekker, three operations)
//   two_prod(a, b)     = (p, e), p = fl(a b), a b = p + e exactly, e taken
//                        by one fused multiply-add
// Sums use the "sloppy" double-word addition (exact sum of the high parts,
// low parts added in FP32, renormalised): its error is a small multiple of
// 2^-48 (|x| + |y|), i.e. bounded by the operands, not by the result -- the
// same kind of bound an FP64 sum has, which is what a stencil sum needs.
// Products keep the cross terms hi lo by FMA and drop lo lo (below 2^-48).
//
// The type and its operators live in a namespace of their own so that only
// argument-dependent lookup finds them: an unqualified fma on FP32 or FP64
// arguments keeps resolving to CUDA's own.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace mglma {
namespace dfl {

struct DF {
  float hi, lo;
  __host__ __device__ DF() : hi(0.f), lo(0.f) {}
  __host__ __device__ DF(float h, float l) : hi(h), lo(l) {}
  // d split into FP32 high and low parts (within 2^-48 relative of d for d
  // inside the FP32 exponent range)
  __host__ __device__ DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ DF(int i) : DF((double)i) {}
};

// FP32 operations the compiler may neither contract into an FMA nor
// reorder (device: the _rn intrinsics; host: plain operators, built without
// contraction)
__host__ __device__ __forceinline__ float df_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float df_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float df_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

__host__ __device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = df_add(a, b);
  const float bb = df_sub(s, a);
  const float e = df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb));
  return DF(s, e);
}
__host__ __device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = df_add(a, b);
  return DF(s, df_sub(b, df_sub(s, a)));
}
__host__ __device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = df_mul(a, b);
  return DF(p, fmaf(a, b, -p));
}

__host__ __device__ __forceinline__ DF operator+(DF x, DF y) {
  const DF s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, df_add(s.lo, df_add(x.lo, y.lo)));
}
__host__ __device__ __forceinline__ DF operator-(DF x) { return DF(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ DF operator-(DF x, DF y) { return x + (-y); }
__host__ __device__ __forceinline__ DF operator*(DF x, DF y) {
  const DF p = two_prod(x.hi, y.hi);
  return fast_two_sum(p.hi, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
}
// x y + z with one renormalisation
__host__ __device__ __forceinline__ DF fma(DF x, DF y, DF z) {
  const DF p = two_prod(x.hi, y.hi);
  const DF s = two_sum(p.hi, z.hi);
  const float t = df_add(fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)), z.lo);
  return fast_two_sum(s.hi, df_add(s.lo, t));
}

// hi + lo rounded once to FP64
__host__ __device__ __forceinline__ double to_double(DF x) { return (double)x.hi + (double)x.lo; }

}  // namespace dfl
using dfl::DF;
}  // namespace mglma
