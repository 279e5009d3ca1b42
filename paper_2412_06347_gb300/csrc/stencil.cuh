// Device building blocks of the Wilson-clover stencil shared by the kernels
// of dslash.cu (full lattice) and evenodd.cu (even-odd halves): spinor,
// link and clover loads in the device layouts of internal.h, the packed
// Hermitian clover blocks, spin projection and the hop term
//     (1 + s gamma_mu) W psi,  W = U_mu(x) or U_mu(x - mu)^dag,
// in the chiral basis gamma_mu = [[0, e_mu], [e_mu^dag, 0]] with e_0 = -1,
// e_k = -i sigma_k: (1 + s gamma_mu) psi has upper half h = u + s e_mu l and
// lower half s e_mu^dag h (u, l: spins {0,1}, {2,3}), so each hop moves one
// two-spin half spinor through the link.
#pragma once
#include <cuda_bf16.h>

#include "cplx.cuh"
#include "df.cuh"
#include "internal.h"
#include "lattice.cuh"

namespace mglma {

// ------------------------------------------------------------ spinor IO
template <typename R>
struct IO;

template <>
struct IO<float> {
  __device__ __forceinline__ static void load(const void* base, int64_t V, int rhs, int64_t site, Cx<float> s[12]) {
    const float4* p = reinterpret_cast<const float4*>(base) + (size_t)rhs * 6 * V + site;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float4 v = __ldg(p + j * V);
      s[2 * j] = cx(v.x, v.y);
      s[2 * j + 1] = cx(v.z, v.w);
    }
  }
  __device__ __forceinline__ static void store(void* base, int64_t V, int rhs, int64_t site, const Cx<float> s[12]) {
    float4* p = reinterpret_cast<float4*>(base) + (size_t)rhs * 6 * V + site;
#pragma unroll
    for (int j = 0; j < 6; ++j) p[j * V] = make_float4(s[2 * j].re, s[2 * j].im, s[2 * j + 1].re, s[2 * j + 1].im);
  }
};

template <>
struct IO<double> {
  __device__ __forceinline__ static void load(const void* base, int64_t V, int rhs, int64_t site, Cx<double> s[12]) {
    const double2* p = reinterpret_cast<const double2*>(base) + (size_t)rhs * 12 * V + site;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      double2 v = __ldg(p + j * V);
      s[j] = cx(v.x, v.y);
    }
  }
  __device__ __forceinline__ static void store(void* base, int64_t V, int rhs, int64_t site, const Cx<double> s[12]) {
    double2* p = reinterpret_cast<double2*>(base) + (size_t)rhs * 12 * V + site;
#pragma unroll
    for (int j = 0; j < 12; ++j) p[j * V] = make_double2(s[j].re, s[j].im);
  }
};

// ------------------------------------------------------------ spinor storage
// Storage of a spinor field, computed on in FP32 or FP64: float ([rhs][6][V]
// float4), double ([rhs][12][V] double2) or SpinBf16 ([rhs][3][V] uint4, each
// holding four complex components as (re, im) BF16 pairs, re in the low half)
struct SpinBf16 {};

__device__ __forceinline__ Cx<float> bf16_unpack(uint32_t u) {
  return cx(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
__device__ __forceinline__ uint32_t bf16_pack(Cx<float> a) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a.re, a.im);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <typename S>
struct SIO;
template <>
struct SIO<float> {
  using R = float;
  __device__ __forceinline__ static void load(const void* b, int64_t V, int rhs, int64_t site, Cx<float> s[12]) {
    IO<float>::load(b, V, rhs, site, s);
  }
  __device__ __forceinline__ static void store(void* b, int64_t V, int rhs, int64_t site, const Cx<float> s[12]) {
    IO<float>::store(b, V, rhs, site, s);
  }
};
template <>
struct SIO<double> {
  using R = double;
  __device__ __forceinline__ static void load(const void* b, int64_t V, int rhs, int64_t site, Cx<double> s[12]) {
    IO<double>::load(b, V, rhs, site, s);
  }
  __device__ __forceinline__ static void store(void* b, int64_t V, int rhs, int64_t site, const Cx<double> s[12]) {
    IO<double>::store(b, V, rhs, site, s);
  }
};
template <>
struct SIO<SpinBf16> {
  using R = float;
  __device__ __forceinline__ static void load(const void* b, int64_t V, int rhs, int64_t site, Cx<float> s[12]) {
    const uint4* p = reinterpret_cast<const uint4*>(b) + (size_t)rhs * 3 * V + site;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint4 v = __ldg(p + j * V);
      s[4 * j] = bf16_unpack(v.x);
      s[4 * j + 1] = bf16_unpack(v.y);
      s[4 * j + 2] = bf16_unpack(v.z);
      s[4 * j + 3] = bf16_unpack(v.w);
    }
  }
  __device__ __forceinline__ static void store(void* b, int64_t V, int rhs, int64_t site, const Cx<float> s[12]) {
    uint4* p = reinterpret_cast<uint4*>(b) + (size_t)rhs * 3 * V + site;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      p[j * V] = make_uint4(bf16_pack(s[4 * j]), bf16_pack(s[4 * j + 1]), bf16_pack(s[4 * j + 2]),
                            bf16_pack(s[4 * j + 3]));
  }
};

// FP32 spinor storage computed on in double-float (each value exact)
struct SpinF32Df {};
template <>
struct SIO<SpinF32Df> {
  using R = DF;
  __device__ __forceinline__ static void load(const void* b, int64_t V, int rhs, int64_t site, Cx<DF> s[12]) {
    Cx<float> f[12];
    IO<float>::load(b, V, rhs, site, f);
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = cx(DF(f[k].re, 0.f), DF(f[k].im, 0.f));
  }
};
// output of the double-float residual update: out (FP64 spinors) -=
// scale[rhs] op(in), op(in) rounded once to FP64 per component
struct ResidF64 {};

// ------------------------------------------------------------ links
template <typename R>
struct Link;

template <>
struct Link<float> {  // reconstruct-12
  __device__ __forceinline__ static void load(const void* U, int64_t V, int mu, int64_t site, M3<float>& m) {
    const float4* p = reinterpret_cast<const float4*>(U) + (size_t)mu * 3 * V + site;
    float4 a = __ldg(p), b = __ldg(p + V), c = __ldg(p + 2 * V);
    m.e[0][0] = cx(a.x, a.y);
    m.e[0][1] = cx(a.z, a.w);
    m.e[0][2] = cx(b.x, b.y);
    m.e[1][0] = cx(b.z, b.w);
    m.e[1][1] = cx(c.x, c.y);
    m.e[1][2] = cx(c.z, c.w);
    // row2 = conj(row0 x row1)
    m.e[2][0] = conj(m.e[0][1] * m.e[1][2] - m.e[0][2] * m.e[1][1]);
    m.e[2][1] = conj(m.e[0][2] * m.e[1][0] - m.e[0][0] * m.e[1][2]);
    m.e[2][2] = conj(m.e[0][0] * m.e[1][1] - m.e[0][1] * m.e[1][0]);
  }
};

template <>
struct Link<double> {  // full 18 reals
  __device__ __forceinline__ static void load(const void* U, int64_t V, int mu, int64_t site, M3<double>& m) {
    const double2* p = reinterpret_cast<const double2*>(U) + (size_t)mu * 9 * V + site;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = __ldg(p + k * V);
      m.e[k / 3][k % 3] = cx(v.x, v.y);
    }
  }
};

// double-float links: the FP64 links split once ([mu][9][V] float4 =
// (re.hi, re.lo, im.hi, im.lo))
template <>
struct Link<DF> {
  __device__ __forceinline__ static void load(const void* U, int64_t V, int mu, int64_t site, M3<DF>& m) {
    const float4* p = reinterpret_cast<const float4*>(U) + (size_t)mu * 9 * V + site;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 v = __ldg(p + k * V);
      m.e[k / 3][k % 3] = cx(DF(v.x, v.y), DF(v.z, v.w));
    }
  }
};

// ------------------------------------------------------------ clover blocks
// packed Hermitian 6x6: 6 real diagonals, then 15 (re, im) upper entries
__device__ __forceinline__ int offdiag_slot(int i, int j) {  // i < j
  // row-major position of (i, j) among the 15 upper entries
  return i * 5 - (i * (i - 1)) / 2 + (j - i - 1);
}

template <typename R>
struct Clover;

template <>
struct Clover<float> {
  __device__ __forceinline__ static void load(const void* C, int64_t V, int chi, int64_t site, float c[36]) {
    const float4* p = reinterpret_cast<const float4*>(C) + (size_t)chi * 9 * V + site;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      float4 v = __ldg(p + j * V);
      c[4 * j] = v.x;
      c[4 * j + 1] = v.y;
      c[4 * j + 2] = v.z;
      c[4 * j + 3] = v.w;
    }
  }
};
template <>
struct Clover<double> {
  __device__ __forceinline__ static void load(const void* C, int64_t V, int chi, int64_t site, double c[36]) {
    const double2* p = reinterpret_cast<const double2*>(C) + (size_t)chi * 18 * V + site;
#pragma unroll
    for (int j = 0; j < 18; ++j) {
      double2 v = __ldg(p + j * V);
      c[2 * j] = v.x;
      c[2 * j + 1] = v.y;
    }
  }
};

// double-float clover: the FP64 packed blocks split once ([chi][18][V]
// float4 = two reals as (hi, lo) pairs)
template <>
struct Clover<DF> {
  __device__ __forceinline__ static void load(const void* C, int64_t V, int chi, int64_t site, DF c[36]) {
    const float4* p = reinterpret_cast<const float4*>(C) + (size_t)chi * 18 * V + site;
#pragma unroll
    for (int j = 0; j < 18; ++j) {
      const float4 v = __ldg(p + j * V);
      c[2 * j] = DF(v.x, v.y);
      c[2 * j + 1] = DF(v.z, v.w);
    }
  }
};

// out[i] (+)= sum_j A_ij in[j] for one packed Hermitian 6x6 block
template <typename R>
__device__ __forceinline__ void clover_apply6(const R c[36], const Cx<R>* in, Cx<R>* out) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    Cx<R> s = c[i] * in[i];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (j == i) continue;
      if (i < j) {
        int k = 6 + 2 * offdiag_slot(i, j);
        cfma(s, cx(c[k], c[k + 1]), in[j]);
      } else {
        int k = 6 + 2 * offdiag_slot(j, i);
        cfma_conj(s, cx(c[k], c[k + 1]), in[j]);
      }
    }
    out[i] = s;
  }
}

// ------------------------------------------------------------ spin projection
// i sigma_k applied to a two-spin half spinor (a, b), per colour
template <typename R>
__device__ __forceinline__ void isigma(int k, const Cx<R> a[3], const Cx<R> b[3], Cx<R> o0[3], Cx<R> o1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (k == 1) {
      o0[c] = mul_i(b[c]);
      o1[c] = mul_i(a[c]);
    } else if (k == 2) {
      o0[c] = b[c];
      o1[c] = -a[c];
    } else {
      o0[c] = mul_i(a[c]);
      o1[c] = -mul_i(b[c]);
    }
  }
}

// h = upper half of (1 + s gamma_mu) psi;  psi[spin*3 + colour]
template <typename R>
__device__ __forceinline__ void project(int mu, R s, const Cx<R> psi[12], Cx<R> h0[3], Cx<R> h1[3]) {
  if (mu == 0) {  // e_0 = -1: h = u - s l
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = psi[c] - s * psi[6 + c];
      h1[c] = psi[3 + c] - s * psi[9 + c];
    }
  } else {  // e_k = -i sigma_k: h = u - s (i sigma_k) l
    Cx<R> t0[3], t1[3];
    isigma<R>(mu, psi + 6, psi + 9, t0, t1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = psi[c] - s * t0[c];
      h1[c] = psi[3 + c] - s * t1[c];
    }
  }
}

// acc += (h, s e_mu^dag h)
template <typename R>
__device__ __forceinline__ void reconstruct_add(int mu, R s, const Cx<R> h0[3], const Cx<R> h1[3], Cx<R> acc[12]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = acc[c] + h0[c];
    acc[3 + c] = acc[3 + c] + h1[c];
  }
  if (mu == 0) {  // e_0^dag = -1
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[6 + c] = acc[6 + c] - s * h0[c];
      acc[9 + c] = acc[9 + c] - s * h1[c];
    }
  } else {  // e_k^dag = i sigma_k
    Cx<R> t0[3], t1[3];
    isigma<R>(mu, h0, h1, t0, t1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[6 + c] = acc[6 + c] + s * t0[c];
      acc[9 + c] = acc[9 + c] + s * t1[c];
    }
  }
}

template <typename R>
__device__ __forceinline__ void mat_vec(const M3<R>& U, const Cx<R> h[3], Cx<R> o[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> s = cx<R>(0, 0);
#pragma unroll
    for (int b = 0; b < 3; ++b) cfma(s, U.e[a][b], h[b]);
    o[a] = s;
  }
}
template <typename R>
__device__ __forceinline__ void mat_dag_vec(const M3<R>& U, const Cx<R> h[3], Cx<R> o[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> s = cx<R>(0, 0);
#pragma unroll
    for (int b = 0; b < 3; ++b) cfma_conj(s, U.e[b][a], h[b]);
    o[a] = s;
  }
}

// one hop term: acc += f * (1 + s gamma_mu) W psi, W = U (fwd) or U^dag (bwd)
template <typename R, bool FWD>
__device__ __forceinline__ void hop_add(int mu, R s, R f, const M3<R>& U, const Cx<R> psi[12], Cx<R> acc[12]) {
  Cx<R> h0[3], h1[3], g0[3], g1[3];
  project<R>(mu, s, psi, h0, h1);
  if (FWD) {
    mat_vec<R>(U, h0, g0);
    mat_vec<R>(U, h1, g1);
  } else {
    mat_dag_vec<R>(U, h0, g0);
    mat_dag_vec<R>(U, h1, g1);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g0[c] = f * g0[c];
    g1[c] = f * g1[c];
  }
  reconstruct_add<R>(mu, s, g0, g1, acc);
}

struct DslashArgs {
  LatIdx q;
  double bc;
  int nrhs;
  int g5out;
  const void* bsub = nullptr;  // dslash_kernel: when set, out = bsub - op(in) (same layout as out)
  const double* scale = nullptr;  // ResidF64 output: per-RHS factor of op(in)
};

}  // namespace mglma
