// Multi-RHS BLAS-1 for the Krylov solvers.
//
// A vector batch is nrhs contiguous blocks of n reals ((re, im) pairs); every
// scalar is per RHS and stays in device memory, so a solver iteration issues
// kernels back to back without reading anything on the host.  Reductions
// accumulate in FP64 (for FP32 data: an FP32 partial over one 16-byte load,
// then FP64) in a fixed two-stage order, so results are bitwise reproducible
// and independent of how RHS are grouped.
#include "internal.h"
#include "minres.cuh"


namespace mglma {

// --------------------------------------------------------------- element access
template <typename R>
struct Pair;  // a 16-byte load: 2 complex (FP32) or 1 complex (FP64)
template <>
struct Pair<float> {
  static constexpr int kCplx = 2;
  using T = float4;
};
template <>
struct Pair<double> {
  static constexpr int kCplx = 1;
  using T = double2;
};

__device__ __forceinline__ float4 lc(float4 x, float4 y, double2 a, double2 b) {
  // a*x + b*y (complex a, b; x, y hold 2 complex each)
  const float ar = (float)a.x, ai = (float)a.y, br = (float)b.x, bi = (float)b.y;
  float4 o;
  o.x = ar * x.x - ai * x.y + br * y.x - bi * y.y;
  o.y = ar * x.y + ai * x.x + br * y.y + bi * y.x;
  o.z = ar * x.z - ai * x.w + br * y.z - bi * y.w;
  o.w = ar * x.w + ai * x.z + br * y.w + bi * y.z;
  return o;
}
__device__ __forceinline__ double2 lc(double2 x, double2 y, double2 a, double2 b) {
  double2 o;
  o.x = a.x * x.x - a.y * x.y + b.x * y.x - b.y * y.y;
  o.y = a.x * x.y + a.y * x.x + b.x * y.y + b.y * y.x;
  return o;
}

// y_r = a_r x_r + b_r y_r (complex, per RHS; a NULL uses a_def, b NULL uses
// b_def); sgn scales a.
template <typename R>
__global__ void axpby_kernel(const typename Pair<R>::T* __restrict__ x, typename Pair<R>::T* __restrict__ y,
                             const double2* __restrict__ a, double2 a_def, const double2* __restrict__ b,
                             double2 b_def, size_t m, double sgn) {
  const int r = blockIdx.y;
  double2 ar = a ? a[r] : a_def;
  ar.x *= sgn;
  ar.y *= sgn;
  const double2 br = b ? b[r] : b_def;
  const auto* xr = x + (size_t)r * m;
  auto* yr = y + (size_t)r * m;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    yr[i] = lc(xr[i], yr[i], ar, br);
}

// x += a p ; r -= a w   (CG / GCR / MR update pair; p may alias r)
template <typename R>
__global__ void axpy2_kernel(const typename Pair<R>::T* p, typename Pair<R>::T* x, const typename Pair<R>::T* w,
                             typename Pair<R>::T* res, const double2* __restrict__ a, size_t m) {
  const int r = blockIdx.y;
  const double2 ar = a[r];
  const double2 na = make_double2(-ar.x, -ar.y);
  const double2 one = make_double2(1, 0);
  const size_t off = (size_t)r * m;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    const auto pv = p[off + i], xv = x[off + i], wv = w[off + i], rv = res[off + i];
    x[off + i] = lc(pv, xv, ar, one);
    res[off + i] = lc(wv, rv, na, one);
  }
}

// y_r -= sum_{j<k} c[j][r] x_j,r  with x_j = x0 + j * jstride (vectors); a
// second pair (x0b, yb) with the same coefficients is updated in the same
// pass when given (the GCR directions and their images).  The block's
// coefficients sit in shared memory.
template <typename R>
__global__ void multi_axpy_kernel(const typename Pair<R>::T* __restrict__ x0, typename Pair<R>::T* __restrict__ y,
                                  const typename Pair<R>::T* __restrict__ x0b, typename Pair<R>::T* __restrict__ yb,
                                  size_t jstride, int k, const double2* __restrict__ c, int nrhs, size_t m) {
  __shared__ double2 cs[64];
  const int r = blockIdx.y;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double2 v = c[(size_t)j * nrhs + r];
    cs[j] = make_double2(-v.x, -v.y);
  }
  __syncthreads();
  const size_t off = (size_t)r * m;
  const double2 one = make_double2(1, 0);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    auto acc = y[off + i];
    for (int j = 0; j < k; ++j) acc = lc(x0[j * jstride + off + i], acc, cs[j], one);
    y[off + i] = acc;
    if (yb) {
      auto accb = yb[off + i];
      for (int j = 0; j < k; ++j) accb = lc(x0b[j * jstride + off + i], accb, cs[j], one);
      yb[off + i] = accb;
    }
  }
}

// ------------------------------------------------------------- reductions
__device__ __forceinline__ double2 dot_pair(float4 a, float4 b) {
  // conj(a) . b over 2 complex, FP32 partial
  float re = a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
  float im = a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
  return make_double2(re, im);
}
__device__ __forceinline__ double2 dot_pair(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double nrm_pair(float4 a) { return (double)(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w); }
__device__ __forceinline__ double nrm_pair(double2 a) { return a.x * a.x + a.y * a.y; }

template <int NT>
__device__ __forceinline__ double2 block_sum2(double2 v) {
  __shared__ double2 sh[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < NT / 32 ? sh[l] : make_double2(0, 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
  }
  __syncthreads();
  return v;
}

constexpr int RT = 256;  // reduction threads per block

// One launch per reduction: every block writes its partial, the last block
// of each RHS (atomic ticket) adds the partials in block order and writes the
// result, then resets the ticket.  Results do not depend on timing.
// MODE 0: |x|^2 -> out1[r]; 1: <x_j, y> for j < k -> out2[j*n + r];
// 2: |x|^2 -> out1[r] and <x, y> -> out2[r].
template <int MODE>
__device__ __forceinline__ bool finish(double2* part, unsigned* count, int k, int nb, int nrhs, double2* out2,
                                       double* out1) {
  __shared__ bool last;
  const int r = blockIdx.y;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(count + r, 1u) == (unsigned)(nb - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int nslot = MODE == 2 ? 2 : k;
  for (int j = 0; j < nslot; ++j) {
    double2 acc = make_double2(0, 0);
    const double2* pj = part + ((size_t)j * nrhs + r) * nb;
    for (int i = threadIdx.x; i < nb; i += RT) {
      const double2 v = __ldcg(pj + i);
      acc.x += v.x;
      acc.y += v.y;
    }
    acc = block_sum2<RT>(acc);
    if (threadIdx.x == 0) {
      if (MODE == 0) out1[r] = acc.x;
      if (MODE == 1) out2[(size_t)j * nrhs + r] = acc;
      if (MODE == 2) {
        if (j == 0) out1[r] = acc.x;
        else out2[r] = acc;
      }
    }
  }
  if (threadIdx.x == 0) count[r] = 0;
  return true;
}

// FP32 data: products of one 16-byte load are summed in FP32, sixteen loads
// are gathered in an FP32 partial, and only that partial enters the FP64
// accumulator (keeps the FP64 pipe, which is narrow on GB300, off the
// critical path).  FP64 data accumulate in FP64 throughout.
template <typename R>
struct RAcc;
template <>
struct RAcc<float> {
  float n = 0.f, dr = 0.f, di = 0.f;
  int c = 0;
  double N = 0, DR = 0, DI = 0;
  __device__ __forceinline__ void add_n(float4 a) {
    n += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
    tick();
  }
  __device__ __forceinline__ void add_d(float4 a, float4 b) {
    dr += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    di += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
    tick();
  }
  __device__ __forceinline__ void add_nd(float4 a, float4 b) {
    n += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
    dr += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    di += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
    tick();
  }
  __device__ __forceinline__ void tick() {
    if (++c == 16) flush();
  }
  __device__ __forceinline__ void flush() {
    N += n;
    DR += dr;
    DI += di;
    n = dr = di = 0.f;
    c = 0;
  }
  __device__ __forceinline__ double norm() {
    flush();
    return N;
  }
  __device__ __forceinline__ double2 dot() {
    flush();
    return make_double2(DR, DI);
  }
};
template <>
struct RAcc<double> {
  double N = 0, DR = 0, DI = 0;
  __device__ __forceinline__ void add_n(double2 a) { N += a.x * a.x + a.y * a.y; }
  __device__ __forceinline__ void add_d(double2 a, double2 b) {
    DR += a.x * b.x + a.y * b.y;
    DI += a.x * b.y - a.y * b.x;
  }
  __device__ __forceinline__ void add_nd(double2 a, double2 b) {
    add_n(a);
    add_d(a, b);
  }
  __device__ __forceinline__ double norm() { return N; }
  __device__ __forceinline__ double2 dot() { return make_double2(DR, DI); }
};

// Grid-stride loops over 16-byte loads.  JM accumulators per pass over y
// (MODE 1) keep the register count, and so the occupancy, low for the usual
// one to four directions.
template <typename R, int MODE, int JM>
__global__ void __launch_bounds__(RT) reduce_kernel(const typename Pair<R>::T* __restrict__ x0, size_t jstride, int k,
                                                    const typename Pair<R>::T* __restrict__ y, size_t m,
                                                    double2* __restrict__ part, unsigned* __restrict__ count,
                                                    double2* out2, double* out1) {
  const int r = blockIdx.y, nrhs = gridDim.y, nb = gridDim.x;
  const size_t off = (size_t)r * m;
  const size_t step = (size_t)nb * RT;
  if (MODE == 1) {
    // directions in chunks of up to JM per pass over y
    for (int j0 = 0; j0 < k; j0 += JM) {
      const int nj = min(JM, k - j0);
      RAcc<R> acc[JM];
      for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < m; i += step) {
        const auto yv = y[off + i];
#pragma unroll
        for (int jj = 0; jj < JM; ++jj)
          if (jj < nj) acc[jj].add_d(x0[(j0 + jj) * jstride + off + i], yv);
      }
#pragma unroll
      for (int jj = 0; jj < JM; ++jj) {
        if (jj >= nj) break;
        const double2 v = block_sum2<RT>(acc[jj].dot());
        if (threadIdx.x == 0) part[((size_t)(j0 + jj) * nrhs + r) * nb + blockIdx.x] = v;
      }
    }
  } else {
    RAcc<R> acc;
    const auto* x = x0 + off;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < m; i += step) {
      if (MODE == 2)
        acc.add_nd(x[i], y[off + i]);
      else
        acc.add_n(x[i]);
    }
    const double nn = acc.norm();
    const double2 dd = MODE == 2 ? acc.dot() : make_double2(0, 0);
    double2 v = block_sum2<RT>(make_double2(nn, 0));
    if (threadIdx.x == 0) part[(size_t)r * nb + blockIdx.x] = v;
    if (MODE == 2) {
      v = block_sum2<RT>(dd);
      if (threadIdx.x == 0) part[((size_t)nrhs + r) * nb + blockIdx.x] = v;
    }
  }
  finish<MODE>(part, count, k, nb, nrhs, out2, out1);
}

// x += a p ; r -= a w ; out1 = |r|^2 (fused GCR / CG update with the new norm)
template <typename R>
__global__ void __launch_bounds__(RT) axpy2_norm_kernel(const typename Pair<R>::T* p, typename Pair<R>::T* x,
                                                        const typename Pair<R>::T* w, typename Pair<R>::T* res,
                                                        const double2* __restrict__ a, size_t m,
                                                        double2* __restrict__ part, unsigned* __restrict__ count,
                                                        double* out1) {
  const int r = blockIdx.y, nrhs = gridDim.y, nb = gridDim.x;
  const double2 ar = a[r];
  const double2 na = make_double2(-ar.x, -ar.y);
  const double2 one = make_double2(1, 0);
  const size_t off = (size_t)r * m;
  RAcc<R> acc;
  for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < m; i += (size_t)nb * RT) {
    const auto pv = p[off + i], xv = x[off + i], wv = w[off + i], rv = res[off + i];
    x[off + i] = lc(pv, xv, ar, one);
    const auto nr = lc(wv, rv, na, one);
    res[off + i] = nr;
    acc.add_n(nr);
  }
  const double2 v = block_sum2<RT>(make_double2(acc.norm(), 0));
  if (threadIdx.x == 0) part[(size_t)r * nb + blockIdx.x] = v;
  finish<0>(part, count, 1, nb, nrhs, nullptr, out1);
}

// r -= a w ; out1 = |r|^2 (GCR residual update when the iterate is formed later)
template <typename R>
__global__ void __launch_bounds__(RT) axpy_norm_kernel(const typename Pair<R>::T* w, typename Pair<R>::T* res,
                                                       const double2* __restrict__ a, size_t m,
                                                       double2* __restrict__ part, unsigned* __restrict__ count,
                                                       double* out1) {
  const int r = blockIdx.y, nrhs = gridDim.y, nb = gridDim.x;
  const double2 ar = a[r];
  const double2 na = make_double2(-ar.x, -ar.y);
  const double2 one = make_double2(1, 0);
  const size_t off = (size_t)r * m;
  RAcc<R> acc;
  for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < m; i += (size_t)nb * RT) {
    const auto nr = lc(w[off + i], res[off + i], na, one);
    res[off + i] = nr;
    acc.add_n(nr);
  }
  const double2 v = block_sum2<RT>(make_double2(acc.norm(), 0));
  if (threadIdx.x == 0) part[(size_t)r * nb + blockIdx.x] = v;
  finish<0>(part, count, 1, nb, nrhs, nullptr, out1);
}

// y_r -= sum_{j<k} c[j][r] x_j,r (and yb from x0b with the same
// coefficients), as multi_axpy, with out1 = |y_new|^2 and out2 = <y_new, w>
// = sum conj(y_new) w per RHS reduced in the same pass (GCR: the
// orthogonalised image, its norm and its overlap with the residual)
template <typename R>
__global__ void __launch_bounds__(RT) multi_axpy_nd_kernel(const typename Pair<R>::T* __restrict__ x0,
                                                           typename Pair<R>::T* __restrict__ y,
                                                           const typename Pair<R>::T* __restrict__ x0b,
                                                           typename Pair<R>::T* __restrict__ yb, size_t jstride, int k,
                                                           const double2* __restrict__ c,
                                                           const typename Pair<R>::T* __restrict__ w, size_t m,
                                                           double2* __restrict__ part, unsigned* __restrict__ count,
                                                           double2* out2, double* out1) {
  __shared__ double2 cs[64];
  const int r = blockIdx.y, nrhs = gridDim.y, nb = gridDim.x;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double2 v = c[(size_t)j * nrhs + r];
    cs[j] = make_double2(-v.x, -v.y);
  }
  __syncthreads();
  const size_t off = (size_t)r * m;
  const double2 one = make_double2(1, 0);
  RAcc<R> acc;
  for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < m; i += (size_t)nb * RT) {
    auto v = y[off + i];
    for (int j = 0; j < k; ++j) v = lc(x0[j * jstride + off + i], v, cs[j], one);
    y[off + i] = v;
    if (yb) {
      auto vb = yb[off + i];
      for (int j = 0; j < k; ++j) vb = lc(x0b[j * jstride + off + i], vb, cs[j], one);
      yb[off + i] = vb;
    }
    acc.add_nd(v, w[off + i]);
  }
  double2 v = block_sum2<RT>(make_double2(acc.norm(), 0));
  if (threadIdx.x == 0) part[(size_t)r * nb + blockIdx.x] = v;
  v = block_sum2<RT>(acc.dot());
  if (threadIdx.x == 0) part[((size_t)nrhs + r) * nb + blockIdx.x] = v;
  finish<2>(part, count, 1, nb, nrhs, out2, out1);
}

// ------------------------------------------------------------- MINRES (real scalars)
__device__ __forceinline__ float4 rlc3(float4 x, float4 y, float4 z, double a, double b, double c) {
  const float fa = (float)a, fb = (float)b, fc = (float)c;
  return make_float4(fa * x.x + fb * y.x + fc * z.x, fa * x.y + fb * y.y + fc * z.y, fa * x.z + fb * y.z + fc * z.z,
                     fa * x.w + fb * y.w + fc * z.w);
}
__device__ __forceinline__ double2 rlc3(double2 x, double2 y, double2 z, double a, double b, double c) {
  return make_double2(a * x.x + b * y.x + c * z.x, a * x.y + b * y.y + c * z.y);
}
__device__ __forceinline__ float4 rlc2(float4 x, float4 y, double a, double b) {
  const float fa = (float)a, fb = (float)b;
  return make_float4(fa * x.x + fb * y.x, fa * x.y + fb * y.y, fa * x.z + fb * y.z, fa * x.w + fb * y.w);
}
__device__ __forceinline__ double2 rlc2(double2 x, double2 y, double a, double b) {
  return make_double2(a * x.x + b * y.x, a * x.y + b * y.y);
}
__device__ __forceinline__ float4 rscale(float4 x, double a) {
  const float f = (float)a;
  return make_float4(f * x.x, f * x.y, f * x.z, f * x.w);
}
__device__ __forceinline__ double2 rscale(double2 x, double a) { return make_double2(a * x.x, a * x.y); }

// Lanczos step z -= a_r v + b_r u with a_r = Re dot[r], b_r = beta[r], and
// out1[r] = |z_r|^2; RHS with active[r] == 0 are left alone (out1 = 0).
// With st, the last block of each RHS then runs that RHS's MINRES scalar
// step (minres.cuh; out1 must be its MR_BN2 slot).
template <typename R>
__global__ void __launch_bounds__(RT) lanczos_norm_kernel(const typename Pair<R>::T* __restrict__ v,
                                                          const typename Pair<R>::T* __restrict__ u,
                                                          typename Pair<R>::T* __restrict__ z,
                                                          const double2* __restrict__ dot,
                                                          const double* __restrict__ beta,
                                                          const int* active, size_t m,
                                                          double2* __restrict__ part, unsigned* __restrict__ count,
                                                          double* out1, double* st, double tol, int cap,
                                                          int* act) {
  const int r = blockIdx.y, nrhs = gridDim.y, nb = gridDim.x;
  const bool on = active[r] != 0;
  const double a = on ? -dot[r].x : 0.0, b = on ? -beta[r] : 0.0;
  const size_t off = (size_t)r * m;
  RAcc<R> acc;
  for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < m; i += (size_t)nb * RT) {
    if (on) {
      const auto nz = rlc3(z[off + i], v[off + i], u[off + i], 1.0, a, b);
      z[off + i] = nz;
      acc.add_n(nz);
    }
  }
  const double2 t = block_sum2<RT>(make_double2(acc.norm(), 0));
  if (threadIdx.x == 0) part[(size_t)r * nb + blockIdx.x] = t;
  if (finish<0>(part, count, 1, nb, nrhs, nullptr, out1) && st && threadIdx.x == 0)
    minres_scalar_step(st, dot, act, tol, cap, r);
}

// w_new = cf0 v + cf1 w1 + cf2 w2 ; x += cf3 w_new ; z *= cf4, for RHS with
// cf5 != 0 (cf_j[r] = cf[j * stride + r])
template <typename R>
__global__ void minres_update_kernel(const typename Pair<R>::T* __restrict__ v, const typename Pair<R>::T* __restrict__ w1,
                                     const typename Pair<R>::T* __restrict__ w2, typename Pair<R>::T* __restrict__ wn,
                                     typename Pair<R>::T* __restrict__ x, typename Pair<R>::T* __restrict__ z,
                                     const double* __restrict__ cf, int stride, size_t m) {
  const int r = blockIdx.y;
  if (cf[5 * (size_t)stride + r] == 0.0) return;
  const double c0 = cf[r], c1 = cf[stride + r], c2 = cf[2 * (size_t)stride + r], c3 = cf[3 * (size_t)stride + r],
               c4 = cf[4 * (size_t)stride + r];
  const size_t off = (size_t)r * m;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    const auto w = rlc3(v[off + i], w1[off + i], w2[off + i], c0, c1, c2);
    wn[off + i] = w;
    x[off + i] = rlc2(x[off + i], w, 1.0, c3);
    z[off + i] = rscale(z[off + i], c4);
  }
}

// y_r = scale_r gamma5hat x_r on coarse fields (complex e of a RHS has dof
// e mod n2; dofs >= nv change sign)
template <typename R>
__global__ void coarse_g5_scale_kernel(const typename Pair<R>::T* __restrict__ x, typename Pair<R>::T* __restrict__ y,
                                       const double* __restrict__ scale, int n2, int nv, size_t m) {
  const int r = blockIdx.y;
  const double sc = scale[r];
  constexpr int kc = Pair<R>::kCplx;
  const size_t off = (size_t)r * m;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    auto v = x[off + i];
    R* e = reinterpret_cast<R*>(&v);
#pragma unroll
    for (int c = 0; c < kc; ++c) {
      const R f = (R)(((i * kc + c) % (size_t)n2) >= (size_t)nv ? -sc : sc);
      e[2 * c] *= f;
      e[2 * c + 1] *= f;
    }
    y[off + i] = v;
  }
}

// --------------------------------------------------------------- host side
static inline size_t pairs(const Vec& v) { return v.prec == MGLMA_FP64 ? v.n / 2 : v.n / 4; }

static inline dim3 ew_grid(mglma_ctx ctx, size_t m, int nrhs) {
  size_t want = (m + 255) / 256;
  size_t cap = (size_t)ctx->sm_count * 8 / (size_t)(nrhs > 0 ? nrhs : 1) + 1;
  if (cap < 4) cap = 4;
  return dim3((unsigned)(want < cap ? want : cap), (unsigned)nrhs, 1);
}

mglma_status axpby(mglma_ctx ctx, const double2* a, double2 a_def, const Vec& x, const double2* b, double2 b_def,
                   Vec& y, cudaStream_t s, double sign) {
  if (x.prec != y.prec || x.n != y.n || x.nrhs != y.nrhs) return fail(MGLMA_ERR_INVALID, "axpby: mismatch");
  if (y.nrhs == 0) return MGLMA_OK;
  ProfScope ps(ctx, K_BLAS, s, 3.0 * y.bytes());
  const size_t m = pairs(y);
  dim3 g = ew_grid(ctx, m, y.nrhs);
  if (y.prec == MGLMA_FP64)
    axpby_kernel<double><<<g, 256, 0, s>>>((const double2*)x.p, (double2*)y.p, a, a_def, b, b_def, m, sign);
  else
    axpby_kernel<float><<<g, 256, 0, s>>>((const float4*)x.p, (float4*)y.p, a, a_def, b, b_def, m, sign);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status caxpy(mglma_ctx ctx, const double2* a, const Vec& x, Vec& y, cudaStream_t s, double sign) {
  return axpby(ctx, a, make_double2(0, 0), x, nullptr, make_double2(1, 0), y, s, sign);
}

mglma_status axpy2(mglma_ctx ctx, const double2* a, const Vec& p, Vec& x, const Vec& w, Vec& r, cudaStream_t s) {
  if (p.prec != x.prec || w.prec != r.prec || p.prec != w.prec || p.n != w.n)
    return fail(MGLMA_ERR_INVALID, "axpy2: mismatch");
  ProfScope ps(ctx, K_BLAS, s, 6.0 * p.bytes());
  const size_t m = pairs(p);
  dim3 g = ew_grid(ctx, m, p.nrhs);
  if (p.prec == MGLMA_FP64)
    axpy2_kernel<double><<<g, 256, 0, s>>>((const double2*)p.p, (double2*)x.p, (const double2*)w.p, (double2*)r.p,
                                           a, m);
  else
    axpy2_kernel<float><<<g, 256, 0, s>>>((const float4*)p.p, (float4*)x.p, (const float4*)w.p, (float4*)r.p, a,
                                          m);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status multi_axpy(mglma_ctx ctx, const Vec& x0, size_t jstride_reals, int k, Vec& y, const double2* c,
                        cudaStream_t s, const Vec* x0b, Vec* yb) {
  if (k == 0) return MGLMA_OK;
  if (k > 64) return fail(MGLMA_ERR_INVALID, "multi_axpy: more than 64 directions");
  ProfScope ps(ctx, K_BLAS, s, (k + 2.0) * y.bytes() * (yb ? 2.0 : 1.0));
  const size_t m = pairs(y);
  dim3 g = ew_grid(ctx, m, y.nrhs);
  if (y.prec == MGLMA_FP64)
    multi_axpy_kernel<double><<<g, 256, 0, s>>>((const double2*)x0.p, (double2*)y.p,
                                                x0b ? (const double2*)x0b->p : nullptr, yb ? (double2*)yb->p : nullptr,
                                                jstride_reals / 2, k, c, y.nrhs, m);
  else
    multi_axpy_kernel<float><<<g, 256, 0, s>>>((const float4*)x0.p, (float4*)y.p,
                                               x0b ? (const float4*)x0b->p : nullptr, yb ? (float4*)yb->p : nullptr,
                                               jstride_reals / 4, k, c, y.nrhs, m);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status copy_vec(mglma_ctx ctx, const Vec& x, Vec& y, cudaStream_t s) {
  if (x.prec != y.prec || x.n != y.n || x.nrhs != y.nrhs) return fail(MGLMA_ERR_INVALID, "copy_vec: mismatch");
  const size_t bytes = x.n * (size_t)x.nrhs * (x.prec == MGLMA_FP64 ? 8 : 4);
  if (x.p != y.p) MG_CUDA(cudaMemcpyAsync(y.p, x.p, bytes, cudaMemcpyDeviceToDevice, s));
  return MGLMA_OK;
}

mglma_status zero_vec(mglma_ctx, Vec& y, cudaStream_t s) {
  const size_t bytes = y.n * (size_t)y.nrhs * (y.prec == MGLMA_FP64 ? 8 : 4);
  MG_CUDA(cudaMemsetAsync(y.p, 0, bytes, s));
  return MGLMA_OK;
}

// Blocks per RHS depend on the vector length only, so a RHS's reduction order
// (and result bits) do not change with the number of RHS in its batch.
static int reduce_blocks(size_t m) {
  size_t want = (m + RT * 8 - 1) / (RT * 8);
  if (want > 592) want = 592;
  return (int)(want < 1 ? 1 : want);
}

// Per-stream partial sums and tickets, allocated once with a fixed capacity
// (blocks per RHS <= 592, RHS <= 64, directions <= 64) and never moved, so
// CUDA graphs that captured reductions stay valid; tickets return to zero
// after every reduction.
constexpr size_t kRedParts = (size_t)592 * 64 * 64;
constexpr int kRedCounts = 64;
static mglma_status red_scratch(mglma_ctx ctx, cudaStream_t s, size_t nparts, int ncount, double2** part,
                                unsigned** count) {
  if (nparts > kRedParts || ncount > kRedCounts)
    return fail(MGLMA_ERR_INVALID, "reduction: more than 64 RHS or 64 directions in one launch");
  auto& R = ctx->red[s];
  if (!R.part) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone)
      return fail(MGLMA_ERR_INVALID, "reduction: first use of a stream inside a graph capture");
    MG_CHECK(dalloc(ctx, (void**)&R.part, kRedParts * sizeof(double2), s));
    MG_CHECK(dalloc(ctx, (void**)&R.count, kRedCounts * sizeof(unsigned), s));
    MG_CUDA(cudaMemsetAsync(R.count, 0, kRedCounts * sizeof(unsigned), s));
    R.part_cap = kRedParts;
    R.count_cap = kRedCounts;
  }
  *part = R.part;
  *count = R.count;
  return MGLMA_OK;
}

mglma_status red_scratch_ready(mglma_ctx ctx, cudaStream_t s) {
  double2* p;
  unsigned* c;
  return red_scratch(ctx, s, 1, 1, &p, &c);
}

// accumulators per pass (jm) only matter for MODE 1 (several directions)
template <typename R, int MODE>
static void launch_reduce(dim3 g, int jm, const typename Pair<R>::T* xp, size_t js, int k,
                          const typename Pair<R>::T* yp, size_t m, double2* part, unsigned* count, double2* out2,
                          double* out1, cudaStream_t s) {
  if constexpr (MODE == 1) {
    if (jm == 1) reduce_kernel<R, MODE, 1><<<g, RT, 0, s>>>(xp, js, k, yp, m, part, count, out2, out1);
    if (jm == 2) reduce_kernel<R, MODE, 2><<<g, RT, 0, s>>>(xp, js, k, yp, m, part, count, out2, out1);
    if (jm == 4) reduce_kernel<R, MODE, 4><<<g, RT, 0, s>>>(xp, js, k, yp, m, part, count, out2, out1);
    if (jm == 8) reduce_kernel<R, MODE, 8><<<g, RT, 0, s>>>(xp, js, k, yp, m, part, count, out2, out1);
  } else {
    (void)jm;
    reduce_kernel<R, MODE, 1><<<g, RT, 0, s>>>(xp, js, k, yp, m, part, count, out2, out1);
  }
}

template <int MODE>
static mglma_status reduce_impl(mglma_ctx ctx, const Vec& x0, size_t jstride_reals, int k, const Vec* y,
                                double2* out2, double* out1, cudaStream_t s) {
  if (k == 0 || x0.nrhs == 0) return MGLMA_OK;
  ProfScope ps(ctx, K_REDUCE, s, (MODE == 0 ? 1.0 : (MODE == 2 ? 2.0 : k + 1.0)) * x0.bytes());
  const size_t m = pairs(x0);
  const int nb = reduce_blocks(m);
  const int nslot = MODE == 2 ? 2 : k;
  double2* part = nullptr;
  unsigned* count = nullptr;
  MG_CHECK(red_scratch(ctx, s, (size_t)nb * x0.nrhs * nslot, x0.nrhs, &part, &count));
  dim3 g(nb, x0.nrhs, 1);
  const int jm = k <= 1 ? 1 : (k <= 2 ? 2 : (k <= 4 ? 4 : 8));
  if (x0.prec == MGLMA_FP64)
    launch_reduce<double, MODE>(g, jm, (const double2*)x0.p, jstride_reals / 2, k,
                                y ? (const double2*)y->p : nullptr, m, part, count, out2, out1, s);
  else
    launch_reduce<float, MODE>(g, jm, (const float4*)x0.p, jstride_reals / 4, k,
                               y ? (const float4*)y->p : nullptr, m, part, count, out2, out1, s);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status cdot(mglma_ctx ctx, const Vec& x, const Vec& y, double2* out, cudaStream_t s) {
  if (x.prec != y.prec || x.n != y.n || x.nrhs != y.nrhs) return fail(MGLMA_ERR_INVALID, "cdot: mismatch");
  return reduce_impl<1>(ctx, x, 0, 1, &y, out, nullptr, s);
}

mglma_status multi_cdot(mglma_ctx ctx, const Vec& x0, size_t jstride_reals, int k, const Vec& y, double2* out,
                        cudaStream_t s) {
  return reduce_impl<1>(ctx, x0, jstride_reals, k, &y, out, nullptr, s);
}

mglma_status norm2(mglma_ctx ctx, const Vec& x, double* out, cudaStream_t s) {
  return reduce_impl<0>(ctx, x, 0, 1, nullptr, nullptr, out, s);
}

mglma_status norm2_cdot(mglma_ctx ctx, const Vec& x, const Vec& y, double* nrm, double2* dot, cudaStream_t s) {
  if (x.prec != y.prec || x.n != y.n || x.nrhs != y.nrhs) return fail(MGLMA_ERR_INVALID, "norm2_cdot: mismatch");
  return reduce_impl<2>(ctx, x, 0, 1, &y, dot, nrm, s);
}

mglma_status multi_axpy_nd(mglma_ctx ctx, const Vec& x0, size_t jstride_reals, int k, Vec& y, const double2* c,
                           const Vec* x0b, Vec* yb, const Vec& w, double* nrm, double2* dot, cudaStream_t s) {
  if (k < 1 || k > 64) return fail(MGLMA_ERR_INVALID, "multi_axpy_nd: 1 to 64 directions");
  if (y.prec != MGLMA_FP32 || w.prec != y.prec || w.n != y.n || w.nrhs != y.nrhs)
    return fail(MGLMA_ERR_INVALID, "multi_axpy_nd: FP32 fields of one shape needed");
  ProfScope ps(ctx, K_BLAS, s, (k + 3.0) * y.bytes() + (yb ? (k + 2.0) * y.bytes() : 0.0));
  const size_t m = pairs(y);
  const int nb = reduce_blocks(m);
  double2* part = nullptr;
  unsigned* count = nullptr;
  MG_CHECK(red_scratch(ctx, s, (size_t)nb * y.nrhs * 2, y.nrhs, &part, &count));
  dim3 g(nb, y.nrhs, 1);
  multi_axpy_nd_kernel<float><<<g, RT, 0, s>>>((const float4*)x0.p, (float4*)y.p,
                                               x0b ? (const float4*)x0b->p : nullptr, yb ? (float4*)yb->p : nullptr,
                                               jstride_reals / 4, k, c, (const float4*)w.p, m, part, count, dot, nrm);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status axpy_norm(mglma_ctx ctx, const double2* a, const Vec& w, Vec& r, double* rr, cudaStream_t s) {
  if (w.prec != MGLMA_FP32 || r.prec != w.prec || w.n != r.n || w.nrhs != r.nrhs)
    return fail(MGLMA_ERR_INVALID, "axpy_norm: FP32 fields of one shape needed");
  ProfScope ps(ctx, K_BLAS, s, 3.0 * r.bytes());
  const size_t m = pairs(r);
  const int nb = reduce_blocks(m);
  double2* part = nullptr;
  unsigned* count = nullptr;
  MG_CHECK(red_scratch(ctx, s, (size_t)nb * r.nrhs, r.nrhs, &part, &count));
  dim3 g(nb, r.nrhs, 1);
  axpy_norm_kernel<float><<<g, RT, 0, s>>>((const float4*)w.p, (float4*)r.p, a, m, part, count, rr);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status axpy2_norm(mglma_ctx ctx, const double2* a, const Vec& p, Vec& x, const Vec& w, Vec& r, double* rr,
                        cudaStream_t s) {
  if (p.prec != x.prec || w.prec != r.prec || p.prec != w.prec || p.n != w.n)
    return fail(MGLMA_ERR_INVALID, "axpy2_norm: mismatch");
  ProfScope ps(ctx, K_BLAS, s, 6.0 * p.bytes());
  const size_t m = pairs(p);
  const int nb = reduce_blocks(m);
  double2* part = nullptr;
  unsigned* count = nullptr;
  MG_CHECK(red_scratch(ctx, s, (size_t)nb * p.nrhs, p.nrhs, &part, &count));
  dim3 g(nb, p.nrhs, 1);
  if (p.prec == MGLMA_FP64)
    axpy2_norm_kernel<double><<<g, RT, 0, s>>>((const double2*)p.p, (double2*)x.p, (const double2*)w.p,
                                               (double2*)r.p, a, m, part, count, rr);
  else
    axpy2_norm_kernel<float><<<g, RT, 0, s>>>((const float4*)p.p, (float4*)x.p, (const float4*)w.p, (float4*)r.p, a,
                                              m, part, count, rr);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status lanczos_norm(mglma_ctx ctx, const double2* dot, const double* beta, int* active, const Vec& v,
                          const Vec& u, Vec& z, double* zz, cudaStream_t s, double* st, double tol, int cap) {
  if (v.prec != z.prec || u.prec != z.prec || v.n != z.n || u.n != z.n)
    return fail(MGLMA_ERR_INVALID, "lanczos_norm: mismatch");
  if (z.nrhs == 0) return MGLMA_OK;
  ProfScope ps(ctx, K_REDUCE, s, 4.0 * z.bytes());
  const size_t m = pairs(z);
  const int nb = reduce_blocks(m);
  double2* part = nullptr;
  unsigned* count = nullptr;
  MG_CHECK(red_scratch(ctx, s, (size_t)nb * z.nrhs, z.nrhs, &part, &count));
  dim3 g(nb, z.nrhs, 1);
  if (z.prec == MGLMA_FP64)
    lanczos_norm_kernel<double><<<g, RT, 0, s>>>((const double2*)v.p, (const double2*)u.p, (double2*)z.p, dot, beta,
                                                 active, m, part, count, zz, st, tol, cap, active);
  else
    lanczos_norm_kernel<float><<<g, RT, 0, s>>>((const float4*)v.p, (const float4*)u.p, (float4*)z.p, dot, beta,
                                                active, m, part, count, zz, st, tol, cap, active);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status minres_update(mglma_ctx ctx, const double* cf, int stride, const Vec& v, const Vec& w1, const Vec& w2,
                           Vec& wn, Vec& x, Vec& z, cudaStream_t s) {
  if (v.prec != x.prec || v.n != x.n || w1.n != x.n || w2.n != x.n || wn.n != x.n || z.n != x.n)
    return fail(MGLMA_ERR_INVALID, "minres_update: mismatch");
  if (x.nrhs == 0) return MGLMA_OK;
  ProfScope ps(ctx, K_BLAS, s, 8.0 * x.bytes());
  const size_t m = pairs(x);
  dim3 g = ew_grid(ctx, m, x.nrhs);
  if (x.prec == MGLMA_FP64)
    minres_update_kernel<double><<<g, 256, 0, s>>>((const double2*)v.p, (const double2*)w1.p, (const double2*)w2.p,
                                                   (double2*)wn.p, (double2*)x.p, (double2*)z.p, cf, stride, m);
  else
    minres_update_kernel<float><<<g, 256, 0, s>>>((const float4*)v.p, (const float4*)w1.p, (const float4*)w2.p,
                                                  (float4*)wn.p, (float4*)x.p, (float4*)z.p, cf, stride, m);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status coarse_g5_scale(mglma_ctx ctx, const Vec& x, Vec& y, const double* scale, int n2, cudaStream_t s) {
  if (x.prec != y.prec || x.n != y.n || x.nrhs != y.nrhs || n2 % 2 || x.n % (2 * (size_t)n2))
    return fail(MGLMA_ERR_INVALID, "coarse_g5_scale: mismatch");
  if (y.nrhs == 0) return MGLMA_OK;
  ProfScope ps(ctx, K_BLAS, s, 2.0 * y.bytes());
  const size_t m = pairs(y);
  dim3 g = ew_grid(ctx, m, y.nrhs);
  if (y.prec == MGLMA_FP64)
    coarse_g5_scale_kernel<double><<<g, 256, 0, s>>>((const double2*)x.p, (double2*)y.p, scale, n2, n2 / 2, m);
  else
    coarse_g5_scale_kernel<float><<<g, 256, 0, s>>>((const float4*)x.p, (float4*)y.p, scale, n2, n2 / 2, m);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

}  // namespace mglma
