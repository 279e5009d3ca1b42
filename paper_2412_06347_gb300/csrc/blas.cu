// Multi-RHS BLAS-1 for the Krylov solvers.
//
// A vector batch is nrhs contiguous blocks of n reals ((re, im) pairs); every
// scalar is per RHS and stays in device memory, so a solver iteration issues
// kernels back to back without reading anything on the host.  Reductions
// accumulate in FP64 (for FP32 data: an FP32 partial over one 16-byte load,
// then FP64) in a fixed two-stage order, so results are bitwise reproducible
// and independent of how RHS are grouped.
#include "internal.h"


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

// y_r -= sum_{j<k} c[j][r] x_j,r  with x_j = x0 + j * jstride (vectors)
template <typename R>
__global__ void multi_axpy_kernel(const typename Pair<R>::T* __restrict__ x0, size_t jstride, int k,
                                  typename Pair<R>::T* __restrict__ y, const double2* __restrict__ c, int nrhs,
                                  size_t m) {
  const int r = blockIdx.y;
  const size_t off = (size_t)r * m;
  const double2 one = make_double2(1, 0);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    auto acc = y[off + i];
    for (int j = 0; j < k; ++j) {
      double2 cj = c[(size_t)j * nrhs + r];
      cj.x = -cj.x;
      cj.y = -cj.y;
      acc = lc(x0[j * jstride + off + i], acc, cj, one);
    }
    y[off + i] = acc;
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

// stage 1: part[j][r][blk] for j < k of <x_j, y> (DOT) or |x|^2 (NORM, k = 1)
template <typename R, bool NORM>
__global__ void __launch_bounds__(RT) reduce1_kernel(const typename Pair<R>::T* __restrict__ x0, size_t jstride, int k,
                                                     const typename Pair<R>::T* __restrict__ y, size_t m,
                                                     double2* __restrict__ part, int nrhs) {
  const int r = blockIdx.y;
  const size_t off = (size_t)r * m;
  for (int j = 0; j < k; ++j) {
    double2 acc = make_double2(0, 0);
    const auto* xj = x0 + j * jstride + off;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < m; i += (size_t)gridDim.x * RT) {
      if (NORM) {
        acc.x += nrm_pair(xj[i]);
      } else {
        double2 d = dot_pair(xj[i], y[off + i]);
        acc.x += d.x;
        acc.y += d.y;
      }
    }
    acc = block_sum2<RT>(acc);
    if (threadIdx.x == 0) part[((size_t)j * nrhs + r) * gridDim.x + blockIdx.x] = acc;
  }
}

// stage 2: out[j][r] = sum over blocks, fixed order
__global__ void __launch_bounds__(RT) reduce2_kernel(const double2* __restrict__ part, int nb, double2* out2,
                                                     double* out1) {
  const int jr = blockIdx.x;
  double2 acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < nb; i += RT) {
    double2 v = part[(size_t)jr * nb + i];
    acc.x += v.x;
    acc.y += v.y;
  }
  acc = block_sum2<RT>(acc);
  if (threadIdx.x == 0) {
    if (out2) out2[jr] = acc;
    if (out1) out1[jr] = acc.x;
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
                        cudaStream_t s) {
  if (k == 0) return MGLMA_OK;
  ProfScope ps(ctx, K_BLAS, s, (k + 2.0) * y.bytes());
  const size_t m = pairs(y);
  dim3 g = ew_grid(ctx, m, y.nrhs);
  if (y.prec == MGLMA_FP64)
    multi_axpy_kernel<double><<<g, 256, 0, s>>>((const double2*)x0.p, jstride_reals / 2, k, (double2*)y.p, c,
                                                y.nrhs, m);
  else
    multi_axpy_kernel<float><<<g, 256, 0, s>>>((const float4*)x0.p, jstride_reals / 4, k, (float4*)y.p, c, y.nrhs,
                                               m);
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
static int reduce_blocks(mglma_ctx, size_t m, int) {
  size_t want = (m + RT * 4 - 1) / (RT * 4);
  if (want > 512) want = 512;
  return (int)(want < 1 ? 1 : want);
}

template <bool NORM>
static mglma_status reduce_impl(mglma_ctx ctx, const Vec& x0, size_t jstride_reals, int k, const Vec* y,
                                double2* out2, double* out1, cudaStream_t s) {
  if (k == 0 || x0.nrhs == 0) return MGLMA_OK;
  ProfScope ps(ctx, K_REDUCE, s, (NORM ? 1.0 : k + 1.0) * x0.bytes());
  const size_t m = pairs(x0);
  const int nb = reduce_blocks(ctx, m, x0.nrhs);
  double2* part = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&part, sizeof(double2) * (size_t)nb * x0.nrhs * k, s));
  dim3 g(nb, x0.nrhs, 1);
  if (x0.prec == MGLMA_FP64)
    reduce1_kernel<double, NORM><<<g, RT, 0, s>>>((const double2*)x0.p, jstride_reals / 2, k,
                                                  y ? (const double2*)y->p : nullptr, m, part, x0.nrhs);
  else
    reduce1_kernel<float, NORM><<<g, RT, 0, s>>>((const float4*)x0.p, jstride_reals / 4, k,
                                                 y ? (const float4*)y->p : nullptr, m, part, x0.nrhs);
  reduce2_kernel<<<x0.nrhs * k, RT, 0, s>>>(part, nb, out2, out1);
  dfree(ctx, part, s);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status cdot(mglma_ctx ctx, const Vec& x, const Vec& y, double2* out, cudaStream_t s) {
  if (x.prec != y.prec || x.n != y.n || x.nrhs != y.nrhs) return fail(MGLMA_ERR_INVALID, "cdot: mismatch");
  return reduce_impl<false>(ctx, x, 0, 1, &y, out, nullptr, s);
}

mglma_status multi_cdot(mglma_ctx ctx, const Vec& x0, size_t jstride_reals, int k, const Vec& y, double2* out,
                        cudaStream_t s) {
  return reduce_impl<false>(ctx, x0, jstride_reals, k, &y, out, nullptr, s);
}

mglma_status norm2(mglma_ctx ctx, const Vec& x, double* out, cudaStream_t s) {
  return reduce_impl<true>(ctx, x, 0, 1, nullptr, nullptr, out, s);
}

}  // namespace mglma
