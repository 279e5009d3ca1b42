// Coarse operator D1 = R0 D T0 (Sec. 2, Eqs. res_mg / pro_mg; App. chirality
// shows coarsening D with the chirality-split basis is Galerkin coarsening of
// Q): a nine-point stencil of dense (2Nv x 2Nv) blocks on the block grid
// (Fig. A).  Slot d < 4 couples y to y + mu, 4..7 to y - mu, 8 to y itself.
//
// Build (FP64, setup): for a batch of basis columns j', the fine field equal
// to phi_{j'} on every block is pushed through each hop-slot piece of D (the
// hops that leave a block through the face of slot d, or for slot 8 the
// clover term plus every hop inside the block) and restricted with R0; column
// j' of Dhat_d(y) is the result at block y.
//
// Apply: Y(y) = sum_d Dhat_d(y) X(nbr_d(y)) for many right-hand sides.  The
// adjoint uses gamma5-hermiticity on the coarse grid, Dhat^dag = g5 Dhat g5
// with g5 = +1 on alpha = 0 dofs and -1 on alpha = 1 (App. chirality).
//
// Operator layout: [V1][9][2Nv (column j)][2Nv (row i)] complex, so threads
// that own consecutive rows read consecutive addresses.
#include <algorithm>

#include "cplx.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "solver.h"
#include "subspace.h"

namespace mglma {

// ------------------------------------------------------------ conversions
__global__ void c2canon_f(const float2* __restrict__ c, double2* __restrict__ o, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = make_double2(c[i].x, c[i].y);
}
__global__ void canon2c_f(const double2* __restrict__ o, float2* __restrict__ c, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = make_float2((float)o[i].x, (float)o[i].y);
}

mglma_status coarse_to_canonical(mglma_ctx, const void* c, int prec, size_t n, double* canon, cudaStream_t s) {
  if (prec == MGLMA_FP64) {
    MG_CUDA(cudaMemcpyAsync(canon, c, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  } else {
    c2canon_f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float2*)c, (double2*)canon, n);
    MG_LAUNCH_CHECK();
  }
  return MGLMA_OK;
}

mglma_status coarse_from_canonical(mglma_ctx, const double* canon, size_t n, void* c, int prec, cudaStream_t s) {
  if (prec == MGLMA_FP64) {
    MG_CUDA(cudaMemcpyAsync(c, canon, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  } else {
    canon2c_f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2*)canon, (float2*)c, n);
    MG_LAUNCH_CHECK();
  }
  return MGLMA_OK;
}

// dst = scale_r src (+ dst if accumulate), coarse fields of `per` complex per RHS
template <typename RI, typename RO>
__global__ void cscale_kernel(const RI* __restrict__ src, RO* dst, const double* __restrict__ scale, size_t per,
                              int accumulate) {
  const int r = blockIdx.y;
  const double f = scale ? scale[r] : 1.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (size_t)gridDim.x * blockDim.x) {
    const size_t t = (size_t)r * per + i;
    double re = f * (double)src[t].x, im = f * (double)src[t].y;
    if (accumulate) {
      re += (double)dst[t].x;
      im += (double)dst[t].y;
    }
    dst[t].x = re;
    dst[t].y = im;
  }
}

mglma_status coarse_scale_convert(mglma_ctx ctx, const void* src, int sprec, void* dst, int dprec,
                                  const double* scale, size_t per, int nrhs, bool accumulate, cudaStream_t s) {
  const unsigned gx = (unsigned)std::min<size_t>((per + 255) / 256, (size_t)ctx->sm_count * 4);
  dim3 g(gx, nrhs, 1);
  const int acc = accumulate ? 1 : 0;
  if (sprec == MGLMA_FP64 && dprec == MGLMA_FP32)
    cscale_kernel<double2, float2><<<g, 256, 0, s>>>((const double2*)src, (float2*)dst, scale, per, acc);
  else if (sprec == MGLMA_FP32 && dprec == MGLMA_FP64)
    cscale_kernel<float2, double2><<<g, 256, 0, s>>>((const float2*)src, (double2*)dst, scale, per, acc);
  else if (sprec == MGLMA_FP64)
    cscale_kernel<double2, double2><<<g, 256, 0, s>>>((const double2*)src, (double2*)dst, scale, per, acc);
  else
    cscale_kernel<float2, float2><<<g, 256, 0, s>>>((const float2*)src, (float2*)dst, scale, per, acc);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// ------------------------------------------------------------ build helpers
__global__ void unit_columns_kernel(double2* __restrict__ u, int nb, int64_t V1, int n2, int j0) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nb * V1 * n2) return;
  const int j = (int)(i % n2), r = (int)(i / ((size_t)V1 * n2));
  u[i] = make_double2(j == j0 + r ? 1.0 : 0.0, 0.0);
}

// A64[y][d][j0 + r][i] = C[r][y][i]
__global__ void scatter_columns_kernel(const double2* __restrict__ C, double2* __restrict__ A, int nb, int64_t V1,
                                       int n2, int j0, int d) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nb * V1 * n2) return;
  const int i = (int)(t % n2);
  const int64_t y = (int64_t)((t / n2) % V1);
  const int r = (int)(t / ((size_t)V1 * n2));
  A[(((size_t)y * 9 + d) * n2 + (j0 + r)) * n2 + i] = C[t];
}

__global__ void a_to32_kernel(const double2* __restrict__ a, float2* __restrict__ o, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void a_to16_kernel(const double2* __restrict__ a, __nv_bfloat162* __restrict__ o, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = __floats2bfloat162_rn((float)a[i].x, (float)a[i].y);
}

// canonical export [d][y][i][j]
__global__ void a_export_kernel(const double2* __restrict__ a, double2* __restrict__ o, int64_t V1, int n2) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)9 * V1 * n2 * n2) return;
  const int j = (int)(t % n2), i = (int)((t / n2) % n2);
  const int64_t y = (int64_t)((t / ((size_t)n2 * n2)) % V1);
  const int d = (int)(t / ((size_t)V1 * n2 * n2));
  o[t] = a[(((size_t)y * 9 + d) * n2 + j) * n2 + i];
}

// ------------------------------------------------------------ apply (CUDA cores)
template <typename AT>
struct AL;
template <>
struct AL<double2> {
  template <typename R>
  __device__ __forceinline__ static Cx<R> get(const double2* a, size_t i) {
    double2 v = __ldg(a + i);
    return cx((R)v.x, (R)v.y);
  }
};
template <>
struct AL<float2> {
  template <typename R>
  __device__ __forceinline__ static Cx<R> get(const float2* a, size_t i) {
    float2 v = __ldg(a + i);
    return cx((R)v.x, (R)v.y);
  }
};
template <>
struct AL<__nv_bfloat162> {
  template <typename R>
  __device__ __forceinline__ static Cx<R> get(const __nv_bfloat162* a, size_t i) {
    float2 v = __bfloat1622float2(a[i]);
    return cx((R)v.x, (R)v.y);
  }
};

// grid (V1, RHS tiles); thread i < n2 owns row i of Y(y) for NRT RHS
template <typename R, typename AT, int NRT>
__global__ void coarse_apply_kernel(const AT* __restrict__ A, const Cx<R>* __restrict__ X, Cx<R>* __restrict__ Y,
                                    LatIdx q, int n2, int nrhs, int mode) {
  extern __shared__ unsigned char smraw[];
  Cx<R>* xs = reinterpret_cast<Cx<R>*>(smraw);  // [9][n2][NRT]
  const int64_t y = blockIdx.x;
  const int r0 = blockIdx.y * NRT;
  const int64_t V1 = q.V;
  int x[4];
  site_coords(q, y, x);
  const int nv = n2 / 2;
  for (int idx = threadIdx.x; idx < 9 * n2 * NRT; idx += blockDim.x) {
    const int r = idx % NRT, j = (idx / NRT) % n2, d = idx / (NRT * n2);
    int64_t z = d == 8 ? y : (d < 4 ? nbr_fwd(q, y, x, d) : nbr_bwd(q, y, x, d - 4));
    Cx<R> v = cx<R>(0, 0);
    if (r0 + r < nrhs) v = X[((size_t)(r0 + r) * V1 + z) * n2 + j];
    if ((mode & 1) && j >= nv) v = -v;
    xs[idx] = v;
  }
  __syncthreads();
  const int i = threadIdx.x;
  if (i >= n2) return;
  Cx<R> acc[NRT];
#pragma unroll
  for (int r = 0; r < NRT; ++r) acc[r] = cx<R>(0, 0);
  const AT* Ay = A + (size_t)y * 9 * n2 * n2;
  for (int d = 0; d < 9; ++d) {
    for (int j = 0; j < n2; ++j) {
      const Cx<R> a = AL<AT>::template get<R>(Ay, ((size_t)d * n2 + j) * n2 + i);
      const Cx<R>* xr = xs + (d * n2 + j) * NRT;
#pragma unroll
      for (int r = 0; r < NRT; ++r) cfma(acc[r], a, xr[r]);
    }
  }
  const bool neg = (mode & 2) && i >= nv;
#pragma unroll
  for (int r = 0; r < NRT; ++r)
    if (r0 + r < nrhs) Y[((size_t)(r0 + r) * V1 + y) * n2 + i] = neg ? -acc[r] : acc[r];
}

template <typename R, typename AT, int NRT>
static mglma_status launch_capply(const AT* A, const void* X, void* Y, const mglma_coarse_s* Cc, int nrhs, int mode,
                                  cudaStream_t s) {
  LatIdx q = make_latidx(Cc->geo.Lb);
  const int threads = ((Cc->n2 + 31) / 32) * 32;
  const int smem = 9 * Cc->n2 * NRT * (int)sizeof(Cx<R>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(coarse_apply_kernel<R, AT, NRT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid((unsigned)Cc->geo.V1, (unsigned)((nrhs + NRT - 1) / NRT), 1);
  coarse_apply_kernel<R, AT, NRT><<<grid, threads, smem, s>>>(A, (const Cx<R>*)X, (Cx<R>*)Y, q, Cc->n2, nrhs,
                                                              mode);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status coarse_apply(mglma_ctx ctx, const mglma_coarse_s* Cc, const void* X, void* Y, int nrhs, int prec,
                          int mode, cudaStream_t s, void* scratch, size_t scratch_bytes) {
  if (mode < 0 || mode > 3) return fail(MGLMA_ERR_INVALID, "coarse apply: unknown gamma5 mode");
  if (nrhs == 0) return MGLMA_OK;
  // algorithmic traffic: the operator once (9 (2Nv)^2 complex per coarse
  // site) plus each RHS's input and output once; 8 flops per complex MAC
  const double V1 = (double)Cc->geo.V1, n2 = Cc->n2, N = nrhs;
  const double ca = prec == MGLMA_FP64 ? 16.0 : ((Cc->A16 || Cc->Aimg) ? 4.0 : (Cc->A32 ? 8.0 : 16.0));
  const double cf = prec == MGLMA_FP64 ? 16.0 : 8.0;
  ProfScope ps(ctx, K_COARSE, s, V1 * (9.0 * n2 * n2 * ca + 2.0 * N * n2 * cf), V1 * 9.0 * n2 * n2 * 8.0 * N);
  if (prec == MGLMA_FP64) {
    if (!Cc->A64) return fail(MGLMA_ERR_INVALID, "coarse apply: FP64 operator not kept");
    return launch_capply<double, double2, 4>(Cc->A64, X, Y, Cc, nrhs, mode, s);
  }
  if (Cc->Aimg)
    return coarse_apply_tc(ctx, Cc, (const float2*)X, (float2*)Y, nrhs, mode, scratch, scratch_bytes, s);
  if (Cc->A16) return launch_capply<float, __nv_bfloat162, 8>(Cc->A16, X, Y, Cc, nrhs, mode, s);
  if (Cc->A32) return launch_capply<float, float2, 8>(Cc->A32, X, Y, Cc, nrhs, mode, s);
  return launch_capply<float, double2, 8>(Cc->A64, X, Y, Cc, nrhs, mode, s);
}

mglma_status dslash_slot64_batch(mglma_ctx ctx, const mglma_gauge_s* G, const int block[4], const Spinor& in,
                                 Spinor& out, int slot, cudaStream_t s);

mglma_status coarse_store_copies(mglma_ctx ctx, mglma_coarse_s* Cc, int store, cudaStream_t s) {
  const size_t na = (size_t)Cc->geo.V1 * 9 * Cc->n2 * Cc->n2;
  cudaError_t e = cudaSuccess;
  if (store == MGLMA_FP32) {
    e = cudaMalloc(&Cc->A32, na * sizeof(float2));
    if (e == cudaSuccess) a_to32_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(Cc->A64, Cc->A32, na);
  } else if (store == MGLMA_BF16 && coarse_tc_supported(Cc->n2)) {
    MG_CHECK(coarse_tc_image(ctx, Cc, s));  // tensor-core operand image
  } else if (store == MGLMA_BF16) {
    e = cudaMalloc(&Cc->A16, na * sizeof(__nv_bfloat162));
    if (e == cudaSuccess) a_to16_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(Cc->A64, Cc->A16, na);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MGLMA_ERR_OOM, "coarse operator: cannot allocate the low-precision copy");
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

}  // namespace mglma

using namespace mglma;

extern "C" {

mglma_status mglma_coarse_build(mglma_ctx ctx, mglma_gauge G, mglma_subspace S, mglma_prec store,
                                mglma_coarse* out) {
  if (!ctx || !G || !S || !out) return fail(MGLMA_ERR_INVALID, "coarse_build: NULL argument");
  if (S->gauge != G) return fail(MGLMA_ERR_INVALID, "coarse_build: subspace belongs to another gauge field");
  if (!S->phi64 && !S->lean) return fail(MGLMA_ERR_INVALID, "coarse_build: the subspace's FP64 basis was released");
  if (store != MGLMA_FP64 && store != MGLMA_FP32 && store != MGLMA_BF16)
    return fail(MGLMA_ERR_INVALID, "coarse_build: store must be FP64, FP32 or BF16");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const BlockGeo g = S->geo;
  const int n2 = 2 * S->nv;
  mglma_coarse_s* Cc = new mglma_coarse_s();
  Cc->ctx = ctx;
  Cc->sub = S;
  Cc->nv = S->nv;
  Cc->n2 = n2;
  Cc->store = store;
  Cc->geo = g;
  const size_t na = (size_t)g.V1 * 9 * n2 * n2;
  if (cudaMalloc(&Cc->A64, na * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    delete Cc;
    return fail(MGLMA_ERR_OOM, "coarse_build: cannot allocate the operator");
  }
  // columns per batch: bounded by free memory (two FP64 fine fields per column)
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  const size_t per_col = (size_t)2 * g.V * 24 * sizeof(double) + (size_t)2 * g.V1 * n2 * sizeof(double2);
  int NB = (int)std::min<size_t>((size_t)n2, std::max<size_t>(1, fr / 3 / per_col));
  NB = std::min(NB, 16);
  mglma_status st = MGLMA_OK;
  {  // column work fields, returned to the pool at the end of this scope
    FreeList fl(ctx, s);
    double2 *U1 = nullptr, *C = nullptr;
    Spinor Phi, H;
    st = dalloc(ctx, (void**)&U1, (size_t)NB * g.V1 * n2 * sizeof(double2), s);
    fl.add(U1);
    if (st == MGLMA_OK) st = dalloc(ctx, (void**)&C, (size_t)NB * g.V1 * n2 * sizeof(double2), s);
    fl.add(C);
    if (st == MGLMA_OK) st = alloc_spinor(ctx, Phi, MGLMA_FP64, NB, g.V, s);
    fl.add(Phi.p);
    if (st == MGLMA_OK) st = alloc_spinor(ctx, H, MGLMA_FP64, NB, g.V, s);
    fl.add(H.p);
    for (int j0 = 0; st == MGLMA_OK && j0 < n2; j0 += NB) {
      const int nb = std::min(NB, n2 - j0);
      Phi.nrhs = H.nrhs = nb;
      const size_t nu = (size_t)nb * g.V1 * n2;
      {
        ProfScope ps(ctx, K_SETUP, s);
        unit_columns_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(U1, nb, g.V1, n2, j0);
      }
      st = prolong_coarse(ctx, S, U1, Phi, false, s);
      for (int d = 0; st == MGLMA_OK && d < 9; ++d) {
        st = dslash_slot64_batch(ctx, G, g.b, Phi, H, d, s);
        if (st == MGLMA_OK) st = restrict_fine(ctx, S, H, C, s);
        if (st == MGLMA_OK) {
          ProfScope ps(ctx, K_SETUP, s);
          scatter_columns_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(C, Cc->A64, nb, g.V1, n2, j0, d);
        }
      }
    }
  }
  if (st == MGLMA_OK && cudaGetLastError() != cudaSuccess) st = fail(MGLMA_ERR_CUDA, "coarse_build: launch failed");
  if (st == MGLMA_OK) st = coarse_store_copies(ctx, Cc, store, s);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaMemPoolTrimTo(ctx->pool, 0);  // hand the build's work fields back to the device
  if (st == MGLMA_OK && e != cudaSuccess) st = fail(MGLMA_ERR_CUDA, cudaGetErrorString(e));
  if (st != MGLMA_OK) {
    mglma_coarse_free(Cc);
    return st;
  }
  *out = Cc;
  return MGLMA_OK;
}

mglma_status mglma_coarse_release_fp64(mglma_coarse Cc) {
  if (!Cc) return fail(MGLMA_ERR_INVALID, "coarse_release_fp64: NULL handle");
  if (!Cc->A32 && !Cc->A16 && !Cc->Aimg)
    return fail(MGLMA_ERR_INVALID, "coarse_release_fp64: the FP64 operator is the only copy");
  if (Cc->ctx) MG_CUDA(cudaSetDevice(Cc->ctx->device));
  // the even-odd set-up needs the FP64 operator: form it now when the coarse
  // grid allows it; with the tensor-core image only its BF16 image is kept
  bool even = true;
  for (int m = 0; m < 4; ++m) even = even && Cc->geo.Lb[m] % 2 == 0;
  if (even && Cc->ctx) MG_CHECK(coarse_eo_setup(Cc->ctx, Cc, Cc->ctx->stream));
  MG_CUDA(cudaDeviceSynchronize());
  cudaFree(Cc->A64);
  Cc->A64 = nullptr;
  if (Cc->Sinv_img) {
    cudaFree(Cc->Sinv64);
    Cc->Sinv64 = nullptr;
  }
  return MGLMA_OK;
}

void mglma_coarse_free(mglma_coarse Cc) {
  if (!Cc) return;
  if (Cc->ctx) cudaSetDevice(Cc->ctx->device);
  cudaFree(Cc->Sinv64);
  cudaFree(Cc->Sinv_img);
  cudaFree(Cc->Ahat_img);
  cudaFree(Cc->A64);
  cudaFree(Cc->A32);
  cudaFree(Cc->A16);
  cudaFree(Cc->Aimg);
  cudaFree(Cc->tc_err);
  cudaFree(Cc->tc_dpart);
  cudaFree(Cc->tc_dcount);
  delete Cc;
}

mglma_status mglma_coarse_export(mglma_coarse Cc, double* dhat) {
  if (!Cc || !dhat) return fail(MGLMA_ERR_INVALID, "coarse_export: NULL argument");
  if (!Cc->A64) return fail(MGLMA_ERR_INVALID, "coarse_export: FP64 operator not kept");
  mglma_ctx ctx = Cc->ctx;
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const size_t n = (size_t)9 * Cc->geo.V1 * Cc->n2 * Cc->n2;
  Staged o;
  MG_CHECK(stage_out_alloc(ctx, dhat, n * sizeof(double2), s, o));
  a_export_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Cc->A64, (double2*)o.dev, Cc->geo.V1, Cc->n2);
  MG_LAUNCH_CHECK();
  MG_CHECK(stage_out_finish(dhat, n * sizeof(double2), s, o));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

mglma_status mglma_coarse_apply(mglma_ctx ctx, mglma_coarse Cc, mglma_op op, int nrhs, const double* in, double* out,
                                mglma_prec compute, void* cuda_stream) {
  if (!ctx || !Cc || !in || !out) return fail(MGLMA_ERR_INVALID, "coarse_apply: NULL argument");
  // gamma5hat on the input (bit 0) and on the output (bit 1)
  const int mode = op == MGLMA_OP_D ? 0 : op == MGLMA_OP_DDAG ? 3 : op == MGLMA_OP_Q ? 2
                 : op == MGLMA_OP_SCHUR ? 0 : op == MGLMA_OP_SCHUR_Q ? 2 : -1;
  if (mode < 0) return fail(MGLMA_ERR_INVALID, "coarse_apply: op must be D, D^dag, Q, SCHUR or SCHUR_Q");
  const bool schur = op == MGLMA_OP_SCHUR || op == MGLMA_OP_SCHUR_Q;
  if (compute != MGLMA_FP64 && compute != MGLMA_FP32)
    return fail(MGLMA_ERR_INVALID, "coarse_apply: compute must be FP64 or FP32");
  if (nrhs <= 0) return nrhs == 0 ? MGLMA_OK : fail(MGLMA_ERR_INVALID, "coarse_apply: nrhs < 0");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, cuda_stream);
  const size_t n = (size_t)nrhs * Cc->geo.V1 * Cc->n2;
  Staged si, so;
  MG_CHECK(stage_in(ctx, in, n * sizeof(double2), s, si));
  MG_CHECK(stage_out_alloc(ctx, out, n * sizeof(double2), s, so));
  FreeList fl(ctx, s);
  void *X = nullptr, *Y = nullptr;
  const size_t cb = compute == MGLMA_FP64 ? sizeof(double2) : sizeof(float2);
  MG_CHECK(dalloc(ctx, &X, n * cb, s));
  fl.add(X);
  MG_CHECK(dalloc(ctx, &Y, n * cb, s));
  fl.add(Y);
  MG_CHECK(coarse_from_canonical(ctx, si.dev, n, X, compute, s));
  if (schur)
    MG_CHECK(coarse_schur_full(ctx, Cc, X, Y, nrhs, compute, mode, s));
  else
    MG_CHECK(coarse_apply(ctx, Cc, X, Y, nrhs, compute, mode, s));
  MG_CHECK(coarse_tc_check(Cc, s));
  MG_CHECK(coarse_to_canonical(ctx, Y, compute, n, so.dev, s));
  MG_CHECK(stage_out_finish(out, n * sizeof(double2), s, so));
  return MGLMA_OK;
}

mglma_status mglma_coarse_info(mglma_coarse Cc, int* nv, int Lb[4], int64_t* coarse_volume) {
  if (!Cc) return fail(MGLMA_ERR_INVALID, "coarse_info: NULL handle");
  if (nv) *nv = Cc->nv;
  if (Lb)
    for (int m = 0; m < 4; ++m) Lb[m] = Cc->geo.Lb[m];
  if (coarse_volume) *coarse_volume = Cc->geo.V1;
  return MGLMA_OK;
}

}  // extern "C"
