// Even-odd (Schur) preconditioning of the coarse operator (the paper's coarse
// solves use the even-odd preconditioned coarse Dirac operator, Sec.
// "Comparison of the cost").
//
// When every extent of the coarse grid is even, every hop slot of the
// nine-point stencil joins sites of opposite parity p(y) = (y0 + y1 + y2 +
// y3) mod 2, so with the sites ordered even then odd
//     D = [[D_ee, D_eo], [D_oe, D_oo]],   D_ee, D_oo block-diagonal (slot 8)
// and D x = b is solved through the Schur complement on the even sites
//     S_ee x_e = b_e - D_eo D_oo^-1 b_o,   S_ee = D_ee - D_eo D_oo^-1 D_oe,
//     x_o = D_oo^-1 (b_o - D_oe x_e).
// g5hat S_ee is Hermitian (the self blocks commute with g5hat), so MINRES runs
// on it as on g5hat D.  Half-lattice fields hold the sites of one parity, site
// y at index y >> 1.
//
// The FP32 path (BF16 operator on the tensor cores) applies S_ee in two
// launches of the stencil kernel restricted to one parity:
//     U_o  = -(D_oo^-1 D_oe) X_e            (odd sites, the eight hop slots
//                                             premultiplied by the inverse
//                                             self block in FP64 at set-up)
//     Y_e  = D_eo U_o + D_ee X_e            (even sites, all nine slots)
// which streams 8 + 9 slot blocks per pair of sites -- about the bytes of one
// full application -- on vectors of half the length.  The FP64 path composes
// full FP64 applications (used for the exact checks through the C ABI).
#include <algorithm>
#include <cmath>

#include "cplx.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "solver.h"
#include "subspace.h"

namespace mglma {

// inverse of one self block per CTA: Gauss-Jordan with partial pivoting on
// an n2 x n2 complex matrix in shared memory (FP64)
__global__ void self_inverse_kernel(const double2* __restrict__ A, double2* __restrict__ Ainv, int n2,
                                    int* __restrict__ singular) {
  extern __shared__ double2 M[];  // row-major n2 x n2
  __shared__ int piv;
  __shared__ double2 pinv;
  const int64_t y = blockIdx.x;
  const double2* Ay = A + ((size_t)y * 9 + 8) * n2 * n2;  // [col j][row i]
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
    const int i = e / n2, j = e % n2;
    M[e] = Ay[(size_t)j * n2 + i];
  }
  __syncthreads();
  __shared__ int perm[128];
  for (int k = 0; k < n2; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = -1;
      for (int r = k; r < n2; ++r) {
        const double2 v = M[r * n2 + k];
        const double m = v.x * v.x + v.y * v.y;
        if (m > best) {
          best = m;
          p = r;
        }
      }
      piv = p;
      perm[k] = p;
      if (!(best > 0)) atomicExch(singular, 1);
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int c = threadIdx.x; c < n2; c += blockDim.x) {
        const double2 t = M[k * n2 + c];
        M[k * n2 + c] = M[p * n2 + c];
        M[p * n2 + c] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double2 a = M[k * n2 + k];
      const double m = a.x * a.x + a.y * a.y;
      pinv = m > 0 ? make_double2(a.x / m, -a.y / m) : make_double2(0, 0);
    }
    __syncthreads();
    const Cx<double> d = cx(pinv.x, pinv.y);
    for (int c = threadIdx.x; c < n2; c += blockDim.x) {  // row k
      if (c == k) continue;
      const double2 v = M[k * n2 + c];
      const Cx<double> w = cx(v.x, v.y) * d;
      M[k * n2 + c] = make_double2(w.re, w.im);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {  // other rows
      const int r = e / n2, c = e % n2;
      if (r == k || c == k) continue;
      const double2 f = M[r * n2 + k], v = M[k * n2 + c], o = M[e];
      const Cx<double> w = cx(o.x, o.y) - cx(f.x, f.y) * cx(v.x, v.y);
      M[e] = make_double2(w.re, w.im);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n2; r += blockDim.x) {  // column k
      if (r == k) continue;
      const double2 f = M[r * n2 + k];
      const Cx<double> w = -(cx(f.x, f.y) * d);
      M[r * n2 + k] = make_double2(w.re, w.im);
    }
    __syncthreads();
    if (threadIdx.x == 0) M[k * n2 + k] = make_double2(d.re, d.im);
    __syncthreads();
  }
  // undo the row swaps as column swaps, last first
  for (int k = n2 - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int r = threadIdx.x; r < n2; r += blockDim.x) {
        const double2 t = M[r * n2 + k];
        M[r * n2 + k] = M[r * n2 + p];
        M[r * n2 + p] = t;
      }
    __syncthreads();
  }
  double2* Oy = Ainv + (size_t)y * n2 * n2;  // one slot: [col j][row i]
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
    const int i = e / n2, j = e % n2;
    Oy[(size_t)j * n2 + i] = M[e];
  }
}

// Ahat[u][d] = Sinv(y) A[y][d] for the odd site y of half-lattice index u and
// the hop slots d = 0..7 (FP64, [u][8][col j][row i]); one CTA per (u, d),
// both factors staged in shared memory
__global__ void ahat_kernel(const double2* __restrict__ A64, const double2* __restrict__ Sinv,
                            double2* __restrict__ Ahat, LatIdx q, int n2) {
  extern __shared__ double2 sh[];
  double2* S = sh;            // [col l][row i]
  double2* A = sh + n2 * n2;  // [col j][row l]
  const int64_t u = blockIdx.x / 8;
  const int d = (int)(blockIdx.x % 8);
  int xc[4];
  site_coords(q, 2 * u, xc);
  const int64_t y = 2 * u + ((1 ^ (xc[0] + xc[1] + xc[2] + xc[3])) & 1);
  const int nn = n2 * n2;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    S[e] = Sinv[(size_t)y * nn + e];
    A[e] = A64[((size_t)y * 9 + d) * nn + e];
  }
  __syncthreads();
  double2* O = Ahat + ((size_t)u * 8 + d) * nn;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int j = e / n2, i = e % n2;
    Cx<double> acc = cx(0.0, 0.0);
    for (int l = 0; l < n2; ++l) {
      const double2 a = S[l * n2 + i], b = A[j * n2 + l];
      cfma(acc, cx(a.x, a.y), cx(b.x, b.y));
    }
    O[e] = make_double2(acc.re, acc.im);
  }
}

// half-lattice field of parity par <-> full field (the other parity of a
// full output is set to zero)
template <typename T>
__global__ void eo_gather_kernel(const T* __restrict__ full, T* __restrict__ half, LatIdx q, int n2, int nrhs,
                                 int par) {
  const int64_t Vh = q.V / 2;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nrhs * Vh * n2) return;
  const int k = (int)(e % n2);
  const int64_t u = (int64_t)((e / n2) % Vh);
  const int r = (int)(e / ((size_t)n2 * Vh));
  int xc[4];
  site_coords(q, 2 * u, xc);
  const int64_t y = 2 * u + ((par ^ (xc[0] + xc[1] + xc[2] + xc[3])) & 1);
  half[e] = full[((size_t)r * q.V + y) * n2 + k];
}
template <typename T>
__global__ void eo_scatter_kernel(const T* __restrict__ half, T* __restrict__ full, LatIdx q, int n2, int nrhs,
                                  int par) {
  const int64_t Vh = q.V / 2;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nrhs * Vh * n2) return;
  const int k = (int)(e % n2);
  const int64_t u = (int64_t)((e / n2) % Vh);
  const int r = (int)(e / ((size_t)n2 * Vh));
  int xc[4];
  site_coords(q, 2 * u, xc);
  const int64_t y = 2 * u + ((par ^ (xc[0] + xc[1] + xc[2] + xc[3])) & 1);
  full[((size_t)r * q.V + y) * n2 + k] = half[e];
}

// Y_u = sgn * Sinv(y(u)) X_u on half-lattice fields of parity par (FP64 or
// FP32 fields, FP64 inverse blocks); one thread per output element
template <typename T>
__global__ void self_inv_apply_kernel(const double2* __restrict__ Sinv, const T* __restrict__ X, T* __restrict__ Y,
                                      LatIdx q, int n2, int nrhs, int par, double sgn) {
  const int64_t Vh = q.V / 2;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nrhs * Vh * n2) return;
  const int i = (int)(e % n2);
  const int64_t u = (int64_t)((e / n2) % Vh);
  const int r = (int)(e / ((size_t)n2 * Vh));
  int xc[4];
  site_coords(q, 2 * u, xc);
  const int64_t y = 2 * u + ((par ^ (xc[0] + xc[1] + xc[2] + xc[3])) & 1);
  const double2* B = Sinv + (size_t)y * n2 * n2;
  const T* x = X + ((size_t)r * Vh + u) * n2;
  Cx<double> acc = cx(0.0, 0.0);
  for (int j = 0; j < n2; ++j) {
    const double2 a = B[(size_t)j * n2 + i];
    cfma(acc, cx(a.x, a.y), cx((double)x[j].x, (double)x[j].y));
  }
  Y[e].x = sgn * acc.re;
  Y[e].y = sgn * acc.im;
}

// y = a x + y on half-lattice coarse fields (FP32 or FP64), a = +-1
template <typename T>
__global__ void eo_axpy_kernel(double a, const T* __restrict__ x, T* y, size_t n) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  y[e].x = a * (double)x[e].x + (double)y[e].x;
  y[e].y = a * (double)x[e].y + (double)y[e].y;
}

// y *= g5hat in place: dofs i >= n2 / 2 (chirality 1) negated
template <typename T>
__global__ void eo_g5_kernel(T* y, int n2, size_t n) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n || (int)(e % n2) < n2 / 2) return;
  y[e].x = -y[e].x;
  y[e].y = -y[e].y;
}

static unsigned nblk(size_t n) { return (unsigned)((n + 255) / 256); }

mglma_status coarse_eo_setup(mglma_ctx ctx, mglma_coarse_s* C, cudaStream_t s) {
  if (C->Sinv64 || C->Sinv_img) return MGLMA_OK;  // formed
  for (int m = 0; m < 4; ++m)
    if (C->geo.Lb[m] % 2)
      return fail(MGLMA_ERR_INVALID, "even-odd: every extent of the coarse grid must be even");
  if (!C->A64) return fail(MGLMA_ERR_INVALID, "even-odd: the set-up needs the FP64 coarse operator");
  if (C->n2 > 128) return fail(MGLMA_ERR_INVALID, "even-odd: more than 128 dofs per coarse site");
  const int n2 = C->n2;
  MG_CUDA(cudaMalloc(&C->Sinv64, (size_t)C->geo.V1 * n2 * n2 * sizeof(double2)));
  int* sing = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&sing, sizeof(int), s));
  MG_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
  const int smem = n2 * n2 * (int)sizeof(double2);
  MG_CUDA(cudaFuncSetAttribute(self_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  {
    ProfScope ps(ctx, K_SETUP, s);
    self_inverse_kernel<<<(unsigned)C->geo.V1, 256, smem, s>>>(C->A64, C->Sinv64, n2, sing);
  }
  MG_LAUNCH_CHECK();
  if (C->Aimg) {
    MG_CHECK(coarse_tc_image_blocks(ctx, C->Sinv64, C->geo.V1, n2, 1, &C->Sinv_img, s));
    // D_oo^-1 D_oe in FP64, rounded to BF16 once in its image
    const int64_t Vh = C->geo.V1 / 2;
    double2* ahat = nullptr;
    MG_CHECK(dalloc(ctx, (void**)&ahat, (size_t)Vh * 8 * n2 * n2 * sizeof(double2), s));
    const int smem2 = 2 * smem;
    MG_CUDA(cudaFuncSetAttribute(ahat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    {
      ProfScope ps(ctx, K_SETUP, s);
      ahat_kernel<<<(unsigned)(Vh * 8), 256, smem2, s>>>(C->A64, C->Sinv64, ahat, make_latidx(C->geo.Lb), n2);
    }
    MG_LAUNCH_CHECK();
    const mglma_status st = coarse_tc_image_blocks(ctx, ahat, Vh, n2, 8, &C->Ahat_img, s);
    dfree(ctx, ahat, s);
    MG_CHECK(st);
  }
  int h = 0;
  MG_CUDA(cudaMemcpyAsync(&h, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
  dfree(ctx, sing, s);
  MG_CUDA(cudaStreamSynchronize(s));
  if (h) return fail(MGLMA_ERR_NUMERIC, "even-odd: a self block of the coarse operator is singular");
  return MGLMA_OK;
}

size_t coarse_eo_scratch_bytes(const mglma_coarse_s* C, int nrhs) {
  // two B images (hop and self inputs) and two half-lattice FP32 fields
  return 2 * coarse_tc_half_image_bytes(C, nrhs) + 2 * (size_t)nrhs * (C->geo.V1 / 2) * C->n2 * sizeof(float2) +
         1024;
}

// the FP64 (or non-tensor-core) Schur apply by composition of full applications:
// full fields, scratch allocated here
static mglma_status schur_composed(mglma_ctx ctx, const mglma_coarse_s* C, const void* Xe, void* Ye, int nrhs,
                                   int prec, int mode, cudaStream_t s) {
  const LatIdx q = make_latidx(C->geo.Lb);
  const int n2 = C->n2;
  const size_t cb = prec == MGLMA_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t nfull = (size_t)nrhs * q.V * n2, nhalf = nfull / 2;
  FreeList fl(ctx, s);
  void *F = nullptr, *T = nullptr, *H = nullptr;
  MG_CHECK(dalloc(ctx, &F, nfull * cb, s));
  fl.add(F);
  MG_CHECK(dalloc(ctx, &T, nfull * cb, s));
  fl.add(T);
  MG_CHECK(dalloc(ctx, &H, nhalf * cb, s));
  fl.add(H);
  const bool dp = prec == MGLMA_FP64;
  // F = embed(X_e); T = D F (T_e = D_ee X_e, T_o = D_oe X_e)
  MG_CUDA(cudaMemsetAsync(F, 0, nfull * cb, s));
  if (dp)
    eo_scatter_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)Xe, (double2*)F, q, n2, nrhs, 0);
  else
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)Xe, (float2*)F, q, n2, nrhs, 0);
  MG_CHECK(coarse_apply(ctx, C, F, T, nrhs, prec, CMODE_D, s));
  // H = -D_oo^-1 T_o ; F = embed_o(H) ; T' = D F (even part: -D_eo D_oo^-1 D_oe X_e)
  void* To = Ye;  // Ye (half) as temporary for T_o
  if (dp) {
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)T, (double2*)To, q, n2, nrhs, 1);
    self_inv_apply_kernel<double2><<<nblk(nhalf), 256, 0, s>>>(C->Sinv64, (const double2*)To, (double2*)H, q, n2,
                                                               nrhs, 1, -1.0);
  } else {
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)T, (float2*)To, q, n2, nrhs, 1);
    self_inv_apply_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(C->Sinv64, (const float2*)To, (float2*)H, q, n2, nrhs,
                                                              1, -1.0);
  }
  // even part of T = D_ee X_e kept in H? gather it first into Ye after using To
  MG_CUDA(cudaMemsetAsync(F, 0, nfull * cb, s));
  if (dp) {
    eo_scatter_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)H, (double2*)F, q, n2, nrhs, 1);
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)T, (double2*)H, q, n2, nrhs, 0);
  } else {
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)H, (float2*)F, q, n2, nrhs, 1);
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)T, (float2*)H, q, n2, nrhs, 0);
  }
  MG_CHECK(coarse_apply(ctx, C, F, T, nrhs, prec, CMODE_D, s));
  // Y_e = H (= D_ee X_e) + (D T')_e, then g5hat on the output by mode bit 1
  if (dp) {
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)T, (double2*)Ye, q, n2, nrhs, 0);
    eo_axpy_kernel<double2><<<nblk(nhalf), 256, 0, s>>>(1.0, (const double2*)H, (double2*)Ye, nhalf);
  } else {
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)T, (float2*)Ye, q, n2, nrhs, 0);
    eo_axpy_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(1.0, (const float2*)H, (float2*)Ye, nhalf);
  }
  MG_LAUNCH_CHECK();
  if (mode & 2) {
    if (dp)
      eo_g5_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((double2*)Ye, n2, nhalf);
    else
      eo_g5_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((float2*)Ye, n2, nhalf);
    MG_LAUNCH_CHECK();
  }
  return MGLMA_OK;
}

bool coarse_schur_dot_ok(mglma_ctx ctx, const mglma_coarse_s* C, int nrhs, int prec) {
  return prec == MGLMA_FP32 && C->Aimg && C->Sinv_img && C->tc_dpart && nrhs >= 1 &&
         nrhs <= tuned(ctx, TUNE_COARSE_NT, nrhs, C->geo.V1, coarse_tc_default_nt(nrhs));
}

mglma_status coarse_schur_apply(mglma_ctx ctx, const mglma_coarse_s* C, const void* Xe, void* Ye, int nrhs, int prec,
                                int mode, void* scratch, size_t scratch_bytes, cudaStream_t s, double2* dot_out,
                                bool x_imaged) {
  if (dot_out && !coarse_schur_dot_ok(ctx, C, nrhs, prec))
    return fail(MGLMA_ERR_INVALID, "schur apply: the fused dot needs the tensor-core path and one RHS tile");
  if (x_imaged && !dot_out) return fail(MGLMA_ERR_INVALID, "schur apply: a given X image goes with the fused dot");
  if (!C->Sinv64 && !C->Sinv_img) return fail(MGLMA_ERR_INVALID, "schur apply: even-odd set-up missing");
  if (!C->Sinv64 && (prec == MGLMA_FP64 || !C->Aimg))
    return fail(MGLMA_ERR_INVALID, "schur apply: the FP64 self-block inverses were released");
  if (nrhs == 0) return MGLMA_OK;
  const double V1 = (double)C->geo.V1, n2 = C->n2, N = nrhs;
  ProfScope ps(ctx, K_COARSE, s, V1 * (9.0 * n2 * n2 * 4.0 + 2.0 * N * n2 * 8.0),
               V1 * 9.0 * n2 * n2 * 8.0 * N);
  if (prec == MGLMA_FP64 || !C->Aimg || !C->Sinv_img) return schur_composed(ctx, C, Xe, Ye, nrhs, prec, mode, s);
  if (!scratch || scratch_bytes < coarse_eo_scratch_bytes(C, nrhs))
    return fail(MGLMA_ERR_INVALID, "schur apply: scratch too small");
  const size_t half = (size_t)nrhs * (C->geo.V1 / 2) * n2;
  uint8_t* img = (uint8_t*)scratch;
  float2* To = reinterpret_cast<float2*>(img + 2 * coarse_tc_half_image_bytes(C, nrhs));
  float2* Uo = To + half;
  const float2* X = (const float2*)Xe;
  // U_o = -D_oo^-1 D_oe X_e (one launch on the D_oo^-1 D_oe image, else
  // T_o = D_oe X_e and U_o = -D_oo^-1 T_o) ; Y_e = D_eo U_o + D_ee X_e
  // (g5hat by mode bit 1).  The image of X_e the first launch writes (first
  // half image) serves the last as its self input; the last writes the image
  // of U_o into the second half image.
  const size_t hb = coarse_tc_half_image_bytes(C, nrhs);
  if (C->Ahat_img) {
    MG_CHECK(coarse_tc_eo_launch(ctx, C, X, nullptr, Uo, nrhs, 0, 1, 0, 7, nullptr, -1.f, img, s, nullptr,
                                 C->Ahat_img, nullptr, nullptr, x_imaged));
  } else {
    MG_CHECK(coarse_tc_eo_launch(ctx, C, X, nullptr, To, nrhs, 0, 1, 0, 7, nullptr, 1.f, img, s, nullptr, nullptr,
                                 nullptr, nullptr, x_imaged));
    MG_CHECK(coarse_tc_eo_launch(ctx, C, nullptr, To, Uo, nrhs, 0, 1, 8, 8, C->Sinv_img, -1.f, img, s));
  }
  return coarse_tc_eo_launch(ctx, C, Uo, X, (float2*)Ye, nrhs, mode & 2, 0, 0, 8, nullptr, 1.f, img + hb, s, img,
                             nullptr, dot_out ? X : nullptr, dot_out);
}

mglma_status coarse_eo_prepare(mglma_ctx ctx, const mglma_coarse_s* C, const void* b, void* be, int nrhs, int prec,
                               void* scratch, size_t scratch_bytes, cudaStream_t s) {
  const LatIdx q = make_latidx(C->geo.Lb);
  const int n2 = C->n2;
  const size_t nhalf = (size_t)nrhs * (q.V / 2) * n2;
  const bool dp = prec == MGLMA_FP64;
  ProfScope ps(ctx, K_COARSE, s);
  if (!dp && C->Aimg && C->Sinv_img) {
    if (!scratch || scratch_bytes < coarse_eo_scratch_bytes(C, nrhs))
      return fail(MGLMA_ERR_INVALID, "even-odd prepare: scratch too small");
    uint8_t* img = (uint8_t*)scratch;
    float2* bo = reinterpret_cast<float2*>(img + 2 * coarse_tc_half_image_bytes(C, nrhs));
    float2* wo = bo + nhalf;
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)b, bo, q, n2, nrhs, 1);
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)b, (float2*)be, q, n2, nrhs, 0);
    MG_LAUNCH_CHECK();
    // w_o = -D_oo^-1 b_o ; b_o <- D_eo w_o (even sites) ; b_e += b_o
    MG_CHECK(coarse_tc_eo_launch(ctx, C, nullptr, bo, wo, nrhs, 0, 1, 8, 8, C->Sinv_img, -1.f, img, s));
    MG_CHECK(coarse_tc_eo_launch(ctx, C, wo, nullptr, bo, nrhs, 0, 0, 0, 7, nullptr, 1.f, img, s));
    eo_axpy_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(1.0, bo, (float2*)be, nhalf);
    MG_LAUNCH_CHECK();
    return MGLMA_OK;
  }
  // composed path: F = embed_o(-D_oo^-1 b_o) ; T = D F ; b_e' = b_e + T_e
  const size_t cb = dp ? sizeof(double2) : sizeof(float2);
  const size_t nfull = 2 * nhalf;
  FreeList fl(ctx, s);
  void *F = nullptr, *T = nullptr, *H = nullptr;
  MG_CHECK(dalloc(ctx, &F, nfull * cb, s));
  fl.add(F);
  MG_CHECK(dalloc(ctx, &T, nfull * cb, s));
  fl.add(T);
  MG_CHECK(dalloc(ctx, &H, nhalf * cb, s));
  fl.add(H);
  MG_CUDA(cudaMemsetAsync(F, 0, nfull * cb, s));
  if (dp) {
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)b, (double2*)be, q, n2, nrhs, 1);
    self_inv_apply_kernel<double2><<<nblk(nhalf), 256, 0, s>>>(C->Sinv64, (const double2*)be, (double2*)H, q, n2,
                                                               nrhs, 1, -1.0);
    eo_scatter_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)H, (double2*)F, q, n2, nrhs, 1);
  } else {
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)b, (float2*)be, q, n2, nrhs, 1);
    self_inv_apply_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(C->Sinv64, (const float2*)be, (float2*)H, q, n2, nrhs,
                                                              1, -1.0);
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)H, (float2*)F, q, n2, nrhs, 1);
  }
  MG_LAUNCH_CHECK();
  MG_CHECK(coarse_apply(ctx, C, F, T, nrhs, prec, CMODE_D, s));
  if (dp) {
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)b, (double2*)be, q, n2, nrhs, 0);
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)T, (double2*)H, q, n2, nrhs, 0);
    eo_axpy_kernel<double2><<<nblk(nhalf), 256, 0, s>>>(1.0, (const double2*)H, (double2*)be, nhalf);
  } else {
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)b, (float2*)be, q, n2, nrhs, 0);
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)T, (float2*)H, q, n2, nrhs, 0);
    eo_axpy_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(1.0, (const float2*)H, (float2*)be, nhalf);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status coarse_eo_reconstruct(mglma_ctx ctx, const mglma_coarse_s* C, const void* b, const void* xe, void* x,
                                   int nrhs, int prec, void* scratch, size_t scratch_bytes, cudaStream_t s) {
  const LatIdx q = make_latidx(C->geo.Lb);
  const int n2 = C->n2;
  const size_t nhalf = (size_t)nrhs * (q.V / 2) * n2;
  const bool dp = prec == MGLMA_FP64;
  ProfScope ps(ctx, K_COARSE, s);
  if (!dp && C->Aimg && C->Sinv_img) {
    if (!scratch || scratch_bytes < coarse_eo_scratch_bytes(C, nrhs))
      return fail(MGLMA_ERR_INVALID, "even-odd reconstruct: scratch too small");
    uint8_t* img = (uint8_t*)scratch;
    float2* to = reinterpret_cast<float2*>(img + 2 * coarse_tc_half_image_bytes(C, nrhs));
    float2* ro = to + nhalf;
    // t_o = D_oe x_e ; r_o = b_o - t_o ; x_o = D_oo^-1 r_o ; x = (x_e, x_o)
    MG_CHECK(coarse_tc_eo_launch(ctx, C, (const float2*)xe, nullptr, to, nrhs, 0, 1, 0, 7, nullptr, 1.f, img, s));
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)b, ro, q, n2, nrhs, 1);
    eo_axpy_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(-1.0, to, ro, nhalf);
    MG_LAUNCH_CHECK();
    MG_CHECK(coarse_tc_eo_launch(ctx, C, nullptr, ro, to, nrhs, 0, 1, 8, 8, C->Sinv_img, 1.f, img, s));
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)xe, (float2*)x, q, n2, nrhs, 0);
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(to, (float2*)x, q, n2, nrhs, 1);
    MG_LAUNCH_CHECK();
    return MGLMA_OK;
  }
  const size_t cb = dp ? sizeof(double2) : sizeof(float2);
  const size_t nfull = 2 * nhalf;
  FreeList fl(ctx, s);
  void *F = nullptr, *T = nullptr, *H = nullptr;
  MG_CHECK(dalloc(ctx, &F, nfull * cb, s));
  fl.add(F);
  MG_CHECK(dalloc(ctx, &T, nfull * cb, s));
  fl.add(T);
  MG_CHECK(dalloc(ctx, &H, nhalf * cb, s));
  fl.add(H);
  MG_CUDA(cudaMemsetAsync(F, 0, nfull * cb, s));
  if (dp) {
    eo_scatter_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)xe, (double2*)F, q, n2, nrhs, 0);
  } else {
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)xe, (float2*)F, q, n2, nrhs, 0);
  }
  MG_LAUNCH_CHECK();
  MG_CHECK(coarse_apply(ctx, C, F, T, nrhs, prec, CMODE_D, s));  // T_o = D_oe x_e
  if (dp) {
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)b, (double2*)H, q, n2, nrhs, 1);
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)T, (double2*)F, q, n2, nrhs, 1);
    eo_axpy_kernel<double2><<<nblk(nhalf), 256, 0, s>>>(-1.0, (const double2*)F, (double2*)H, nhalf);
    self_inv_apply_kernel<double2><<<nblk(nhalf), 256, 0, s>>>(C->Sinv64, (const double2*)H, (double2*)F, q, n2,
                                                               nrhs, 1, 1.0);
    eo_scatter_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)xe, (double2*)x, q, n2, nrhs, 0);
    eo_scatter_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)F, (double2*)x, q, n2, nrhs, 1);
  } else {
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)b, (float2*)H, q, n2, nrhs, 1);
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)T, (float2*)F, q, n2, nrhs, 1);
    eo_axpy_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(-1.0, (const float2*)F, (float2*)H, nhalf);
    self_inv_apply_kernel<float2><<<nblk(nhalf), 256, 0, s>>>(C->Sinv64, (const float2*)H, (float2*)F, q, n2, nrhs,
                                                              1, 1.0);
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)xe, (float2*)x, q, n2, nrhs, 0);
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)F, (float2*)x, q, n2, nrhs, 1);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status coarse_schur_full(mglma_ctx ctx, mglma_coarse_s* C, const void* X, void* Y, int nrhs, int prec,
                               int mode, cudaStream_t s) {
  MG_CHECK(coarse_eo_setup(ctx, C, s));
  const LatIdx q = make_latidx(C->geo.Lb);
  const int n2 = C->n2;
  const size_t nhalf = (size_t)nrhs * (q.V / 2) * n2;
  const size_t cb = prec == MGLMA_FP64 ? sizeof(double2) : sizeof(float2);
  FreeList fl(ctx, s);
  void *Xe = nullptr, *Ye = nullptr, *scr = nullptr;
  MG_CHECK(dalloc(ctx, &Xe, nhalf * cb, s));
  fl.add(Xe);
  MG_CHECK(dalloc(ctx, &Ye, nhalf * cb, s));
  fl.add(Ye);
  const size_t sb = coarse_eo_scratch_bytes(C, nrhs);
  MG_CHECK(dalloc(ctx, &scr, sb, s));
  fl.add(scr);
  MG_CUDA(cudaMemsetAsync(Y, 0, 2 * nhalf * cb, s));
  if (prec == MGLMA_FP64)
    eo_gather_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)X, (double2*)Xe, q, n2, nrhs, 0);
  else
    eo_gather_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)X, (float2*)Xe, q, n2, nrhs, 0);
  MG_LAUNCH_CHECK();
  MG_CHECK(coarse_schur_apply(ctx, C, Xe, Ye, nrhs, prec, mode, scr, sb, s));
  if (prec == MGLMA_FP64)
    eo_scatter_kernel<double2><<<nblk(nhalf), 256, 0, s>>>((const double2*)Ye, (double2*)Y, q, n2, nrhs, 0);
  else
    eo_scatter_kernel<float2><<<nblk(nhalf), 256, 0, s>>>((const float2*)Ye, (float2*)Y, q, n2, nrhs, 0);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

}  // namespace mglma
