// Exact estimator on the coarsest grid (Sec. "Exact estimator on the
// coarsest grid", Eq. G_LL:exact).  When the coarse space of a level is small
// (complex dimension n = V_c 2 Nv below about 10^4), its contribution to the
// translation-averaged correlator is evaluated exactly:
//     C(x0, y0) = -(1 / (3 L^3)) sum_{k=1}^{3} tr{ Gam_k(y0) Q_c^-1 Gam_k(x0) Q_c^-1 }
//     G(t)      = (1 / L0) sum_{y0} C(t + y0, y0)
// with Q_c = g5hat D_c the Hermitian coarse operator and Gam_k(x0) =
// calR gamma5 gamma_k P_{x0} calT the coarse matrices of Eq. coarse:gamma with
// an open fine time index x0.  Gam_k(x0) is block-diagonal over coarse sites
// (a block meets the slice x0 or not); level 1 computes it from the basis,
// an inner-level transfer sums it over the sites of a block times
// V_{l+1} / V_l.
//
// Q_c^-1 is formed densely in FP64 by Gauss-Jordan elimination with partial
// pivoting (Q_c is Hermitian but indefinite).  The trace is summed per
// (k, coarse site y, local time t) over all y2 in a fixed order, then over
// (k, y) per (x0, y0) in a fixed order, so the result does not depend on the
// launch configuration.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cplx.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "solver.h"
#include "subspace.h"

namespace mglma {

constexpr int64_t kExactMaxDim = 16384;  // largest dense coarse dimension accepted

// Gam on the next level: out[y][t2][i][j] = f sum_{z in B_y, local time of z
// = t2 / tbz} in[z][t2 % tbz][i][j], tbz the time extent of a parent block
__global__ void gamma_next_kernel(const double2* __restrict__ in, double2* __restrict__ out, BlockGeo g, int tbz,
                                  int n2, double f) {
  const int tb = tbz * g.b[0];
  const size_t per = (size_t)n2 * n2;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= (size_t)g.V1 * tb * per) return;
  const size_t ij = u % per;
  const int t2 = (int)((u / per) % tb);
  const int64_t y = (int64_t)(u / (per * tb));
  int yc[4];
  int64_t r = y;
  for (int m = 3; m >= 0; --m) {
    yc[m] = (int)(r % g.Lb[m]);
    r /= g.Lb[m];
  }
  const int zt = t2 / tbz;  // local time coordinate of z inside B_y
  double re = 0, im = 0;
  for (int j = 0; j < g.nB; ++j) {
    int kc[4];
    int q = j;
    for (int m = 3; m >= 0; --m) {
      kc[m] = q % g.b[m];
      q /= g.b[m];
    }
    if (kc[0] != zt) continue;
    int64_t z = 0;
    for (int m = 0; m < 4; ++m) z = z * g.L[m] + (int64_t)yc[m] * g.b[m] + kc[m];
    const double2 v = in[((size_t)z * tbz + (t2 % tbz)) * per + ij];
    re += v.x;
    im += v.y;
  }
  out[u] = make_double2(f * re, f * im);
}

// dense Q = g5hat D_c, row-major n x n: Q[(y,i), (y2,j)] = s_i sum_{d: nbr_d(y) = y2} A_d(y)[i][j]
__global__ void dense_q_kernel(const double2* __restrict__ A, double2* __restrict__ Q, LatIdx q, int n2) {
  const int64_t n = q.V * n2;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  const int64_t row = (int64_t)(e / n), col = (int64_t)(e % n);
  const int64_t y = row / n2, y2 = col / n2;
  const int i = (int)(row % n2), j = (int)(col % n2);
  int x[4];
  site_coords(q, y, x);
  double re = 0, im = 0;
  for (int d = 0; d < 9; ++d) {
    const int64_t z = d == 8 ? y : (d < 4 ? nbr_fwd(q, y, x, d) : nbr_bwd(q, y, x, d - 4));
    if (z != y2) continue;
    const double2 a = A[(((size_t)y * 9 + d) * n2 + j) * n2 + i];
    re += a.x;
    im += a.y;
  }
  const double sgn = i < n2 / 2 ? 1.0 : -1.0;
  Q[e] = make_double2(sgn * re, sgn * im);
}

// ---- Gauss-Jordan with partial pivoting, in place (row-major n x n)
// step k, 1: pivot row p = argmax_{r >= k} |Q[r][k]| (one CTA), swap rows k and p
__global__ void gj_pivot_kernel(double2* Q, int64_t n, int64_t k, int* perm, int* singular) {
  __shared__ double best[1024];
  __shared__ int64_t arg[1024];
  double b = -1;
  int64_t a = k;
  for (int64_t r = k + threadIdx.x; r < n; r += blockDim.x) {
    const double2 v = Q[r * n + k];
    const double m = v.x * v.x + v.y * v.y;
    if (m > b) {
      b = m;
      a = r;
    }
  }
  best[threadIdx.x] = b;
  arg[threadIdx.x] = a;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      const double o = best[threadIdx.x + h];
      const int64_t oa = arg[threadIdx.x + h];
      if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oa < arg[threadIdx.x])) {
        best[threadIdx.x] = o;
        arg[threadIdx.x] = oa;
      }
    }
    __syncthreads();
  }
  const int64_t p = arg[0];
  if (threadIdx.x == 0) {
    perm[k] = (int)p;
    if (!(best[0] > 0)) *singular = 1;
  }
  if (p != k)
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      const double2 t = Q[k * n + c];
      Q[k * n + c] = Q[p * n + c];
      Q[p * n + c] = t;
    }
}

// step k, 2: keep column k (before scaling) and 1 / Q[k][k]
__global__ void gj_column_kernel(const double2* __restrict__ Q, int64_t n, int64_t k, double2* col, double2* inv) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) col[r] = Q[r * n + k];
  if (r == 0) {
    const double2 a = Q[k * n + k];
    const double m = a.x * a.x + a.y * a.y;
    *inv = m > 0 ? make_double2(a.x / m, -a.y / m) : make_double2(0, 0);
  }
}

// step k, 3: row k scaled by 1 / Q[k][k], its pivot entry set to 1 / Q[k][k]
__global__ void gj_row_kernel(double2* Q, int64_t n, int64_t k, const double2* __restrict__ inv) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const Cx<double> d = cx(inv->x, inv->y);
  if (c == k) {
    Q[k * n + k] = make_double2(d.re, d.im);
  } else {
    const double2 v = Q[k * n + c];
    const Cx<double> w = cx(v.x, v.y) * d;
    Q[k * n + c] = make_double2(w.re, w.im);
  }
}

// step k, 4: every other row r: Q[r][c] -= col[r] Q[k][c] (c != k), Q[r][k] = -col[r] / Q[k][k]
__global__ void gj_eliminate_kernel(double2* Q, int64_t n, int64_t k, const double2* __restrict__ col,
                                    const double2* __restrict__ inv) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  const int64_t r = (int64_t)(e / n), c = (int64_t)(e % n);
  if (r == k) return;
  const double2 cr = col[r];
  if (c == k) {
    const Cx<double> w = -(cx(cr.x, cr.y) * cx(inv->x, inv->y));
    Q[e] = make_double2(w.re, w.im);
  } else {
    const double2 kc = Q[k * n + c], v = Q[e];
    Cx<double> w = cx(v.x, v.y);
    w = w - cx(cr.x, cr.y) * cx(kc.x, kc.y);
    Q[e] = make_double2(w.re, w.im);
  }
}

// the row swaps of the pivoting become column swaps of the inverse, applied
// in reverse order (one thread per row)
__global__ void gj_unpermute_kernel(double2* Q, int64_t n, const int* __restrict__ perm) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int64_t k = n - 1; k >= 0; --k) {
    const int64_t p = perm[k];
    if (p != k) {
      const double2 t = Q[r * n + k];
      Q[r * n + k] = Q[r * n + p];
      Q[r * n + p] = t;
    }
  }
}

// one CTA per (k, y, t): for every y2, X = Gam_k[y][t] M(y, y2), Y = M(y2, y) X,
// then part[(k V + y) tb + t][x0] += sum_{b,c} Gam_k[y2][t2][b][c] Y[c][b] for the
// time x0 of (y2, t2); the y2 loop runs in order, so the sum is fixed
__global__ void exact_trace_kernel(const double2* __restrict__ M, const double2* __restrict__ Gam, int64_t V,
                                   int n2, int tb, LatIdx q, int L0, double2* __restrict__ part) {
  extern __shared__ double2 sm[];
  double2* X = sm;             // n2 x n2
  double2* Y = sm + n2 * n2;   // n2 x n2
  double2* acc = Y + n2 * n2;  // L0 sums
  __shared__ double red[2][256];
  const int64_t n = V * n2;
  const int t = (int)(blockIdx.x % tb);
  const int64_t y = (int64_t)((blockIdx.x / tb) % V);
  const int kk = (int)(blockIdx.x / (tb * V));
  const double2* Gk = Gam + (size_t)kk * V * tb * n2 * n2;
  const double2* Gy = Gk + ((size_t)y * tb + t) * n2 * n2;
  for (int i = threadIdx.x; i < L0; i += blockDim.x) acc[i] = make_double2(0, 0);
  for (int64_t y2 = 0; y2 < V; ++y2) {
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {  // X = Gam[y][t] M(y, y2)
      const int a = e / n2, b = e % n2;
      Cx<double> s = cx(0.0, 0.0);
      for (int c = 0; c < n2; ++c) {
        const double2 g = Gy[a * n2 + c], m = M[(y * n2 + c) * n + y2 * n2 + b];
        cfma(s, cx(g.x, g.y), cx(m.x, m.y));
      }
      X[e] = make_double2(s.re, s.im);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {  // Y = M(y2, y) X
      const int a = e / n2, b = e % n2;
      Cx<double> s = cx(0.0, 0.0);
      for (int c = 0; c < n2; ++c) {
        const double2 m = M[(y2 * n2 + a) * n + y * n2 + c], x = X[c * n2 + b];
        cfma(s, cx(m.x, m.y), cx(x.x, x.y));
      }
      Y[e] = make_double2(s.re, s.im);
    }
    __syncthreads();
    int yc[4];
    site_coords(q, y2, yc);
    for (int t2 = 0; t2 < tb; ++t2) {
      const double2* G2 = Gk + ((size_t)y2 * tb + t2) * n2 * n2;
      double re = 0, im = 0;
      for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {  // sum_{b,c} G2[b][c] Y[c][b]
        const int b = e / n2, c = e % n2;
        const double2 g = G2[e], v = Y[c * n2 + b];
        re += g.x * v.x - g.y * v.y;
        im += g.x * v.y + g.y * v.x;
      }
      red[0][threadIdx.x] = re;
      red[1][threadIdx.x] = im;
      __syncthreads();
      for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
          red[0][threadIdx.x] += red[0][threadIdx.x + h];
          red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        const int x0 = yc[0] * tb + t2;
        acc[x0] = make_double2(acc[x0].x + red[0][0], acc[x0].y + red[1][0]);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L0; i += blockDim.x) part[(size_t)blockIdx.x * L0 + i] = acc[i];
}

// C[x0][y0] = -(1 / (3 L^3)) sum_k sum_{y on y0's coarse time slice} part[k][y][y0 % tb][x0]
__global__ void exact_reduce_kernel(const double2* __restrict__ part, LatIdx q, int tb, int L0, double scale,
                                    double2* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L0 * L0) return;
  const int x0 = e / L0, y0 = e % L0;
  const int64_t V = q.V;
  const int yt = y0 / tb, t = y0 % tb;
  const int64_t slice = V / q.L[0];
  double re = 0, im = 0;
  for (int kk = 0; kk < 3; ++kk)
    for (int64_t s = 0; s < slice; ++s) {
      const int64_t y = (int64_t)yt * slice + s;
      const double2 v = part[(((size_t)kk * V + y) * tb + t) * L0 + x0];
      re += v.x;
      im += v.y;
    }
  C[e] = make_double2(scale * re, scale * im);
}

// G(t) = (1 / L0) sum_{y0} C[(t + y0) mod L0][y0] (Eq. timetrans), one thread per t
__global__ void translation_average_kernel(const double2* __restrict__ C, int L0, double2* __restrict__ G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L0) return;
  double re = 0, im = 0;
  for (int y0 = 0; y0 < L0; ++y0) {
    const double2 v = C[(size_t)((t + y0) % L0) * L0 + y0];
    re += v.x;
    im += v.y;
  }
  G[t] = make_double2(re / L0, im / L0);
}

// out[x0][y][i][j] = Gam[y][x0 - yt tb][i][j] when block y (coarse time yt) covers
// fine slice x0, else 0
__global__ void gamma_scatter_kernel(const double2* __restrict__ Gam, double2* __restrict__ out, int64_t V,
                                     int64_t slice, int tb, int L0, int n2) {
  const size_t per = (size_t)n2 * n2;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= (size_t)L0 * V * per) return;
  const size_t ij = u % per;
  const int64_t y = (int64_t)((u / per) % V);
  const int x0 = (int)(u / (per * V));
  const int t = x0 - (int)(y / slice) * tb;
  out[u] = (t >= 0 && t < tb) ? Gam[((size_t)y * tb + t) * per + ij] : make_double2(0, 0);
}

// Gam_k for k = 1..3 of level C, [k][V_c][tb][n2][n2] FP64 (device, allocated here)
static mglma_status level_gamma(mglma_ctx ctx, const mglma_coarse_s* C, double2** out, int* tb_out, FreeList& fl,
                                cudaStream_t s) {
  if (!C->parent) {
    const size_t per = (size_t)C->geo.V1 * C->geo.b[0] * C->n2 * C->n2;
    MG_CHECK(dalloc(ctx, (void**)out, 3 * per * sizeof(double2), s));
    fl.add(*out);
    for (int k = 1; k <= 3; ++k) MG_CHECK(coarse_gamma_level1(ctx, C->sub, k, *out + (k - 1) * per, s));
    *tb_out = C->geo.b[0];
    return MGLMA_OK;
  }
  double2* in = nullptr;
  int tbz = 0;
  MG_CHECK(level_gamma(ctx, C->parent, &in, &tbz, fl, s));
  const int tb = tbz * C->geo.b[0];
  const size_t per = (size_t)C->geo.V1 * tb * C->n2 * C->n2;
  const size_t per_in = (size_t)C->geo.V * tbz * C->n2 * C->n2;
  MG_CHECK(dalloc(ctx, (void**)out, 3 * per * sizeof(double2), s));
  fl.add(*out);
  const double f = (double)C->geo.V1 / (double)C->geo.V;
  for (int k = 0; k < 3; ++k) {
    ProfScope ps(ctx, K_SETUP, s);
    gamma_next_kernel<<<(unsigned)((per + 255) / 256), 256, 0, s>>>(in + k * per_in, *out + k * per, C->geo, tbz,
                                                                    C->n2, f);
  }
  MG_LAUNCH_CHECK();
  *tb_out = tb;
  return MGLMA_OK;
}

// Q_c^-1 of level C into the caller's device buffer (n x n)
static mglma_status dense_inverse(mglma_ctx ctx, const mglma_coarse_s* C, double2* Q, cudaStream_t s) {
  const int64_t n = C->geo.V1 * C->n2;
  const size_t nn = (size_t)n * n;
  LatIdx q = make_latidx(C->geo.Lb);
  FreeList fl(ctx, s);
  double2 *col = nullptr, *inv = nullptr;
  int *perm = nullptr, *sing = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&col, n * sizeof(double2), s));
  fl.add(col);
  MG_CHECK(dalloc(ctx, (void**)&inv, sizeof(double2), s));
  fl.add(inv);
  MG_CHECK(dalloc(ctx, (void**)&perm, n * sizeof(int), s));
  fl.add(perm);
  MG_CHECK(dalloc(ctx, (void**)&sing, sizeof(int), s));
  fl.add(sing);
  MG_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
  ProfScope ps(ctx, K_SETUP, s);
  dense_q_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(C->A64, Q, q, C->n2);
  const unsigned gr = (unsigned)((n + 255) / 256), ge = (unsigned)((nn + 255) / 256);
  for (int64_t k = 0; k < n; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, s>>>(Q, n, k, perm, sing);
    gj_column_kernel<<<gr, 256, 0, s>>>(Q, n, k, col, inv);
    gj_row_kernel<<<gr, 256, 0, s>>>(Q, n, k, inv);
    gj_eliminate_kernel<<<ge, 256, 0, s>>>(Q, n, k, col, inv);
  }
  gj_unpermute_kernel<<<gr, 256, 0, s>>>(Q, n, perm);
  MG_LAUNCH_CHECK();
  int hs = 0;
  MG_CUDA(cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  if (hs) return fail(MGLMA_ERR_NUMERIC, "exact coarse level: Q_c is singular");
  return MGLMA_OK;
}

static mglma_status exact_checks(mglma_ctx ctx, mglma_coarse C, const char* who) {
  if (!ctx || !C) return fail(MGLMA_ERR_INVALID, std::string(who) + ": NULL argument");
  if (!C->A64) return fail(MGLMA_ERR_INVALID, std::string(who) + ": the level's FP64 operator was released");
  const int64_t n = C->geo.V1 * C->n2;
  if (n > kExactMaxDim)
    return fail(MGLMA_ERR_INVALID, std::string(who) + ": coarse dimension " + std::to_string(n) + " above the " +
                                       std::to_string(kExactMaxDim) + " of a dense inverse");
  return MGLMA_OK;
}

}  // namespace mglma

using namespace mglma;

extern "C" {

mglma_status mglma_coarse_gamma5_gamma(mglma_ctx ctx, mglma_coarse C, int k, double* out) {
  if (!ctx || !C || !out) return fail(MGLMA_ERR_INVALID, "coarse_gamma5_gamma: NULL argument");
  if (k < 1 || k > 3) return fail(MGLMA_ERR_INVALID, "coarse_gamma5_gamma: k must be 1, 2 or 3");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  FreeList fl(ctx, s);
  double2* G = nullptr;
  int tb = 0;
  MG_CHECK(level_gamma(ctx, C, &G, &tb, fl, s));
  const int L0 = C->sub->geo.L[0];
  const int n2 = C->n2;
  const int64_t V = C->geo.V1;
  const size_t per = (size_t)n2 * n2;
  const size_t total = (size_t)L0 * V * per;
  Staged so;
  MG_CHECK(stage_out_alloc(ctx, out, total * sizeof(double2), s, so));
  const double2* Gk = G + (size_t)(k - 1) * V * tb * per;
  gamma_scatter_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Gk, (double2*)so.dev, V,
                                                                       V / C->geo.Lb[0], tb, L0, n2);
  MG_LAUNCH_CHECK();
  MG_CHECK(stage_out_finish(out, total * sizeof(double2), s, so));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

mglma_status mglma_coarse_dense_inverse(mglma_ctx ctx, mglma_coarse C, double* out) {
  MG_CHECK(exact_checks(ctx, C, "coarse_dense_inverse"));
  if (!out) return fail(MGLMA_ERR_INVALID, "coarse_dense_inverse: NULL output");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const int64_t n = C->geo.V1 * C->n2;
  Staged so;
  MG_CHECK(stage_out_alloc(ctx, out, (size_t)n * n * sizeof(double2), s, so));
  MG_CHECK(dense_inverse(ctx, C, (double2*)so.dev, s));
  MG_CHECK(stage_out_finish(out, (size_t)n * n * sizeof(double2), s, so));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

mglma_status mglma_exact_correlator(mglma_ctx ctx, mglma_coarse C, double* corr, double* G) {
  MG_CHECK(exact_checks(ctx, C, "exact_correlator"));
  if (!corr && !G) return fail(MGLMA_ERR_INVALID, "exact_correlator: no output");
  if (C->n2 > 80) return fail(MGLMA_ERR_INVALID, "exact_correlator: more than 80 coarse dofs per site");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const int64_t V = C->geo.V1, n = V * C->n2;
  const int n2 = C->n2;
  const int L0 = C->sub->geo.L[0];
  const int64_t L3 = C->sub->geo.V / L0;
  FreeList fl(ctx, s);
  double2 *M = nullptr, *gam = nullptr, *part = nullptr, *Cd = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&M, (size_t)n * n * sizeof(double2), s));
  fl.add(M);
  MG_CHECK(dense_inverse(ctx, C, M, s));
  int tb = 0;
  MG_CHECK(level_gamma(ctx, C, &gam, &tb, fl, s));
  const size_t nblk = (size_t)3 * V * tb;
  MG_CHECK(dalloc(ctx, (void**)&part, nblk * L0 * sizeof(double2), s));
  fl.add(part);
  MG_CHECK(dalloc(ctx, (void**)&Cd, (size_t)L0 * L0 * sizeof(double2), s));
  fl.add(Cd);
  LatIdx q = make_latidx(C->geo.Lb);
  const int smem = (int)((2 * (size_t)n2 * n2 + L0) * sizeof(double2));
  MG_CUDA(cudaFuncSetAttribute(exact_trace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  {
    ProfScope ps(ctx, K_CONTRACT, s);
    exact_trace_kernel<<<(unsigned)nblk, 256, smem, s>>>(M, gam, V, n2, tb, q, L0, part);
    exact_reduce_kernel<<<(L0 * L0 + 255) / 256, 256, 0, s>>>(part, q, tb, L0, -1.0 / (3.0 * (double)L3), Cd);
  }
  MG_LAUNCH_CHECK();
  double2* Gd = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&Gd, (size_t)L0 * sizeof(double2), s));
  fl.add(Gd);
  translation_average_kernel<<<(L0 + 63) / 64, 64, 0, s>>>(Cd, L0, Gd);
  MG_LAUNCH_CHECK();
  if (corr) MG_CUDA(cudaMemcpyAsync(corr, Cd, (size_t)L0 * L0 * sizeof(double2), cudaMemcpyDefault, s));
  if (G) MG_CUDA(cudaMemcpyAsync(G, Gd, (size_t)L0 * sizeof(double2), cudaMemcpyDefault, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

}  // extern "C"
