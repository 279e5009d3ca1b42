// Inner levels of the multigrid hierarchy (Sec. "Multigrid decompositions").
//
// Level l >= 1 of the nested block decomposition has the coarse grid
// Lambda_l of V_l sites and 2 Nv dofs per site (chirality alpha, vector c).
// For l >= 1 the restrictor and prolongator to the next level act on each
// (alpha, c) separately:
//     (R_l psi_l)(y)     = sqrt(V_{l+1} / V_l) sum_{z in B_y} psi_l(z)
//     (T_l psi_{l+1})(z) = sqrt(V_{l+1} / V_l) psi_{l+1}(y(z))
// (R_l T_l = 1), and the operator of the next level is Q_{l+1} = R_l Q_l T_l.
// Because R_l acts per (alpha, c) it commutes with gamma5hat, so this is
// gamma5hat D_{l+1} with D_{l+1} = R_l D_l T_l -- again a nine-slot stencil
// of dense (2Nv x 2Nv) blocks on Lambda_{l+1}: slot d < 8 of y sums the
// slot-d blocks of the sites z in B_y whose slot-d hop crosses the face of
// B_y, slot 8 the self blocks and every block whose hop stays inside, all
// times V_{l+1} / V_l.  Every level's operator is applied by the same
// kernels as D1 (tensor cores for the BF16 copy).
//
// The pieces of the telescoping decomposition S = S_0 + ... + S_{N-1} act
// on a source through psi_l = calT_l D_l^-1 calR_l b with the compound
// transfers calR_l = R_{l-1} ... R_0 and calT_l = T_0 ... T_{l-1} (App.
// chirality turns calT_l Q_l^-1 calR_l gamma5 into this form):
// S_0 b = D^-1 b - psi_1, S_l b = psi_l - psi_{l+1}, S_{N-1} b = psi_{N-1}.
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "solver.h"
#include "subspace.h"

namespace mglma {

__device__ __forceinline__ void decompose(int64_t t, const int L[4], int c[4]) {
  for (int m = 3; m >= 0; --m) {
    c[m] = (int)(t % L[m]);
    t /= L[m];
  }
}
__device__ __forceinline__ int64_t compose(const int c[4], const int L[4]) {
  return (((int64_t)c[0] * L[1] + c[1]) * L[2] + c[2]) * L[3] + c[3];
}

// out[r][y][k] = f sum_{j < nB} in[r][z(y, j)][k], z(y, j) = y b + j on the parent grid
template <typename T>
__global__ void restrict_level_kernel(const T* __restrict__ in, T* __restrict__ out, BlockGeo g, int n2, int nrhs,
                                      double f) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nrhs * g.V1 * n2) return;
  const int k = (int)(t % n2);
  const int64_t y = (int64_t)((t / n2) % g.V1);
  const int r = (int)(t / ((size_t)n2 * g.V1));
  int yc[4], kc[4], zc[4];
  decompose(y, g.Lb, yc);
  double re = 0, im = 0;
  for (int j = 0; j < g.nB; ++j) {
    decompose(j, g.b, kc);
    for (int m = 0; m < 4; ++m) zc[m] = yc[m] * g.b[m] + kc[m];
    const T v = in[((size_t)r * g.V + compose(zc, g.L)) * n2 + k];
    re += (double)v.x;
    im += (double)v.y;
  }
  out[t].x = f * re;
  out[t].y = f * im;
}

// out[r][z][k] = f in[r][y(z)][k] (+ out)
template <typename T>
__global__ void prolong_level_kernel(const T* __restrict__ in, T* out, BlockGeo g, int n2, int nrhs, double f,
                                     int accumulate) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nrhs * g.V * n2) return;
  const int k = (int)(t % n2);
  const int64_t z = (int64_t)((t / n2) % g.V);
  const int r = (int)(t / ((size_t)n2 * g.V));
  int zc[4], yc[4];
  decompose(z, g.L, zc);
  for (int m = 0; m < 4; ++m) yc[m] = zc[m] / g.b[m];
  const T v = in[((size_t)r * g.V1 + compose(yc, g.Lb)) * n2 + k];
  double re = f * (double)v.x, im = f * (double)v.y;
  if (accumulate) {
    re += (double)out[t].x;
    im += (double)out[t].y;
  }
  out[t].x = re;
  out[t].y = im;
}

// A[y][t][j][i] of the next level (layout of mglma_coarse_s::A64) from the
// parent's A1[z][d][j][i]: one thread per (y, t, j, i)
__global__ void build_next_kernel(const double2* __restrict__ A1, double2* __restrict__ A, BlockGeo g, int n2,
                                  double f) {
  const size_t per = (size_t)n2 * n2;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= (size_t)g.V1 * 9 * per) return;
  const size_t ji = u % per;
  const int t = (int)((u / per) % 9);
  const int64_t y = (int64_t)(u / (per * 9));
  int yc[4], kc[4], zc[4];
  decompose(y, g.Lb, yc);
  double re = 0, im = 0;
  for (int j = 0; j < g.nB; ++j) {
    decompose(j, g.b, kc);
    for (int m = 0; m < 4; ++m) zc[m] = yc[m] * g.b[m] + kc[m];
    const double2* Az = A1 + (size_t)compose(zc, g.L) * 9 * per;
    for (int d = 0; d < 9; ++d) {
      int slot = 8;
      if (d < 8) {
        const int mu = d & 3;
        const bool leaves = d < 4 ? kc[mu] == g.b[mu] - 1 : kc[mu] == 0;
        slot = leaves ? d : 8;
      }
      if (slot != t) continue;
      const double2 a = Az[(size_t)d * per + ji];
      re += a.x;
      im += a.y;
    }
  }
  A[u] = make_double2(f * re, f * im);
}

static inline unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

mglma_status restrict_level(mglma_ctx ctx, const mglma_coarse_s* Cc, const void* in, void* out, int nrhs, int prec,
                            cudaStream_t s) {
  const BlockGeo& g = Cc->geo;
  const size_t n = (size_t)nrhs * g.V1 * Cc->n2;
  if (n == 0) return MGLMA_OK;
  const double f = std::sqrt((double)g.V1 / (double)g.V);
  const double cb = prec == MGLMA_FP64 ? 16.0 : 8.0;
  ProfScope ps(ctx, K_RESTRICT, s, (double)nrhs * (g.V + g.V1) * Cc->n2 * cb);
  if (prec == MGLMA_FP64)
    restrict_level_kernel<double2><<<blocks_for(n, 256), 256, 0, s>>>((const double2*)in, (double2*)out, g, Cc->n2,
                                                                      nrhs, f);
  else
    restrict_level_kernel<float2><<<blocks_for(n, 256), 256, 0, s>>>((const float2*)in, (float2*)out, g, Cc->n2,
                                                                     nrhs, f);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status prolong_level(mglma_ctx ctx, const mglma_coarse_s* Cc, const void* in, void* out, int nrhs, int prec,
                           bool accumulate, cudaStream_t s) {
  const BlockGeo& g = Cc->geo;
  const size_t n = (size_t)nrhs * g.V * Cc->n2;
  if (n == 0) return MGLMA_OK;
  const double f = std::sqrt((double)g.V1 / (double)g.V);
  const double cb = prec == MGLMA_FP64 ? 16.0 : 8.0;
  ProfScope ps(ctx, K_PROLONG, s, (double)nrhs * (g.V * (accumulate ? 2 : 1) + g.V1) * Cc->n2 * cb);
  const int acc = accumulate ? 1 : 0;
  if (prec == MGLMA_FP64)
    prolong_level_kernel<double2><<<blocks_for(n, 256), 256, 0, s>>>((const double2*)in, (double2*)out, g, Cc->n2,
                                                                     nrhs, f, acc);
  else
    prolong_level_kernel<float2><<<blocks_for(n, 256), 256, 0, s>>>((const float2*)in, (float2*)out, g, Cc->n2,
                                                                    nrhs, f, acc);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// one level-transfer entry point's shared checks and staging
static mglma_status level_transfer(mglma_ctx ctx, mglma_coarse Cc, int nrhs, const double* in, double* out,
                                   void* cuda_stream, bool down, const char* who) {
  if (!ctx || !Cc || !in || !out) return fail(MGLMA_ERR_INVALID, std::string(who) + ": NULL argument");
  if (Cc->level < 2 || !Cc->parent)
    return fail(MGLMA_ERR_INVALID, std::string(who) + ": needs an operator of level >= 2 (mglma_coarse_build_next)");
  if (nrhs < 0) return fail(MGLMA_ERR_INVALID, std::string(who) + ": nrhs < 0");
  if (nrhs == 0) return MGLMA_OK;
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, cuda_stream);
  const size_t nin = (size_t)nrhs * (down ? Cc->geo.V : Cc->geo.V1) * Cc->n2;
  const size_t nout = (size_t)nrhs * (down ? Cc->geo.V1 : Cc->geo.V) * Cc->n2;
  Staged si, so;
  MG_CHECK(stage_in(ctx, in, nin * sizeof(double2), s, si));
  MG_CHECK(stage_out_alloc(ctx, out, nout * sizeof(double2), s, so));
  if (down)
    MG_CHECK(restrict_level(ctx, Cc, si.dev, so.dev, nrhs, MGLMA_FP64, s));
  else
    MG_CHECK(prolong_level(ctx, Cc, si.dev, so.dev, nrhs, MGLMA_FP64, false, s));
  MG_CHECK(stage_out_finish(out, nout * sizeof(double2), s, so));
  return MGLMA_OK;
}

}  // namespace mglma

using namespace mglma;

extern "C" {

mglma_status mglma_coarse_build_next(mglma_ctx ctx, mglma_coarse parent, const int block[4], mglma_prec store,
                                     mglma_coarse* out) {
  if (!ctx || !parent || !block || !out) return fail(MGLMA_ERR_INVALID, "coarse_build_next: NULL argument");
  if (!parent->A64) return fail(MGLMA_ERR_INVALID, "coarse_build_next: the parent's FP64 operator was released");
  if (store != MGLMA_FP64 && store != MGLMA_FP32 && store != MGLMA_BF16)
    return fail(MGLMA_ERR_INVALID, "coarse_build_next: store must be FP64, FP32 or BF16");
  for (int m = 0; m < 4; ++m)
    if (block[m] < 1 || parent->geo.Lb[m] % block[m])
      return fail(MGLMA_ERR_INVALID, "coarse_build_next: block sides must divide the parent's coarse grid");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  mglma_coarse_s* Cc = new mglma_coarse_s();
  Cc->ctx = ctx;
  Cc->sub = parent->sub;
  Cc->nv = parent->nv;
  Cc->n2 = parent->n2;
  Cc->store = store;
  Cc->geo = make_blockgeo(parent->geo.Lb, block);
  Cc->level = parent->level + 1;
  Cc->parent = parent;
  const int n2 = Cc->n2;
  const size_t na = (size_t)Cc->geo.V1 * 9 * n2 * n2;
  if (cudaMalloc(&Cc->A64, na * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    delete Cc;
    return fail(MGLMA_ERR_OOM, "coarse_build_next: cannot allocate the operator");
  }
  mglma_status st = MGLMA_OK;
  {
    ProfScope ps(ctx, K_SETUP, s);
    build_next_kernel<<<blocks_for(na, 256), 256, 0, s>>>(parent->A64, Cc->A64, Cc->geo, n2,
                                                          (double)Cc->geo.V1 / (double)Cc->geo.V);
  }
  if (cudaGetLastError() != cudaSuccess) st = fail(MGLMA_ERR_CUDA, "coarse_build_next: launch failed");
  if (st == MGLMA_OK) st = coarse_store_copies(ctx, Cc, store, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == MGLMA_OK && e != cudaSuccess) st = fail(MGLMA_ERR_CUDA, cudaGetErrorString(e));
  if (st != MGLMA_OK) {
    mglma_coarse_free(Cc);
    return st;
  }
  *out = Cc;
  return MGLMA_OK;
}

mglma_status mglma_coarse_restrict(mglma_ctx ctx, mglma_coarse level, int nrhs, const double* in, double* out,
                                   void* cuda_stream) {
  return level_transfer(ctx, level, nrhs, in, out, cuda_stream, true, "coarse_restrict");
}

mglma_status mglma_coarse_prolong(mglma_ctx ctx, mglma_coarse level, int nrhs, const double* in, double* out,
                                  void* cuda_stream) {
  return level_transfer(ctx, level, nrhs, in, out, cuda_stream, false, "coarse_prolong");
}

mglma_status mglma_pieces(mglma_ctx ctx, mglma_gauge G, const mglma_coarse* levels, int nlevels, int nrhs,
                          const double* b, double* psi, double tol, void* cuda_stream) {
  if (!ctx || !G || !levels || !b || !psi) return fail(MGLMA_ERR_INVALID, "pieces: NULL argument");
  if (nlevels < 1 || nlevels > 8 || nrhs < 0 || !(tol > 0)) return fail(MGLMA_ERR_INVALID, "pieces: bad sizes");
  MG_CHECK(check_gauge_device(ctx, G, "pieces"));
  for (int k = 0; k < nlevels; ++k) {
    const mglma_coarse_s* C = levels[k];
    if (!C || !C->A64) return fail(MGLMA_ERR_INVALID, "pieces: every level needs its FP64 operator");
    if (C->level != k + 1 || (k > 0 && C->parent != levels[k - 1]))
      return fail(MGLMA_ERR_INVALID, "pieces: levels[k] must be the child of levels[k-1], levels[0] of level 1");
  }
  const mglma_subspace_s* S = levels[0]->sub;
  if (S->gauge != G) return fail(MGLMA_ERR_INVALID, "pieces: the basis belongs to another gauge field");
  if (nrhs == 0) return MGLMA_OK;
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, cuda_stream);
  const int64_t V = G->g.V;
  const size_t per = (size_t)V * 24 * sizeof(double);
  Staged sb, sp;
  MG_CHECK(stage_in(ctx, b, per * nrhs, s, sb));
  MG_CHECK(stage_out_alloc(ctx, psi, per * nrhs * nlevels, s, sp));
  FreeList fl(ctx, s);
  Spinor B;
  MG_CHECK(alloc_spinor(ctx, B, MGLMA_FP64, nrhs, V, s));
  fl.add(B.p);
  MG_CHECK(pack_spinor(ctx, sb.dev, B, s));
  // compound restrictions calR_l b, l = 1 .. nlevels (FP64)
  std::vector<void*> chain(nlevels, nullptr), X(nlevels, nullptr);
  for (int k = 0; k < nlevels; ++k) {
    const size_t nc = (size_t)nrhs * levels[k]->geo.V1 * levels[k]->n2 * sizeof(double2);
    MG_CHECK(dalloc(ctx, &chain[k], nc, s));
    fl.add(chain[k]);
    MG_CHECK(dalloc(ctx, &X[k], nc, s));
    fl.add(X[k]);
  }
  MG_CHECK(restrict_fine(ctx, S, B, chain[0], s));
  for (int k = 1; k < nlevels; ++k) MG_CHECK(restrict_level(ctx, levels[k], chain[k - 1], chain[k], nrhs, MGLMA_FP64, s));
  for (int k = 0; k < nlevels; ++k) {
    // X_k = D_k^-1 calR_k b, then back through T_{k-1} ... T_1 and T_0
    MG_CHECK(coarse_solve64(ctx, levels[k], chain[k], X[k], nrhs, tol, s));
    for (int j = k; j > 0; --j) MG_CHECK(prolong_level(ctx, levels[j], X[j], X[j - 1], nrhs, MGLMA_FP64, false, s));
    MG_CHECK(prolong_coarse(ctx, S, X[0], B, false, s));
    MG_CHECK(unpack_spinor(ctx, B, sp.dev + (size_t)k * nrhs * V * 24, s));
  }
  MG_CHECK(stage_out_finish(psi, per * nrhs * nlevels, s, sp));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

}  // extern "C"
