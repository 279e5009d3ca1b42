// Mixed-precision multigrid solve of D x = b and the propagator pieces.
//
// Outer FP64 defect correction (iterative refinement): r = b - D x in FP64,
// e = D^-1 (r / |r|) to a modest relative accuracy in FP32, x += |r| e, until
// the FP64 residual reaches tol.  Inner FP32 flexible GCR(m) preconditioned by
// the two-level correction of Sec. 2:
//     z = T0 D1^-1 R0 r      (coarse solve: GCR on the stencil D1, BF16/FP32
//                              operator, FP32 accumulation, loose tolerance)
//     z += MR_nu(D, r - D z) (nu minimal-residual smoothing steps)
// The pieces of Sec. 2: psi1 = T0 D1^-1 R0 b with D1^-1 solved to tol by a
// coarse FP64 defect correction, psi0 = x - psi1 (App. chirality:
// T Q1^-1 R gamma5 = T D1^-1 R when [P, gamma5] = 0).
//
// All RHS of a group advance together; every scalar is per RHS on the device
// and converged RHS are frozen by device-side masks, so a RHS's iterates do
// not depend on the other RHS of its group.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <thread>

#include "cplx.cuh"
#include "internal.h"
#include "minres.cuh"
#include "solver.h"
#include "subspace.h"

namespace mglma {

__global__ void gcr_coef_kernel(const double2* dots, const double* nw, double2* coef, int k, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * n) return;
  const double d = nw[t];
  coef[t] = d > 0 ? make_double2(dots[t].x / d, dots[t].y / d) : make_double2(0, 0);
}

__global__ void gcr_alpha_kernel(const double2* num, const double* nwk, const int* active, double2* a, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double d = nwk[r];
  a[r] = (active[r] && d > 0) ? make_double2(num[r].x / d, num[r].y / d) : make_double2(0, 0);
}

// Deferred FGCR iterate of slots 0..K: Z'_k = Z_k - sum_{j<k} c_kj Z'_j (c_kj =
// cz[(k m + j) n' + r] with n' = n) gives Z' = Z T, T unit upper triangular,
// and x += sum_k alpha_k Z'_k = sum_i beta_i Z_i with beta = T alpha; writes
// -beta_i into out[i n + r] (multi_axpy subtracts)
__global__ void gcr_beta_kernel(const double2* __restrict__ cz, const double2* __restrict__ az, int K, int m, int n,
                                double2* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  Cx<double> T[4][4];
  for (int k = 0; k <= K; ++k) {
    for (int i = 0; i <= K; ++i) T[i][k] = cx(i == k ? 1.0 : 0.0, 0.0);
    for (int j = 0; j < k; ++j) {
      const double2 c = cz[((size_t)k * m + j) * n + r];
      for (int i = 0; i <= j; ++i) T[i][k] = T[i][k] - cx(c.x, c.y) * T[i][j];
    }
  }
  for (int i = 0; i <= K; ++i) {
    Cx<double> b = cx(0.0, 0.0);
    for (int k = i; k <= K; ++k) {
      const double2 a = az[(size_t)k * n + r];
      b = b + T[i][k] * cx(a.x, a.y);
    }
    out[(size_t)i * n + r] = make_double2(-b.re, -b.im);
  }
}

__global__ void gcr_mask_kernel(const double* rr, const double* bb, double tol2, int* active, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  active[r] = active[r] && (rr[r] > tol2 * bb[r]) && (rr[r] == rr[r]);
}

__global__ void sqrt_kernel(const double* in, double* out, int n, int inverse) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double v = sqrt(in[r]);
  out[r] = inverse ? (v > 0 ? 1.0 / v : 0.0) : v;
}

using OpFn = std::function<mglma_status(const Vec& in, Vec& out)>;

struct GcrResult {
  int iterations = 0;
  std::vector<int> per_rhs;  // iterations while active (when polled every step)
};

// Persistent workspace of batched GCR(m) for up to `cap` RHS: m search
// directions Z and their images W (direction j of RHS r at j*cap + r), the
// residual, and the per-RHS scalars.  Reused across solves so CUDA graphs
// that captured its kernels stay valid.
// The operator with the FGCR dots of direction slot k taken in its own pass
// (dslash_gcr): out = A in; k = 0 -> nw = |out|^2, num = <out, r>; k > 0 ->
// dots[j n + r] = <W_j, out>, j < k
using AdFn = std::function<mglma_status(const Vec& in, Vec& out, int k, const Vec& W0, size_t wslot_reals,
                                        const Vec& r, double* nw, double2* num, double2* dots)>;

struct GcrWork {
  mglma_ctx ctx = nullptr;
  cudaStream_t s = nullptr;
  int cap = 0, m = 0;
  const AdFn* Ad = nullptr;  // when set, used for slots k <= 3 instead of A plus separate dots
  Vec proto;  // precision and reals per RHS
  void *Zp = nullptr, *Wp = nullptr, *rp = nullptr;
  Scalars sc;
  // deferred iterate (with Ad and m <= 4): the directions Z_k stay as the
  // preconditioner returned them; cz[k][j][n] holds the orthogonalisation
  // coefficients of slot k, az[k][n] its step, and the end of a restart
  // cycle adds sum_i beta_i Z_i to x (beta = T alpha, Z' = Z T)
  double2 *cz = nullptr, *az = nullptr;
  bool defer() const { return Ad && m <= 4; }
  ~GcrWork() {
    if (ctx) {
      dfree(ctx, Zp, s);
      dfree(ctx, Wp, s);
      dfree(ctx, rp, s);
      dfree(ctx, cz, s);
      dfree(ctx, az, s);
    }
  }
  mglma_status setup(mglma_ctx c, cudaStream_t st, const Vec& like, int capacity, int mm) {
    ctx = c;
    s = st;
    cap = capacity;
    m = mm;
    proto = like;
    proto.nrhs = cap;
    MG_CHECK(dalloc(ctx, &Zp, proto.bytes() * m, s));
    MG_CHECK(dalloc(ctx, &Wp, proto.bytes() * m, s));
    MG_CHECK(dalloc(ctx, &rp, proto.bytes(), s));
    MG_CHECK(sc.alloc(ctx, cap, m + 2, 2 * m + 2, s));
    MG_CHECK(dalloc(ctx, (void**)&cz, sizeof(double2) * (size_t)m * m * cap, s));
    MG_CHECK(dalloc(ctx, (void**)&az, sizeof(double2) * (size_t)m * cap, s));
    return red_scratch_ready(ctx, s);
  }
  size_t stride() const { return (size_t)cap * proto.n; }  // reals between directions
  Vec view(void* base, int j, int n) const {
    Vec v = proto;
    v.nrhs = n;
    v.p = (char*)base + (size_t)j * proto.bytes();
    return v;
  }
};

// x = 0, r = b, bb = |b|^2, active = (bb > 0)
static mglma_status gcr_init(GcrWork& w, const Vec& b, Vec& x) {
  const int n = b.nrhs;
  Vec r = w.view(w.rp, 0, n);
  double* bb = w.sc.d + (size_t)(w.m + 1) * w.cap;
  MG_CHECK(zero_vec(w.ctx, x, w.s));
  MG_CHECK(copy_vec(w.ctx, b, r, w.s));
  MG_CHECK(norm2(w.ctx, b, bb, w.s));
  ProfScope ps(w.ctx, K_SCALAR, w.s);
  MG_CHECK(fill_int(w.sc.active, 1, n, w.s));
  gcr_mask_kernel<<<(n + 63) / 64, 64, 0, w.s>>>(bb, bb, 0.0, w.sc.active, n);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// x += sum_{i<=K} beta_i Z_i: the deferred iterate of slots 0..K (see GcrWork)
static mglma_status gcr_flush(GcrWork& w, Vec& x, int n, int K) {
  double2* nb = w.sc.z;  // the dots of slot K are used up: -beta [i][n]
  {
    ProfScope ps(w.ctx, K_SCALAR, w.s);
    gcr_beta_kernel<<<(n + 63) / 64, 64, 0, w.s>>>(w.cz, w.az, K, w.m, n, nb);
    MG_LAUNCH_CHECK();
  }
  Vec Z0 = w.view(w.Zp, 0, n);
  return multi_axpy(w.ctx, Z0, w.stride(), K + 1, x, nb, w.s);
}

// iteration with direction slot k (no host interaction)
static mglma_status gcr_iter(GcrWork& w, const OpFn& A, const OpFn* M, Vec& x, int n, int k, double tol2) {
  mglma_ctx ctx = w.ctx;
  cudaStream_t s = w.s;
  const int cap = w.cap;
  double* nw = w.sc.d;  // [m][cap]
  double* rr = w.sc.d + (size_t)w.m * cap;
  double* bb = w.sc.d + (size_t)(w.m + 1) * cap;
  double2* dots = w.sc.z;
  double2* coef = w.sc.z + (size_t)w.m * cap;
  double2* num = w.sc.z + (size_t)2 * w.m * cap;
  double2* a = w.sc.z + (size_t)(2 * w.m + 1) * cap;
  Vec r = w.view(w.rp, 0, n), Z0 = w.view(w.Zp, 0, n), W0 = w.view(w.Wp, 0, n);
  Vec Zk = w.view(w.Zp, k, n), Wk = w.view(w.Wp, k, n);
  const int tb = 64, nb = (n + tb - 1) / tb;
  if (M) {
    MG_CHECK((*M)(r, Zk));
  } else {
    MG_CHECK(copy_vec(ctx, r, Zk, s));
  }
  if (w.Ad && k <= 3) {
    // the image with its dots in one pass; the orthogonalisation returns the
    // new image's norm and overlap with r in its own pass
    MG_CHECK((*w.Ad)(Zk, Wk, k, W0, w.stride(), r, nw + (size_t)k * n, num, dots));
    if (k > 0) {
      double2* ck = w.defer() ? w.cz + (size_t)k * w.m * n : coef;
      {
        ProfScope ps(ctx, K_SCALAR, s);
        gcr_coef_kernel<<<(k * n + 63) / 64, 64, 0, s>>>(dots, nw, ck, k, n);
      }
      if (w.defer())
        MG_CHECK(multi_axpy_nd(ctx, W0, w.stride(), k, Wk, ck, nullptr, nullptr, r, nw + (size_t)k * n, num, s));
      else
        MG_CHECK(multi_axpy_nd(ctx, W0, w.stride(), k, Wk, ck, &Z0, &Zk, r, nw + (size_t)k * n, num, s));
    }
  } else {
  MG_CHECK(A(Zk, Wk));
  if (k > 0) {
    // dots and coefficients are stored [j][n] (dense in n) for j < k
    MG_CHECK(multi_cdot(ctx, W0, w.stride(), k, Wk, dots, s));
    {
      ProfScope ps(ctx, K_SCALAR, s);
      gcr_coef_kernel<<<(k * n + 63) / 64, 64, 0, s>>>(dots, nw, coef, k, n);
    }
    MG_CHECK(multi_axpy(ctx, W0, w.stride(), k, Wk, coef, s, &Z0, &Zk));
  }
  MG_CHECK(norm2_cdot(ctx, Wk, r, nw + (size_t)k * n, num, s));
  }
  double2* ak = w.defer() ? w.az + (size_t)k * n : a;
  {
    ProfScope ps(ctx, K_SCALAR, s);
    gcr_alpha_kernel<<<nb, tb, 0, s>>>(num, nw + (size_t)k * n, w.sc.active, ak, n);
  }
  if (w.defer())
    MG_CHECK(axpy_norm(ctx, ak, Wk, r, rr, s));
  else
    MG_CHECK(axpy2_norm(ctx, a, Zk, x, Wk, r, rr, s));
  {
    ProfScope ps(ctx, K_SCALAR, s);
    gcr_mask_kernel<<<nb, tb, 0, s>>>(rr, bb, tol2, w.sc.active, n);
  }
  MG_LAUNCH_CHECK();
  if (w.defer() && k == w.m - 1) MG_CHECK(gcr_flush(w, x, n, k));
  return MGLMA_OK;
}

static mglma_status read_active(GcrWork& w, int n, std::vector<int>& h) {
  h.resize(n);
  MG_CUDA(cudaMemcpyAsync(h.data(), w.sc.active, sizeof(int) * n, cudaMemcpyDeviceToHost, w.s));
  MG_CUDA(cudaStreamSynchronize(w.s));
  return MGLMA_OK;
}

// Batched flexible GCR(m): x = A^-1 b per RHS to |r| <= tol |b| (or max_iter).
// M (nullable) is the right preconditioner.  poll_every > 0 reads the active
// mask on the host every that many iterations and stops when all converged.
// tol_scale (nullable, host, n entries): RHS r stops at |r| <= tol *
// tol_scale[r] * |b_r| instead of tol * |b_r|.
// Graphs of whole FGCR iterations, one per direction slot k, captured on
// first use; valid while the workspace, the iterate and the operators keep
// their buffers (one defect-correction solve).
struct IterGraphs {
  std::vector<cudaGraphExec_t> ex;
  std::function<mglma_status(bool)> set_capturing;  // preconditioner: record its coarse loop on the device
  std::function<bool()> ready;                       // the operators were used once uncaptured
  ~IterGraphs() {
    for (auto e : ex)
      if (e) cudaGraphExecDestroy(e);
  }
};

static mglma_status gcr_run(GcrWork& w, const OpFn& A, const OpFn* M, const Vec& b, Vec& x, int max_iter, double tol,
                            int poll_every, GcrResult& res, const std::vector<double>* tol_scale,
                            IterGraphs* graphs);

static mglma_status gcr(mglma_ctx ctx, cudaStream_t s, const OpFn& A, const OpFn* M, const Vec& b, Vec& x, int m,
                        int max_iter, double tol, int poll_every, GcrResult& res,
                        const std::vector<double>* tol_scale = nullptr) {
  res = GcrResult();
  res.per_rhs.assign(b.nrhs, 0);
  if (b.nrhs == 0) return MGLMA_OK;
  GcrWork w;
  MG_CHECK(w.setup(ctx, s, b, b.nrhs, m));
  return gcr_run(w, A, M, b, x, max_iter, tol, poll_every, res, tol_scale, nullptr);
}

// one FGCR iteration of slot k as a graph (captured on first use)
static mglma_status gcr_iter_graphed(GcrWork& w, const OpFn& A, const OpFn* M, Vec& x, int n, int k, double tol2,
                                     IterGraphs& G) {
  if ((int)G.ex.size() < w.m) G.ex.assign(w.m, nullptr);
  if (!G.ex[k]) {
    MG_CHECK(G.set_capturing(true));
    MG_CUDA(cudaStreamBeginCapture(w.s, cudaStreamCaptureModeThreadLocal));
    mglma_status st = gcr_iter(w, A, M, x, n, k, tol2);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(w.s, &g);
    G.set_capturing(false);
    if (st != MGLMA_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != MGLMA_OK ? st : fail(MGLMA_ERR_CUDA, std::string("FGCR iteration capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      return fail(MGLMA_ERR_CUDA, std::string("FGCR iteration instantiate: ") + cudaGetErrorString(ei));
    }
    G.ex[k] = ex;
  }
  MG_CUDA(cudaGraphLaunch(G.ex[k], w.s));
  return MGLMA_OK;
}

static mglma_status gcr_run(GcrWork& w, const OpFn& A, const OpFn* M, const Vec& b, Vec& x, int max_iter, double tol,
                            int poll_every, GcrResult& res, const std::vector<double>* tol_scale,
                            IterGraphs* graphs) {
  const int n = b.nrhs;
  const int m = w.m;
  cudaStream_t s = w.s;
  res = GcrResult();
  res.per_rhs.assign(n, 0);
  if (n == 0) return MGLMA_OK;
  MG_CHECK(gcr_init(w, b, x));
  if (tol_scale) {
    // the mask compares |r|^2 with tol^2 |b|^2: scale the stored |b|^2
    double* bb = w.sc.d + (size_t)(w.m + 1) * w.cap;
    std::vector<double> hb;
    MG_CHECK(read_doubles(bb, hb, n, s));
    for (int i = 0; i < n; ++i) hb[i] *= (*tol_scale)[i] * (*tol_scale)[i];
    MG_CUDA(cudaMemcpyAsync(bb, hb.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    MG_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int> hact, prev;
  if (poll_every == 1) MG_CHECK(read_active(w, n, prev));
  int it = 0;
  while (it < max_iter) {
    if (graphs && graphs->ready())
      MG_CHECK(gcr_iter_graphed(w, A, M, x, n, it % m, tol * tol, *graphs));
    else
      MG_CHECK(gcr_iter(w, A, M, x, n, it % m, tol * tol));
    ++it;
    if (poll_every > 0 && (it % poll_every == 0 || it == max_iter)) {
      MG_CHECK(read_active(w, n, hact));
      bool any = false;
      for (int i = 0; i < n; ++i) {
        if (poll_every == 1 && prev[i]) res.per_rhs[i]++;  // active going into this iteration
        any = any || hact[i];
      }
      prev = hact;
      if (!any) break;
    }
  }
  // the deferred iterate of a cycle cut short
  if (w.defer() && it > 0 && (it - 1) % m != m - 1) MG_CHECK(gcr_flush(w, x, n, (it - 1) % m));
  res.iterations = it;
  if (poll_every != 1)
    for (int i = 0; i < n; ++i) res.per_rhs[i] = it;
  return MGLMA_OK;
}

// ------------------------------------------------------------------ MINRES
// Batched MINRES on the Hermitian coarse operator Qhat = g5hat Dhat, solving
// Qhat e = g5hat b (the same e as Dhat e = b; g5hat is unitary, so the
// recurrence's residual estimate |eta| is |b - Dhat e|).  Per RHS, iteration
// k (v_0 = g5hat b / beta_1, beta_0 = 0, v_-1 = w_-1 = w_-2 = 0):
//   Lanczos  z = Qhat v_k - alpha_k v_k - beta_k v_(k-1),  alpha_k = <v_k, Qhat v_k>,
//            beta_(k+1) = |z|,  v_(k+1) = z / beta_(k+1)
//   QR of the tridiagonal by Givens rotations (c, s):
//            eps = s'' beta_k, d' = c'' beta_k, delta = c' d' + s' alpha_k,
//            g' = c' alpha_k - s' d', gamma = hypot(g', beta_(k+1)),
//            c = g' / gamma, s = beta_(k+1) / gamma
//   update   w_k = (v_k - delta w_(k-1) - eps w_(k-2)) / gamma,
//            e += c eta w_k,  eta <- -s eta
// stopping at |eta| <= tol beta_1.  Vectors rotate through three slots
// (v_j, w_j in slot j mod 3), so a captured cycle is a multiple of three
// iterations long.

__global__ void minres_init_kernel(double* st, int* active, int cap, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  auto S = [&](int j) -> double& { return st[(size_t)j * cap + r]; };
  const double b1 = sqrt(S(MR_BB));
  const bool on = b1 > 0 && b1 < INFINITY;
  S(MR_BETA1) = b1;
  S(MR_ETA) = b1;
  S(MR_BETA) = 0;
  S(MR_C2) = S(MR_C1) = 1;
  S(MR_S2) = S(MR_S1) = 0;
  S(MR_CF + 4) = on ? 1.0 / b1 : 0.0;
  active[r] = on ? 1 : 0;
}

__global__ void minres_scalar_kernel(double* st, const double2* dot, int* active, double tol, int cap, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) minres_scalar_step(st, dot, active, tol, cap, r);
}

struct MinresWork {
  mglma_ctx ctx = nullptr;
  cudaStream_t s = nullptr;
  int cap = 0;
  Vec proto;
  void *Vp = nullptr, *Wp = nullptr;  // three Lanczos vectors, three directions
  Scalars sc;                         // d: MR_COUNT per RHS, z: <v, Qhat v>
  ~MinresWork() {
    if (ctx) {
      dfree(ctx, Vp, s);
      dfree(ctx, Wp, s);
    }
  }
  mglma_status setup(mglma_ctx c, cudaStream_t st, const Vec& like, int capacity) {
    ctx = c;
    s = st;
    cap = capacity;
    proto = like;
    proto.nrhs = cap;
    MG_CHECK(dalloc(ctx, &Vp, proto.bytes() * 3, s));
    MG_CHECK(dalloc(ctx, &Wp, proto.bytes() * 3, s));
    MG_CHECK(sc.alloc(ctx, cap, MR_COUNT, 1, s));
    return red_scratch_ready(ctx, s);
  }
  double* st(int j) const { return sc.d + (size_t)j * cap; }
  Vec view(void* base, int j, int n) const {
    Vec v = proto;
    v.nrhs = n;
    v.p = (char*)base + (size_t)j * proto.bytes();
    return v;
  }
};

static mglma_status minres_init(MinresWork& w, const mglma_coarse_s* C, const Vec& b, Vec& x) {
  const int n = b.nrhs;
  Vec v0 = w.view(w.Vp, 0, n), vm = w.view(w.Vp, 2, n), w1 = w.view(w.Wp, 1, n), w2 = w.view(w.Wp, 2, n);
  MG_CHECK(zero_vec(w.ctx, x, w.s));
  MG_CHECK(zero_vec(w.ctx, vm, w.s));
  MG_CHECK(zero_vec(w.ctx, w1, w.s));
  MG_CHECK(zero_vec(w.ctx, w2, w.s));
  MG_CHECK(norm2(w.ctx, b, w.st(MR_BB), w.s));
  {
    ProfScope ps(w.ctx, K_SCALAR, w.s);
    minres_init_kernel<<<(n + 63) / 64, 64, 0, w.s>>>(w.sc.d, w.sc.active, w.cap, n);
    MG_LAUNCH_CHECK();
  }
  return coarse_g5_scale(w.ctx, b, v0, w.st(MR_CF + 4), C->n2, w.s);
}

// eo: the vectors hold the even sites only and the operator is g5hat S_ee
// (even-odd preconditioning, coarse_eo.cu), else all sites and g5hat D1
static mglma_status minres_iter(MinresWork& w, const mglma_coarse_s* C, Vec& x, int n, int k, double tol,
                                void* scr, size_t scr_bytes, bool eo = false) {
  const int a = k % 3, b = (k + 1) % 3, c = (k + 2) % 3;
  Vec v = w.view(w.Vp, a, n), vo = w.view(w.Vp, c, n), z = w.view(w.Vp, b, n);
  Vec wn = w.view(w.Wp, a, n), w1 = w.view(w.Wp, c, n), w2 = w.view(w.Wp, b, n);
  // alpha = <v, Qhat v>: in the last tensor-core launch's epilogue when it
  // can; then the operator's input image of v was written by the previous
  // update (or by the initialisation), the scalar step runs at the end of the
  // Lanczos-norm kernel, and the update writes the image of the next v
  const bool fused_dot = eo && coarse_schur_dot_ok(w.ctx, C, n, MGLMA_FP32);
  if (eo)
    MG_CHECK(coarse_schur_apply(w.ctx, C, v.p, z.p, n, MGLMA_FP32, CMODE_Q, scr, scr_bytes, w.s,
                                fused_dot ? w.sc.z : nullptr, fused_dot));
  else
    MG_CHECK(coarse_apply(w.ctx, C, v.p, z.p, n, MGLMA_FP32, CMODE_Q, w.s, scr, scr_bytes));
  if (fused_dot) {
    MG_CHECK(lanczos_norm(w.ctx, w.sc.z, w.st(MR_BETA), w.sc.active, v, vo, z, w.st(MR_BN2), w.s, w.sc.d, tol,
                          w.cap));
    return minres_update_image(w.ctx, C, w.st(MR_CF), w.cap, v, w1, w2, wn, x, z, scr, w.s);
  }
  MG_CHECK(cdot(w.ctx, v, z, w.sc.z, w.s));
  MG_CHECK(lanczos_norm(w.ctx, w.sc.z, w.st(MR_BETA), w.sc.active, v, vo, z, w.st(MR_BN2), w.s));
  {
    ProfScope ps(w.ctx, K_SCALAR, w.s);
    minres_scalar_kernel<<<(n + 63) / 64, 64, 0, w.s>>>(w.sc.d, w.sc.z, w.sc.active, tol, w.cap, n);
    MG_LAUNCH_CHECK();
  }
  return minres_update(w.ctx, w.st(MR_CF), w.cap, v, w1, w2, wn, x, z, w.s);
}

static mglma_status read_mask(const int* dev, int n, std::vector<int>& h, cudaStream_t s) {
  h.resize(n);
  MG_CUDA(cudaMemcpyAsync(h.data(), dev, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

// Body-end kernel of the captured coarse loop (a conditional WHILE node): one
// more cycle ran; the loop goes on while some RHS is still active and fewer
// than max_cycles cycles ran in this solve, so it always ends.  total counts
// the cycles of every solve (iteration statistics).
__global__ void coarse_loop_cond_kernel(const int* __restrict__ active, int n, int* cycles, long long* total,
                                        int max_cycles, cudaGraphConditionalHandle h) {
  int any = 0;
  for (int r = 0; r < n; ++r) any |= active[r];
  const int c = *cycles + 1;
  *cycles = c;
  *total += 1;
  cudaGraphSetConditional(h, (any && c < max_cycles) ? 1u : 0u);
}

// Coarse solve of the preconditioner with a persistent workspace: MINRES on
// Qhat (default), MINRES on g5hat S_ee of the even-odd preconditioned
// operator (the odd sites follow by back-substitution), or GCR(m) on Dhat.
// One cycle (m GCR iterations = one restart; 12 MINRES iterations) is
// captured as a CUDA graph and replayed, with one host poll of the
// convergence mask per cycle.  With profiling on, a separately captured copy
// records event brackets around every launch.
struct CoarseSolver {
  mglma_ctx ctx = nullptr;
  cudaStream_t s = nullptr;
  const mglma_coarse_s* C = nullptr;
  int method = MGLMA_COARSE_MINRES;
  int m = 16;
  int cap_hint = 0;
  GcrWork w;
  MinresWork mw;
  void* scr = nullptr;  // tensor-core apply work space (B images of X)
  size_t scr_bytes = 0;
  Vec be, xe;  // even-odd: the prepared source and the solution on the even sites
  // captured form (inside a graph of a whole FGCR iteration): the loop body is
  // captured on `side`; d_loop[0] counts the cycles of the current solve,
  // d_total (long long) all cycles since the last read
  cudaStream_t side = nullptr;
  int* d_loop = nullptr;
  long long* d_total = nullptr;
  struct Graphs {
    cudaGraphExec_t init = nullptr, cycle = nullptr;
    int n = -1;
    std::vector<mglma_ctx_s::Pending> ev_init, ev_cycle;
  } g[2];  // [0] plain, [1] with profiling events
  const void* gb = nullptr;
  void* gx = nullptr;
  double gtol = -1;
  bool warmed = false;
  ~CoarseSolver() {
    reset();
    if (scr) dfree(ctx, scr, s);
    if (be.p) dfree(ctx, be.p, s);
    if (xe.p) dfree(ctx, xe.p, s);
    if (d_loop) dfree(ctx, d_loop, s);
    if (d_total) dfree(ctx, d_total, s);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
  }
  // streams of this solver and of its workspaces (the captured loop body is
  // recorded on the side stream)
  void use_stream(cudaStream_t st) {
    s = st;
    w.s = st;
    mw.s = st;
    mw.sc.s = st;
    w.sc.s = st;
  }
  // prepares the captured form: side stream, its reduction scratch, counters
  mglma_status capture_ready() {
    if (side) return MGLMA_OK;
    MG_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    MG_CHECK(red_scratch_ready(ctx, side));
    MG_CHECK(dalloc(ctx, (void**)&d_loop, sizeof(int), s));
    MG_CHECK(dalloc(ctx, (void**)&d_total, sizeof(long long), s));
    MG_CUDA(cudaMemsetAsync(d_total, 0, sizeof(long long), s));
    MG_CUDA(cudaStreamSynchronize(side));
    MG_CUDA(cudaStreamSynchronize(s));
    return MGLMA_OK;
  }
  // cycles run by captured solves since the last call, times the cycle length
  mglma_status take_captured_iters(long long* iters) {
    if (!d_total) return MGLMA_OK;
    long long h = 0;
    MG_CUDA(cudaMemcpyAsync(&h, d_total, sizeof(long long), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaMemsetAsync(d_total, 0, sizeof(long long), s));
    MG_CUDA(cudaStreamSynchronize(s));
    *iters += h * cycle_len();
    return MGLMA_OK;
  }
  // e1 = D1^-1 b1 recorded into the graph being captured on s: init, then a
  // conditional WHILE node running whole cycles until every RHS converged or
  // ceil(max_iter / cycle) cycles ran, then (even-odd) the back-substitution
  mglma_status solve_captured(const Vec& b, Vec& x, double tol, int max_iter) {
    CoarseLevelScope level(ctx);
    const int n = b.nrhs;
    const int L = cycle_len();
    const int max_cycles = (max_iter + L - 1) / L;
    MG_CHECK(init(b, x));
    MG_CUDA(cudaMemsetAsync(d_loop, 0, sizeof(int), s));
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    MG_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &ed, &nd));
    if (cst != cudaStreamCaptureStatusActive) return fail(MGLMA_ERR_INVALID, "coarse solve: not inside a capture");
    cudaGraphConditionalHandle h;
    MG_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    MG_CUDA(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    MG_CUDA(cudaStreamBeginCaptureToGraph(side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const cudaStream_t main = s;
    use_stream(side);
    OpFn A = op();
    mglma_status st = MGLMA_OK;
    for (int k = 0; k < L && st == MGLMA_OK; ++k) st = iter(A, x, n, k, tol);
    if (st == MGLMA_OK) {
      coarse_loop_cond_kernel<<<1, 1, 0, side>>>(active(), n, d_loop, d_total, max_cycles, h);
      if (cudaGetLastError() != cudaSuccess) st = fail(MGLMA_ERR_CUDA, "coarse loop: condition launch failed");
    }
    use_stream(main);
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(side, &out);
    MG_CHECK(st);
    if (e != cudaSuccess) return fail(MGLMA_ERR_CUDA, std::string("coarse loop capture: ") + cudaGetErrorString(e));
    MG_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return finish(b, x);
  }
  // destroys one graph set (both execs, its event brackets) and marks it empty
  static void drop(Graphs& G) {
    if (G.init) cudaGraphExecDestroy(G.init);
    if (G.cycle) cudaGraphExecDestroy(G.cycle);
    G.init = G.cycle = nullptr;
    G.n = -1;
    for (auto* L : {&G.ev_init, &G.ev_cycle})
      for (auto& p : *L) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
      }
    G.ev_init.clear();
    G.ev_cycle.clear();
  }
  void reset() {
    for (auto& G : g) drop(G);
  }
  // even-odd runs on the tensor-core operator (whose parity-restricted
  // launches need no work memory beyond the solver's scratch, so they can be
  // recorded in graphs) with every coarse extent even and its set-up formed or
  // formable (the FP64 operator held); elsewhere it runs as MINRES on Q1
  bool eo() const {
    if (method != MGLMA_COARSE_MINRES_EO || !C->Aimg) return false;
    for (int m = 0; m < 4; ++m)
      if (C->geo.Lb[m] % 2) return false;
    return C->Sinv_img || C->A64;
  }
  bool minres() const { return method == MGLMA_COARSE_MINRES || eo(); }
  int cycle_len() const { return minres() ? 12 : m; }
  int capacity() const { return minres() ? mw.cap : w.cap; }
  const int* active() const { return minres() ? mw.sc.active : w.sc.active; }
  OpFn op() {
    return [this](const Vec& in, Vec& out) {
      return coarse_apply(ctx, C, in.p, out.p, in.nrhs, MGLMA_FP32, CMODE_D, s, scr, scr_bytes);
    };
  }
  mglma_status init(const Vec& b, Vec& x) {
    if (eo()) {  // b_e' = b_e - D_eo D_oo^-1 b_o, MINRES for x_e
      Vec bn = be, xn = xe;
      bn.nrhs = xn.nrhs = b.nrhs;
      MG_CHECK(coarse_eo_prepare(ctx, C, b.p, bn.p, b.nrhs, MGLMA_FP32, scr, scr_bytes, s));
      MG_CHECK(minres_init(mw, C, bn, xn));
      // the first Lanczos vector's operator image (the iterations' updates
      // write the later ones)
      if (coarse_schur_dot_ok(ctx, C, b.nrhs, MGLMA_FP32))
        MG_CHECK(coarse_x_image_half(ctx, C, mw.view(mw.Vp, 0, b.nrhs).p, b.nrhs, scr, s));
      return MGLMA_OK;
    }
    return minres() ? minres_init(mw, C, b, x) : gcr_init(w, b, x);
  }
  mglma_status iter(const OpFn& A, Vec& x, int n, int k, double tol) {
    if (eo()) {
      Vec xn = xe;
      xn.nrhs = n;
      return minres_iter(mw, C, xn, n, k, tol, scr, scr_bytes, true);
    }
    return minres() ? minres_iter(mw, C, x, n, k, tol, scr, scr_bytes) : gcr_iter(w, A, nullptr, x, n, k, tol * tol);
  }
  // even-odd: x_o = D_oo^-1 (b_o - D_oe x_e), x = (x_e, x_o)
  mglma_status finish(const Vec& b, Vec& x) {
    if (!eo()) return MGLMA_OK;
    return coarse_eo_reconstruct(ctx, C, b.p, xe.p, x.p, b.nrhs, MGLMA_FP32, scr, scr_bytes, s);
  }
  // captures the init and cycle graphs of n RHS into G; on any failure G is
  // left empty (no half-built set survives to be launched)
  mglma_status capture(Graphs& G, const Vec& b, Vec& x, double tol, bool prof) {
    drop(G);
    const mglma_status st = capture_parts(G, b, x, tol, prof);
    if (st != MGLMA_OK) {
      cudaGetLastError();
      drop(G);
    }
    return st;
  }
  mglma_status capture_parts(Graphs& G, const Vec& b, Vec& x, double tol, bool prof) {
    const int n = b.nrhs;
    OpFn A = op();
    for (int part = 0; part < 2; ++part) {
      cudaGraph_t graph = nullptr;
      ctx->capture_events = prof ? (part == 0 ? &G.ev_init : &G.ev_cycle) : nullptr;
      MG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      mglma_status st = MGLMA_OK;
      if (part == 0) {
        st = init(b, x);
      } else {
        for (int k = 0; k < cycle_len() && st == MGLMA_OK; ++k) st = iter(A, x, n, k, tol);
      }
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      ctx->capture_events = nullptr;
      if (st != MGLMA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return fail(MGLMA_ERR_CUDA, std::string("coarse graph capture: ") + cudaGetErrorString(e));
      cudaGraphExec_t ex = nullptr;
      e = cudaGraphInstantiate(&ex, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(MGLMA_ERR_CUDA, std::string("coarse graph instantiate: ") + cudaGetErrorString(e));
      (part == 0 ? G.init : G.cycle) = ex;
    }
    G.n = n;
    return MGLMA_OK;
  }
  // e1 = D1^-1 b1 to tol (or max_iter, rounded up to whole cycles)
  mglma_status solve(const Vec& b, Vec& x, double tol, int max_iter, long long* iters) {
    CoarseLevelScope level(ctx);
    const int n = b.nrhs;
    if (!capacity()) {
      const int c = std::max(n, cap_hint);
      if (eo()) {
        MG_CHECK(coarse_eo_setup(ctx, const_cast<mglma_coarse_s*>(C), s));
        be = b;
        be.nrhs = c;
        be.n = b.n / 2;  // the even sites
        xe = be;
        be.p = xe.p = nullptr;
        MG_CHECK(dalloc(ctx, &be.p, be.bytes(), s));
        MG_CHECK(dalloc(ctx, &xe.p, xe.bytes(), s));
        MG_CHECK(mw.setup(ctx, s, be, c));
      } else if (minres()) {
        MG_CHECK(mw.setup(ctx, s, b, c));
      } else {
        MG_CHECK(w.setup(ctx, s, b, c, m));
      }
      if (C->Aimg) {
        scr_bytes = std::max(coarse_tc_scratch_bytes(C, c), eo() ? coarse_eo_scratch_bytes(C, c) : (size_t)0);
        MG_CHECK(dalloc(ctx, &scr, scr_bytes, s));
      }
    }
    if (n > capacity()) return fail(MGLMA_ERR_INVALID, "coarse solve: more RHS than the workspace holds");
    const int L = cycle_len();
    const int cycles = (max_iter + L - 1) / L;
    std::vector<int> hact;
    const bool prof = ctx->profile;
    if (!warmed) {
      // first use runs uncaptured (kernel attributes and scratch get set up)
      OpFn A = op();
      MG_CHECK(init(b, x));
      int c = 0;
      for (; c < cycles; ++c) {
        for (int k = 0; k < L; ++k) MG_CHECK(iter(A, x, n, k, tol));
        MG_CHECK(read_mask(active(), n, hact, s));
        bool any = false;
        for (int v : hact) any = any || v;
        if (!any) {
          ++c;
          break;
        }
      }
      *iters += (long long)c * L;
      warmed = true;
      return finish(b, x);
    }
    if (b.p != gb || x.p != gx || tol != gtol) {
      reset();
      gb = b.p;
      gx = x.p;
      gtol = tol;
    }
    Graphs& G = g[prof ? 1 : 0];
    if (G.n != n || !G.init || !G.cycle) MG_CHECK(capture(G, b, x, tol, prof));
    MG_CUDA(cudaGraphLaunch(G.init, s));
    int c = 0;
    for (; c < cycles; ++c) {
      MG_CUDA(cudaGraphLaunch(G.cycle, s));
      MG_CHECK(read_mask(active(), n, hact, s));
      if (prof && c == 0) resolve_graph_events(ctx, G.ev_init);
      if (prof) resolve_graph_events(ctx, G.ev_cycle);
      bool any = false;
      for (int v : hact) any = any || v;
      if (!any) {
        ++c;
        break;
      }
    }
    *iters += (long long)c * L;
    return finish(b, x);
  }
};

static Spinor as_spinor(const Vec& v, int64_t V) {
  Spinor f;
  f.p = v.p;
  f.prec = v.prec;
  f.nrhs = v.nrhs;
  f.V = V;
  return f;
}

// The preconditioner K r = z (FP32): coarse correction then MR smoothing.
// Scratch is allocated on the first call and reused.
struct TwoLevel {
  mglma_ctx ctx;
  cudaStream_t s;
  const mglma_gauge_s* G;
  const mglma_coarse_s* C;
  const MgParams* p;
  long long coarse_iters = 0;
  int cap = 0;  // RHS the scratch is sized for (0: the first call's count)
  Vec b1, e1, sv, tv, tv2;
  double* part = nullptr;  // per-block partial sums of the fused MR reductions
  Scalars sc;
  CoarseSolver cs;
  bool ready = false;
  bool fused = false;      // fused MR steps on BF16 s, t
  bool tc_r0 = false;      // R0 on the tensor cores (BF16 operands; the coarse solve is BF16 already)
  bool tc_t0 = false;      // T0 on the tensor cores (BF16 operands)
  bool capturing = false;  // recording into a graph: the coarse loop runs on the device
  ~TwoLevel() {
    dfree(ctx, b1.p, s);
    dfree(ctx, e1.p, s);
    dfree(ctx, sv.p, s);
    dfree(ctx, tv.p, s);
    dfree(ctx, tv2.p, s);
    dfree(ctx, part, s);
  }
  mglma_status setup(const Vec& r) {
    const int n = std::max(cap, r.nrhs);
    cap = n;
    b1.prec = e1.prec = MGLMA_FP32;
    b1.nrhs = e1.nrhs = n;
    b1.n = e1.n = (size_t)C->geo.V1 * C->n2 * 2;
    MG_CHECK(dalloc(ctx, &b1.p, b1.bytes(), s));
    MG_CHECK(dalloc(ctx, &e1.p, e1.bytes(), s));
    // the smoother's s and t: BF16 on the fused path (the flexible outer
    // solve takes the rounded preconditioner; measured: same FGCR and coarse
    // iteration counts as FP32 at 64x32^3), FP32 otherwise
    fused = p->nu > 1 && dslash_mr_fused(ctx, G, n);
    tc_r0 = n >= 8 && restrict_tc_supported(C->sub);
    tc_t0 = n >= 8 && prolong_tc_supported(C->sub);
    sv = r;
    sv.nrhs = n;
    sv.p = nullptr;
    if (fused) sv.prec = MGLMA_BF16;
    tv = tv2 = sv;
    MG_CHECK(dalloc(ctx, &sv.p, sv.bytes(), s));
    MG_CHECK(dalloc(ctx, &tv.p, tv.bytes(), s));
    if (fused) MG_CHECK(dalloc(ctx, &tv2.p, tv2.bytes(), s));
    MG_CHECK(dalloc(ctx, (void**)&part, dslash_dot_part_doubles(C->sub->geo.V, n) * sizeof(double), s));
    MG_CHECK(sc.alloc(ctx, n, 1, 1, s));
    cs.ctx = ctx;
    cs.s = s;
    cs.C = C;
    cs.method = p->coarse_solver;
    cs.cap_hint = n;
    ready = true;
    return MGLMA_OK;
  }
  mglma_status operator()(const Vec& r, Vec& z) {
    if (!ready || r.nrhs > cap) {
      if (ready) return fail(MGLMA_ERR_INVALID, "preconditioner: more RHS than its scratch holds");
      MG_CHECK(setup(r));
    }
    const int n = r.nrhs;
    const mglma_subspace_s* S = C->sub;
    const int64_t V = S->geo.V;
    Vec b1n = b1, e1n = e1, svn = sv, tvn = tv, tv2n = tv2;
    b1n.nrhs = e1n.nrhs = svn.nrhs = tvn.nrhs = tv2n.nrhs = n;
    Spinor rs = as_spinor(r, V), zs = as_spinor(z, V);
    if (tc_r0)
      MG_CHECK(restrict_tc(ctx, const_cast<mglma_subspace_s*>(S), rs, b1n.p, s));
    else
      MG_CHECK(restrict_fine(ctx, S, rs, b1n.p, s));
    if (capturing)
      MG_CHECK(cs.solve_captured(b1n, e1n, p->coarse_tol, p->coarse_max_iter));
    else
      MG_CHECK(cs.solve(b1n, e1n, p->coarse_tol, p->coarse_max_iter, &coarse_iters));
    if (tc_t0)
      MG_CHECK(prolong_tc(ctx, const_cast<mglma_subspace_s*>(S), e1n.p, zs, s));
    else
      MG_CHECK(prolong_coarse(ctx, S, e1n.p, zs, false, s));
    if (p->nu > 0) {
      // s = r - D z (in the stencil's epilogue) ; nu MR steps on D e = s,
      // accumulated into z (the last one leaves s as it is)
      Spinor ss = as_spinor(svn, V), ts = as_spinor(tvn, V);
      MG_CHECK(dslash_resid(ctx, G, zs, rs, ss, s));
      if (fused) {
        // t_0 = D s_0 ; then each step's vector update rides on the next
        // step's stencil, t_{k+1} = t_k - alpha_k D t_k (dslash_mr_step)
        Spinor t2s = as_spinor(tv2n, V);
        Spinor *tc = &ts, *tn = &t2s;
        MG_CHECK(dslash_dot(ctx, G, ss, ts, part, sc.d, sc.z, s));
        MG_CHECK(mr_alpha(ctx, sc.z, sc.d, sc.z, n, s));
        for (int k = 1; k < p->nu; ++k) {
          MG_CHECK(dslash_mr_step(ctx, G, *tc, *tn, ss, zs, sc.z, part, sc.d, sc.z, s));
          MG_CHECK(mr_alpha(ctx, sc.z, sc.d, sc.z, n, s));
          std::swap(tc, tn);
        }
        MG_CHECK(mr_zupdate(ctx, sc.z, ss, zs, s));
      } else {
        for (int k = 0; k < p->nu; ++k) {
          // t = D s with |D s|^2 and <D s, s> reduced in the same pass
          MG_CHECK(dslash_dot(ctx, G, ss, ts, part, sc.d, sc.z, s));
          MG_CHECK(mr_alpha(ctx, sc.z, sc.d, sc.z, n, s));
          if (k + 1 < p->nu)
            MG_CHECK(axpy2(ctx, sc.z, svn, z, tvn, svn, s));
          else
            MG_CHECK(caxpy(ctx, sc.z, svn, z, s));
        }
      }
    }
    return MGLMA_OK;
  }
};

// Inner-tolerance factor for a RHS at FP64 relative residual `rel`: when
// this cycle can reach the target (inner_tol * rel < 10 tol), the inner solve
// aims at 0.3 tol / rel instead of inner_tol -- tighter when two cycles of
// inner_tol would land just above tol, looser when the RHS needs less than
// inner_tol to finish (no FGCR iterations spent below 0.3 tol).
static double final_cycle_scale(const MgParams& p, double rel) {
  if (!(rel > 0) || p.inner_tol * rel >= 10.0 * p.tol) return 1.0;
  return 0.3 * p.tol / (rel * p.inner_tol);
}

// x (FP64, zero on entry) = D^-1 b to p.tol in the FP64 residual.
mglma_status mg_solve(mglma_ctx ctx, const mglma_gauge_s* G, const mglma_coarse_s* C, const Spinor& b, Spinor& x,
                      const MgParams& p, std::vector<RhsStat>& out, cudaStream_t s) {
  const int n = b.nrhs;
  const int64_t V = b.V;
  out.assign(n, RhsStat());
  FreeList fl(ctx, s);
  Spinor r, r32, e32;
  MG_CHECK(alloc_spinor(ctx, r, MGLMA_FP64, n, V, s));
  fl.add(r.p);
  MG_CHECK(alloc_spinor(ctx, r32, MGLMA_FP32, n, V, s));
  fl.add(r32.p);
  MG_CHECK(alloc_spinor(ctx, e32, MGLMA_FP32, n, V, s));
  fl.add(e32.p);
  Scalars sc;
  MG_CHECK(sc.alloc(ctx, n, 4, 1, s));
  double* bb = sc.d;
  double* rr = sc.d + n;
  double* rn = sc.d + 2 * n;
  double* rinv = sc.d + 3 * n;
  Vec vb = as_vec(b), vx = as_vec(x), vr = as_vec(r);
  MG_CHECK(norm2(ctx, vb, bb, s));
  std::vector<double> hbb, hrr;
  MG_CHECK(read_doubles(bb, hbb, n, s));
  MG_CHECK(zero_vec(ctx, vx, s));
  MG_CHECK(copy_vec(ctx, vb, vr, s));
  TwoLevel K;
  K.ctx = ctx;
  K.s = s;
  K.G = G;
  K.C = C;
  K.p = &p;
  OpFn A = [&](const Vec& in, Vec& o) {
    Spinor a = as_spinor(in, V), bo = as_spinor(o, V);
    return dslash(ctx, G, a, bo, false, false, s);
  };
  OpFn Kf = [&](const Vec& in, Vec& o) { return K(in, o); };
  const int tb = 64, nb = (n + tb - 1) / tb;
  int total_inner = 0;
  // FGCR workspace kept over the defect-correction cycles; with p.graph each
  // FGCR iteration after the first runs as one captured graph (the coarse
  // loop as a device-side conditional node), unless per-launch profiling is on
  GcrWork gw;
  {
    Vec like = as_vec(r32);
    MG_CHECK(gw.setup(ctx, s, like, n, p.gcr_m));
  }
  double* gpart = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&gpart, dslash_gcr_part_doubles(V, n) * sizeof(double), s));
  fl.add(gpart);
  const AdFn Ad = [&](const Vec& in, Vec& o, int k, const Vec& W0, size_t wslot, const Vec& res, double* nw,
                      double2* num, double2* dots) {
    Spinor a = as_spinor(in, V), bo = as_spinor(o, V);
    return dslash_gcr(ctx, G, a, bo, k, W0.p, wslot, res.p, gpart, nw, num, dots, s);
  };
  gw.Ad = &Ad;
  IterGraphs graphs;
  const bool use_graphs = p.graph && !ctx->profile;
  graphs.set_capturing = [&](bool on) -> mglma_status {
    K.capturing = on;
    return on ? K.cs.capture_ready() : MGLMA_OK;
  };
  graphs.ready = [&]() { return K.ready && K.cs.warmed; };
  for (int cycle = 0;; ++cycle) {
    MG_CHECK(norm2(ctx, vr, rr, s));
    MG_CHECK(read_doubles(rr, hrr, n, s));
    bool any = false;
    for (int i = 0; i < n; ++i) {
      out[i].residual = hbb[i] > 0 ? std::sqrt(hrr[i] / hbb[i]) : 0.0;
      if (!std::isfinite(out[i].residual)) return fail(MGLMA_ERR_NUMERIC, "mg solve: non-finite residual");
      out[i].converged = out[i].residual <= p.tol;
      if (!out[i].converged) any = true;
    }
    if (!any) break;
    if (total_inner >= p.max_iter || cycle >= 50) return fail(MGLMA_ERR_NOT_CONVERGED, "mg solve: iteration cap reached");
    // r32 = r / |r| for RHS still above tol (converged RHS get a zero source)
    for (int i = 0; i < n; ++i)
      if (out[i].converged) hrr[i] = 0;
    MG_CUDA(cudaMemcpyAsync(rr, hrr.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    sqrt_kernel<<<nb, tb, 0, s>>>(rr, rinv, n, 1);
    sqrt_kernel<<<nb, tb, 0, s>>>(rr, rn, n, 0);
    MG_CHECK(convert_spinor(ctx, r, r32, s, rinv, false));
    Vec v32 = as_vec(r32), e = as_vec(e32);
    // a cycle that can finish a RHS aims at 0.3 tol: a little below what it
    // needs, and no further
    std::vector<double> scale(n, 1.0);
    for (int i = 0; i < n; ++i) scale[i] = final_cycle_scale(p, out[i].residual);
    GcrResult gr;
    MG_CHECK(gcr_run(gw, A, &Kf, v32, e, p.max_iter - total_inner, p.inner_tol, 1, gr, &scale,
                     use_graphs ? &graphs : nullptr));
    total_inner += gr.iterations;
    for (int i = 0; i < n; ++i) {
      out[i].iterations += gr.per_rhs[i];
      if (!out[i].converged) out[i].outer++;
    }
    // x += |r| e ; r -= |r| D e with D e taken in double-float on the exact
    // FP32 values of e, so r tracks b - D x to about 1e-14 |b| (the FP64
    // products |r| e that enter x are rounded once, below that)
    MG_CHECK(convert_spinor(ctx, e32, x, s, rn, true));
    MG_CHECK(dslash_resid_df(ctx, G, e32, r, rn, s));
  }
  MG_CHECK(K.cs.take_captured_iters(&K.coarse_iters));
  for (int i = 0; i < n; ++i) out[i].coarse_iterations = K.coarse_iters;
  if (K.tc_r0 || K.tc_t0) MG_CHECK(restrict_tc_check(C->sub, s));
  return coarse_tc_check(const_cast<mglma_coarse_s*>(C), s);
}

// X (FP64 coarse, [n][V1][n2]) = D1^-1 b1 to tol by FP64 defect correction
// around FP32 coarse GCR.
mglma_status coarse_solve64(mglma_ctx ctx, const mglma_coarse_s* C, const void* b1, void* X, int n, double tol,
                            cudaStream_t s) {
  CoarseLevelScope level(ctx);
  const size_t per = (size_t)C->geo.V1 * C->n2;  // complex per RHS
  FreeList fl(ctx, s);
  Vec vb, vx, vr, vw, r32, e32;
  vb.prec = vx.prec = vr.prec = vw.prec = MGLMA_FP64;
  r32.prec = e32.prec = MGLMA_FP32;
  vb.nrhs = vx.nrhs = vr.nrhs = vw.nrhs = r32.nrhs = e32.nrhs = n;
  vb.n = vx.n = vr.n = vw.n = r32.n = e32.n = per * 2;
  vb.p = const_cast<void*>(b1);
  vx.p = X;
  MG_CHECK(dalloc(ctx, &vr.p, vr.bytes(), s));
  fl.add(vr.p);
  MG_CHECK(dalloc(ctx, &vw.p, vw.bytes(), s));
  fl.add(vw.p);
  MG_CHECK(dalloc(ctx, &r32.p, r32.bytes(), s));
  fl.add(r32.p);
  MG_CHECK(dalloc(ctx, &e32.p, e32.bytes(), s));
  fl.add(e32.p);
  Scalars sc;
  MG_CHECK(sc.alloc(ctx, n, 4, 1, s));
  double *bb = sc.d, *rr = sc.d + n, *rn = sc.d + 2 * n, *rinv = sc.d + 3 * n;
  MG_CHECK(norm2(ctx, vb, bb, s));
  std::vector<double> hbb, hrr;
  MG_CHECK(read_doubles(bb, hbb, n, s));
  MG_CHECK(zero_vec(ctx, vx, s));
  MG_CHECK(copy_vec(ctx, vb, vr, s));
  OpFn Ac = [&](const Vec& in, Vec& out) { return coarse_apply(ctx, C, in.p, out.p, in.nrhs, MGLMA_FP32, CMODE_D, s); };
  const int tb = 64, nb = (n + tb - 1) / tb;
  for (int cycle = 0; cycle < 40; ++cycle) {
    MG_CHECK(norm2(ctx, vr, rr, s));
    MG_CHECK(read_doubles(rr, hrr, n, s));
    bool any = false;
    for (int i = 0; i < n; ++i) {
      if (hbb[i] > 0 && std::sqrt(hrr[i] / hbb[i]) > tol) {
        any = true;
      } else {
        hrr[i] = 0;
      }
    }
    if (!any) return MGLMA_OK;
    MG_CUDA(cudaMemcpyAsync(rr, hrr.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    sqrt_kernel<<<nb, tb, 0, s>>>(rr, rinv, n, 1);
    sqrt_kernel<<<nb, tb, 0, s>>>(rr, rn, n, 0);
    // r32 = r / |r| ; e = D1^-1 r32 (FP32) ; X += |r| e ; r = b1 - D1 X (FP64)
    MG_CHECK(coarse_scale_convert(ctx, vr.p, MGLMA_FP64, r32.p, MGLMA_FP32, rinv, per, n, false, s));
    GcrResult gr;
    MG_CHECK(gcr(ctx, s, Ac, nullptr, r32, e32, 24, 4000, 1e-6, 20, gr));
    MG_CHECK(coarse_scale_convert(ctx, e32.p, MGLMA_FP32, vx.p, MGLMA_FP64, rn, per, n, true, s));
    MG_CHECK(coarse_apply(ctx, C, vx.p, vw.p, n, MGLMA_FP64, CMODE_D, s));
    MG_CHECK(copy_vec(ctx, vb, vr, s));
    MG_CHECK(axpby(ctx, nullptr, CM1, vw, nullptr, C1, vr, s));
  }
  return fail(MGLMA_ERR_NOT_CONVERGED, "coarse solve: FP64 defect correction did not reach tol");
}

// ============================================================ continuous-batching engine
// One resident lattice (gauge field, basis, coarse operator) and `cap` RHS
// slots.  The engine runs the same mixed-precision solve as mg_solve, but a
// slot can be filled or emptied at every restart boundary of the inner FGCR:
// a new RHS starts its own FP64 defect correction there, a RHS whose inner
// solve converged takes its FP64 update there, and a RHS that reached the
// FP64 tolerance leaves.  Every RHS follows exactly the recurrence it would
// follow alone (its own scalars, masks and restart points), so its result
// does not depend on what else is in flight.
static Vec vsub(const Vec& v, int r0, int n) {
  Vec o = v;
  o.p = (char*)v.p + (size_t)r0 * v.n * (v.prec == MGLMA_FP64 ? 8 : 4);
  o.nrhs = n;
  return o;
}
static Spinor ssub(const Spinor& v, int r0, int n) {
  Spinor o = v;
  o.p = (char*)v.p + (size_t)r0 * v.rhs_reals() * (v.prec == MGLMA_FP64 ? 8 : 4);
  o.nrhs = n;
  return o;
}

struct Engine {
  struct Slot {
    int req = -1;   // request index, -1 when free
    int rhs = 0;    // RHS of the request held here
    int inner = 0;  // FGCR iterations of the current inner solve
    RhsStat st;
    double bb = 0;
  };
  struct Done {
    int slot, req, rhs;
  };
  mglma_ctx ctx = nullptr;
  cudaStream_t s = nullptr;
  const mglma_gauge_s* G = nullptr;
  const mglma_coarse_s* C = nullptr;
  MgParams p;
  int cap = 0;
  int64_t V = 0;
  Spinor b64, x64, r64, r32, e32;
  double* dsc = nullptr;  // per slot: |r|^2 [cap], |r| [cap], 1/|r| [cap]
  double* stage = nullptr;  // one canonical spinor: host requests pass through it
  double* gpart = nullptr;  // partials of the FGCR image's dots
  GcrWork gw;
  TwoLevel K;
  std::vector<Slot> slots;
  FreeList* fl = nullptr;
  static constexpr int kInnerCap = 400;

  // device bytes one slot needs (FP64 b, x, r -- r also holds D x while the
  // residual is formed; FP32 r, e, FGCR directions and images, preconditioner
  // scratch)
  static size_t slot_bytes(int64_t V, int m) { return (size_t)V * (3 * 192 + (size_t)(6 + 2 * m) * 96); }
  // one canonical spinor that host requests pass through, allocated on the
  // first host request (device requests need none)
  static size_t fixed_bytes(int64_t) { return 0; }
  mglma_status ensure_stage() {
    if (stage) return MGLMA_OK;
    MG_CHECK(dalloc(ctx, (void**)&stage, (size_t)V * 24 * sizeof(double), s));
    fl->add(stage);
    return MGLMA_OK;
  }

  ~Engine() { delete fl; }

  mglma_status setup(mglma_ctx c, cudaStream_t st, const mglma_gauge_s* g, const mglma_coarse_s* co,
                     const MgParams& prm, int capacity) {
    ctx = c;
    s = st;
    G = g;
    C = co;
    p = prm;
    cap = capacity;
    V = g->g.V;
    fl = new FreeList(ctx, s);
    for (Spinor* f : {&b64, &x64, &r64}) {
      MG_CHECK(alloc_spinor(ctx, *f, MGLMA_FP64, cap, V, s));
      fl->add(f->p);
    }
    for (Spinor* f : {&r32, &e32}) {
      MG_CHECK(alloc_spinor(ctx, *f, MGLMA_FP32, cap, V, s));
      fl->add(f->p);
    }
    MG_CHECK(dalloc(ctx, (void**)&dsc, sizeof(double) * 3 * cap, s));
    fl->add(dsc);
    MG_CHECK(gw.setup(ctx, s, as_vec(r32), cap, p.gcr_m));
    MG_CHECK(dalloc(ctx, (void**)&gpart, dslash_gcr_part_doubles(V, cap) * sizeof(double), s));
    fl->add(gpart);
    K.ctx = ctx;
    K.s = s;
    K.G = G;
    K.C = C;
    K.p = &p;
    K.cap = cap;
    MG_CHECK(fill_int(gw.sc.active, 0, cap, s));
    slots.assign(cap, Slot());
    return MGLMA_OK;
  }

  int used_prefix() const {
    int hi = 0;
    for (int i = 0; i < cap; ++i)
      if (slots[i].req >= 0) hi = i + 1;
    return hi;
  }
  int first_free() const {
    for (int i = 0; i < cap; ++i)
      if (slots[i].req < 0) return i;
    return -1;
  }

  // start the inner FP32 solve of slot i from its FP64 residual r64[i]
  mglma_status start_inner(int i) {
    std::vector<double> h;
    MG_CHECK(norm2(ctx, as_vec(ssub(r64, i, 1)), dsc + i, s));
    MG_CHECK(read_doubles(dsc + i, h, 1, s));
    const double rn = std::sqrt(h[0]);
    const double pr[2] = {rn, rn > 0 ? 1.0 / rn : 0.0};
    MG_CUDA(cudaMemcpyAsync(dsc + cap + i, &pr[0], sizeof(double), cudaMemcpyHostToDevice, s));
    MG_CUDA(cudaMemcpyAsync(dsc + 2 * cap + i, &pr[1], sizeof(double), cudaMemcpyHostToDevice, s));
    Spinor rs = ssub(r32, i, 1);
    MG_CHECK(convert_spinor(ctx, ssub(r64, i, 1), rs, s, dsc + 2 * cap + i, false));
    Vec ri = vsub(as_vec(r32), i, 1), xi = vsub(as_vec(e32), i, 1);
    Vec gr = vsub(gw.view(gw.rp, 0, cap), i, 1);
    double* bb = gw.sc.d + (size_t)(gw.m + 1) * gw.cap;
    MG_CHECK(zero_vec(ctx, xi, s));
    MG_CHECK(copy_vec(ctx, ri, gr, s));
    // |r32| = 1: the stopping reference is the squared inner-tolerance factor
    const double sc = final_cycle_scale(p, slots[i].bb > 0 ? rn / std::sqrt(slots[i].bb) : 1.0);
    const double ref = sc * sc;
    MG_CUDA(cudaMemcpyAsync(bb + i, &ref, sizeof(double), cudaMemcpyHostToDevice, s));
    MG_CHECK(fill_int(gw.sc.active + i, 1, 1, s));
    MG_CUDA(cudaStreamSynchronize(s));
    slots[i].inner = 0;
    return MGLMA_OK;
  }

  // a new RHS in slot i from a canonical device spinor; returns true in
  // *finished when the source is zero (x = 0, nothing to iterate)
  mglma_status admit(int i, int req, int rhs, const double* canon, bool* finished) {
    Slot& sl = slots[i];
    sl.req = req;
    sl.rhs = rhs;
    sl.st = RhsStat();
    Spinor bi = ssub(b64, i, 1), ri = ssub(r64, i, 1);
    MG_CHECK(pack_spinor(ctx, canon, bi, s));
    Vec xv = as_vec(ssub(x64, i, 1));
    MG_CHECK(zero_vec(ctx, xv, s));
    Vec rv = as_vec(ri);
    MG_CHECK(copy_vec(ctx, as_vec(bi), rv, s));
    std::vector<double> h;
    MG_CHECK(norm2(ctx, as_vec(bi), dsc + i, s));
    MG_CHECK(read_doubles(dsc + i, h, 1, s));
    sl.bb = h[0];
    *finished = !(h[0] > 0);
    if (*finished) {
      sl.st.residual = 0;
      sl.st.converged = true;
      return MGLMA_OK;
    }
    return start_inner(i);
  }

  void release(int i) {
    slots[i].req = -1;
    fill_int(gw.sc.active + i, 0, 1, s);
  }

  // one restart cycle of the inner FGCR over the occupied prefix, then the
  // FP64 updates of every slot whose inner solve finished
  mglma_status cycle(std::vector<Done>& done) {
    const int hi = used_prefix();
    if (hi == 0) return MGLMA_OK;
    OpFn A = [&](const Vec& in, Vec& o) {
      Spinor a = as_spinor(in, V), bo = as_spinor(o, V);
      return dslash(ctx, G, a, bo, false, false, s);
    };
    OpFn M = [&](const Vec& in, Vec& o) { return K(in, o); };
    const AdFn Ad = [&](const Vec& in, Vec& o, int k, const Vec& W0, size_t wslot, const Vec& res, double* nw,
                        double2* num, double2* dots) {
      Spinor a = as_spinor(in, V), bo = as_spinor(o, V);
      return dslash_gcr(ctx, G, a, bo, k, W0.p, wslot, res.p, gpart, nw, num, dots, s);
    };
    gw.Ad = &Ad;
    Vec x = vsub(as_vec(e32), 0, hi);
    mglma_status st = MGLMA_OK;
    for (int k = 0; k < gw.m && st == MGLMA_OK; ++k) st = gcr_iter(gw, A, &M, x, hi, k, p.inner_tol * p.inner_tol);
    gw.Ad = nullptr;
    MG_CHECK(st);
    std::vector<int> act;
    MG_CHECK(read_active(gw, hi, act));
    for (int i = 0; i < hi; ++i) {
      Slot& sl = slots[i];
      if (sl.req < 0) continue;
      sl.inner += gw.m;
      if (act[i] && sl.inner < kInnerCap) continue;
      // FP64 update: x += |r| e ; r = b - D x
      Spinor xi = ssub(x64, i, 1), ri = ssub(r64, i, 1);
      MG_CHECK(convert_spinor(ctx, ssub(e32, i, 1), xi, s, dsc + cap + i, true));
      MG_CHECK(dslash(ctx, G, xi, ri, false, false, s));  // r = D x, then r = b - r
      Vec rv = as_vec(ri);
      MG_CHECK(axpby(ctx, nullptr, C1, as_vec(ssub(b64, i, 1)), nullptr, CM1, rv, s));
      std::vector<double> h;
      MG_CHECK(norm2(ctx, rv, dsc + i, s));
      MG_CHECK(read_doubles(dsc + i, h, 1, s));
      sl.st.outer++;
      sl.st.iterations += sl.inner;
      sl.st.residual = std::sqrt(h[0] / sl.bb);
      if (!std::isfinite(sl.st.residual)) return fail(MGLMA_ERR_NUMERIC, "serve: non-finite residual");
      sl.st.converged = sl.st.residual <= p.tol;
      if (sl.st.converged || sl.st.outer >= 50 || sl.st.iterations >= p.max_iter) {
        sl.st.coarse_iterations = K.coarse_iters;
        done.push_back({i, sl.req, sl.rhs});
      } else {
        MG_CHECK(start_inner(i));
      }
    }
    return MGLMA_OK;
  }
};

}  // namespace mglma

using namespace mglma;

extern "C" mglma_status mglma_serve(mglma_ctx ctx, const mglma_serve_config* cfg, mglma_request_fn next,
                                    mglma_done_fn done, void* user, mglma_serve_stats* out) {
  if (!ctx || !cfg || !next || !cfg->lattices || cfg->nlattices < 1 || cfg->nlattices > 8)
    return fail(MGLMA_ERR_INVALID, "serve: bad configuration");
  if (cfg->max_slots < 1 || !(cfg->hbm_fraction > 0) || cfg->hbm_fraction > 1)
    return fail(MGLMA_ERR_INVALID, "serve: max_slots >= 1 and 0 < hbm_fraction <= 1 required");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const mglma_solve_params* prm = &cfg->params;
  const MgParams mp = mg_params(*prm);
  // admission by free HBM: the slots of each lattice take a share of
  // hbm_fraction of the memory free now in proportion to its volume (a slot's
  // size is proportional to the volume)
  size_t fr = 0, tot = 0;
  MG_CUDA(cudaStreamSynchronize(s));
  MG_CUDA(cudaMemPoolTrimTo(ctx->pool, 0));  // cached set-up blocks count as free
  MG_CUDA(cudaMemGetInfo(&fr, &tot));
  const int NL = cfg->nlattices;
  double vsum = 0;
  for (int l = 0; l < NL; ++l)
    if (cfg->lattices[l].gauge) vsum += (double)cfg->lattices[l].gauge->g.V;
  std::vector<std::unique_ptr<Engine>> eng(NL);
  mglma_serve_stats st;
  memset(&st, 0, sizeof(st));
  for (int l = 0; l < NL; ++l) {
    const mglma_serve_lattice& L = cfg->lattices[l];
    if (!L.gauge || !L.coarse || L.coarse->sub->gauge != L.gauge)
      return fail(MGLMA_ERR_INVALID, "serve: lattice entries need a gauge field and its coarse operator");
    const size_t per = Engine::slot_bytes(L.gauge->g.V, mp.gcr_m);
    const double share =
        cfg->hbm_fraction * (double)fr * ((double)L.gauge->g.V / vsum) - (double)Engine::fixed_bytes(L.gauge->g.V);
    const int cap = share > 0 ? (int)std::min<size_t>((size_t)cfg->max_slots, (size_t)(share / per)) : 0;
    if (cap < 1) return fail(MGLMA_ERR_OOM, "serve: not enough free HBM for one slot of lattice " + std::to_string(l));
    eng[l].reset(new Engine());
    MG_CHECK(eng[l]->setup(ctx, s, L.gauge, L.coarse, mp, cap));
    st.slots[l] = cap;
    st.slot_bytes[l] = (double)per;
  }
  MG_CUDA(cudaStreamSynchronize(s));
  struct Req {
    mglma_request r;
    int next_rhs = 0, remaining = 0;
    bool bhost = false, xhost = false;
    std::vector<mglma_solve_stats> stats;
    mglma_status status = MGLMA_OK;
  };
  std::vector<Req> reqs;
  std::vector<std::deque<int>> queue(NL);
  std::vector<double> lat;
  auto t0 = std::chrono::steady_clock::now();
  auto now = [&] { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  bool ended = false;
  long long rhs_done = 0;
  mglma_status err = MGLMA_OK;
  auto finish_req = [&](int q) {
    Req& R = reqs[q];
    cudaStreamSynchronize(s);
    const double l = now() - R.r.arrival;
    if (R.status == MGLMA_OK) lat.push_back(l);
    if (done) done(user, &R.r, R.status, l, R.stats.data());
  };
  while (err == MGLMA_OK) {
    // pull every request that has arrived
    while (!ended) {
      mglma_request rq;
      memset(&rq, 0, sizeof(rq));
      const int got = next(user, now(), &rq);
      if (got < 0) ended = true;
      if (got != 1) break;
      Req R;
      R.r = rq;
      R.remaining = rq.nrhs;
      R.stats.assign(std::max(rq.nrhs, 1), mglma_solve_stats());
      const int l = rq.lattice;
      const bool bad = l < 0 || l >= NL || rq.nrhs < 1 || !rq.b || !rq.x;
      reqs.push_back(R);
      const int q = (int)reqs.size() - 1;
      st.requests++;
      if (bad) {
        reqs[q].status = MGLMA_ERR_INVALID;
        st.rejected++;
        if (done) done(user, &reqs[q].r, reqs[q].status, 0.0, reqs[q].stats.data());
        continue;
      }
      queue[l].push_back(q);
    }
    bool active = false;
    for (int l = 0; l < NL && err == MGLMA_OK; ++l) {
      Engine& E = *eng[l];
      // admit waiting RHS into free slots (a request may be spread over cycles)
      while (!queue[l].empty() && err == MGLMA_OK) {
        const int q = queue[l].front();
        Req& R = reqs[q];
        const size_t one = (size_t)E.V * 24;
        if (R.next_rhs == 0) {
          R.bhost = !is_device_pointer(R.r.b);
          R.xhost = !is_device_pointer(R.r.x);
          if (R.bhost || R.xhost) {
            err = E.ensure_stage();
            if (err != MGLMA_OK) break;
          }
        }
        int slot;
        while (R.next_rhs < R.r.nrhs && (slot = E.first_free()) >= 0) {
          bool fin = false;
          const int rhs = R.next_rhs++;
          const double* src = R.r.b + (size_t)rhs * one;
          if (R.bhost) {
            cudaMemcpyAsync(E.stage, src, one * sizeof(double), cudaMemcpyHostToDevice, s);
            src = E.stage;
          }
          err = E.admit(slot, q, rhs, src, &fin);
          if (err != MGLMA_OK) break;
          if (fin) {  // zero source: x = 0
            if (R.xhost)
              memset(R.r.x + (size_t)rhs * one, 0, one * sizeof(double));
            else
              cudaMemsetAsync(R.r.x + (size_t)rhs * one, 0, one * sizeof(double), s);
            R.stats[rhs].converged = 1;
            E.release(slot);
            if (--R.remaining == 0) finish_req(q);
          }
        }
        if (err != MGLMA_OK || R.next_rhs < R.r.nrhs) break;
        queue[l].pop_front();
      }
      if (err != MGLMA_OK || E.used_prefix() == 0) continue;
      active = true;
      std::vector<Engine::Done> fin;
      err = E.cycle(fin);
      for (auto& d : fin) {
        if (err != MGLMA_OK) break;
        Req& R = reqs[d.req];
        const Engine::Slot& sl = E.slots[d.slot];
        Spinor xi = ssub(E.x64, d.slot, 1);
        const size_t one = (size_t)E.V * 24;
        if (R.xhost) {
          err = unpack_spinor(ctx, xi, E.stage, s);
          if (err == MGLMA_OK && cudaMemcpyAsync(R.r.x + (size_t)d.rhs * one, E.stage, one * sizeof(double),
                                                 cudaMemcpyDeviceToHost, s) != cudaSuccess)
            err = fail(MGLMA_ERR_CUDA, "serve: copy of a solution to the host failed");
          cudaStreamSynchronize(s);
        } else {
          err = unpack_spinor(ctx, xi, R.r.x + (size_t)d.rhs * one, s);
        }
        mglma_solve_stats& o = R.stats[d.rhs];
        o.iterations = sl.st.iterations;
        o.outer = sl.st.outer;
        o.coarse_iterations = sl.st.coarse_iterations;
        o.residual = sl.st.residual;
        o.converged = sl.st.converged ? 1 : 0;
        if (!sl.st.converged) R.status = MGLMA_ERR_NOT_CONVERGED;
        E.release(d.slot);
        rhs_done++;
        if (--R.remaining == 0) finish_req(d.req);
      }
    }
    if (err != MGLMA_OK) break;
    if (!active) {
      bool waiting = false;
      for (auto& qd : queue) waiting = waiting || !qd.empty();
      if (ended && !waiting) break;
      if (!waiting) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  cudaStreamSynchronize(s);
  const double wall = now();
  if (out) {
    st.rhs = rhs_done;
    st.wall_s = wall;
    st.solves_per_s = wall > 0 ? rhs_done / wall : 0;
    if (!lat.empty()) {
      std::vector<double> v = lat;
      std::sort(v.begin(), v.end());
      auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)std::ceil(q * v.size()) - 1)]; };
      st.p50_s = pct(0.50);
      st.p99_s = pct(0.99);
      st.max_s = v.back();
      double sum = 0;
      for (double x : v) sum += x;
      st.mean_s = sum / v.size();
    }
    *out = st;
  }
  return err;
}
