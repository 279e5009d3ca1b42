// Even-odd (Schur) preconditioning of the fine Wilson-clover operator.
//
// With every lattice extent even, every hop of D joins sites of opposite
// parity p(x) = (x0 + x1 + x2 + x3) mod 2, so with the sites ordered even then
// odd
//     D = [[A_ee, H_eo], [H_oe, A_oo]]
// (A the site-local clover term, H the hops) and D x = b is solved through
// the Schur complement on the even sites
//     S x_e = b_e - H_eo A_oo^-1 b_o,   S = A_ee - H_eo A_oo^-1 H_oe,
//     x_o = A_oo^-1 (b_o - H_oe x_e),
// S^dag = A_ee - H^dag_eo A_oo^-1 H^dag_oe (A is Hermitian) and gamma5 S is
// Hermitian.  The plain method MGLMA_SOLVER_CGNE_EO runs FP64 CG on
// S^dag S x_e = S^dag b_e', reconstructs x_o and corrects against the true
// residual of the full system.
//
// Fields of one parity ("half" fields) hold the sites of that parity in the
// FP64 internal layout [rhs][12 chunks][V / 2], site x at index x >> 1 (the
// extent L3 is even, so x and x + 1 differ in parity).  The clover inverses
// are two Hermitian 6x6 blocks per site in the packed layout of the clover
// term, formed once per gauge field.
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "solver.h"
#include "stencil.cuh"

namespace mglma {

__device__ __forceinline__ int64_t eo_site(const LatIdx& q, int64_t u, int par) {
  const int64_t y0 = 2 * u;
  int xc[4];
  site_coords(q, y0, xc);
  return y0 + ((par ^ (xc[0] + xc[1] + xc[2] + xc[3])) & 1);
}

// inverse of each packed Hermitian 6x6 clover block (one thread per (site,
// chirality)): Gauss-Jordan with partial pivoting in FP64; the inverse of a
// Hermitian matrix is Hermitian and is packed the same way.  Every loop is
// unrolled and every index static (row and column exchanges are predicated
// swaps), so the 6x6 matrix stays in registers: a version that indexed a
// local array by the pivot row gave wrong inverses when built with -O3 on
// sm_103a (exact in a debug build and on the host).
__global__ void clover_inverse_kernel(const double2* __restrict__ C, double2* __restrict__ Ci, int64_t V,
                                      int* __restrict__ singular) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * V) return;
  const int chi = (int)(t / V);
  const int64_t site = t % V;
  double c[36];
  Clover<double>::load(C, V, chi, site, c);
  Cx<double> M[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i) M[i][i] = cx(c[i], 0.0);
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      const int k = 6 + 2 * offdiag_slot(i, j);
      M[i][j] = cx(c[k], c[k + 1]);
      M[j][i] = cx(c[k], -c[k + 1]);
    }
  int perm[6];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    int p = k;
    double best = M[k][k].re * M[k][k].re + M[k][k].im * M[k][k].im;
#pragma unroll
    for (int r = k + 1; r < 6; ++r) {
      const double m = M[r][k].re * M[r][k].re + M[r][k].im * M[r][k].im;
      if (m > best) {
        best = m;
        p = r;
      }
    }
    perm[k] = p;
    ok = ok && best > 0;
    if (!(best > 0)) best = 1;  // singular: finish with harmless numbers, report below
#pragma unroll
    for (int r = k + 1; r < 6; ++r)
      if (r == p)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const Cx<double> tmp = M[k][j];
          M[k][j] = M[r][j];
          M[r][j] = tmp;
        }
    const double m = M[k][k].re * M[k][k].re + M[k][k].im * M[k][k].im;
    const Cx<double> d = m > 0 ? cx(M[k][k].re / m, -M[k][k].im / m) : cx(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (j != k) M[k][j] = M[k][j] * d;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      if (r == k) continue;
      const Cx<double> f = M[r][k];
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if (j != k) M[r][j] = M[r][j] - f * M[k][j];
      M[r][k] = -(f * d);
    }
    M[k][k] = d;
  }
  // undo the row exchanges as column exchanges, last first
#pragma unroll
  for (int k = 5; k >= 0; --k)
#pragma unroll
    for (int c2 = k + 1; c2 < 6; ++c2)
      if (perm[k] == c2)
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          const Cx<double> tmp = M[r][k];
          M[r][k] = M[r][c2];
          M[r][c2] = tmp;
        }
  if (!ok) {
    atomicExch(singular, 1);
    return;
  }
  double pk[36];
#pragma unroll
  for (int i = 0; i < 6; ++i) pk[i] = M[i][i].re;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      const int k = 6 + 2 * offdiag_slot(i, j);
      pk[k] = M[i][j].re;
      pk[k + 1] = M[i][j].im;
    }
#pragma unroll
  for (int j = 0; j < 18; ++j) Ci[((size_t)chi * 18 + j) * V + site] = make_double2(pk[2 * j], pk[2 * j + 1]);
}

struct EoArgs {
  LatIdx q;
  double bc;
  int nrhs;
  int par;  // parity of the output sites
};

// out (parity par) = the hops of D (DAG: of D^dag) from in (the other parity),
// -1/2 and the time-boundary sign included; one thread per (output site, RHS)
template <bool DAG>
__global__ void __launch_bounds__(128) eo_hop_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                                     const double2* __restrict__ U, EoArgs a) {
  const int64_t Vh = a.q.V / 2;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (u >= Vh || r >= a.nrhs) return;
  const int64_t site = eo_site(a.q, u, a.par);
  int x[4];
  site_coords(a.q, site, x);
  const double sF = DAG ? 1.0 : -1.0;
  Cx<double> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cx(0.0, 0.0);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    M3<double> Um;
    Cx<double> psi[12];
    {
      const int64_t nf = nbr_fwd(a.q, site, x, mu);
      const double f = -0.5 * ((mu == 0 && x[0] == a.q.L[0] - 1) ? a.bc : 1.0);
      Link<double>::load(U, a.q.V, mu, site, Um);
      IO<double>::load(in, Vh, r, nf >> 1, psi);
      hop_add<double, true>(mu, sF, f, Um, psi, acc);
    }
    {
      const int64_t nb = nbr_bwd(a.q, site, x, mu);
      const double f = -0.5 * ((mu == 0 && x[0] == 0) ? a.bc : 1.0);
      Link<double>::load(U, a.q.V, mu, nb, Um);
      IO<double>::load(in, Vh, r, nb >> 1, psi);
      hop_add<double, false>(mu, -sF, f, Um, psi, acc);
    }
  }
  IO<double>::store(out, Vh, r, u, acc);
}

// out (parity par) = A(x) in (+ sgn * add when add != NULL), A the clover term
// or its inverse in the packed layout; g5 multiplies the result by gamma5
__global__ void __launch_bounds__(128) eo_clover_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                                        const double2* __restrict__ Cb, const double2* __restrict__ add,
                                                        double sgn, int g5, EoArgs a) {
  const int64_t Vh = a.q.V / 2;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (u >= Vh || r >= a.nrhs) return;
  const int64_t site = eo_site(a.q, u, a.par);
  Cx<double> psi[12], acc[12];
  IO<double>::load(in, Vh, r, u, psi);
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    double c[36];
    Clover<double>::load(Cb, a.q.V, chi, site, c);
    clover_apply6<double>(c, psi + 6 * chi, acc + 6 * chi);
  }
  if (add) {
    Cx<double> w[12];
    IO<double>::load(add, Vh, r, u, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = acc[k] + sgn * w[k];
  }
  if (g5) {
#pragma unroll
    for (int k = 6; k < 12; ++k) acc[k] = -acc[k];
  }
  IO<double>::store(out, Vh, r, u, acc);
}

// half field of parity par <-> full internal FP64 field (the other parity of
// a full output is left as it is)
template <bool TO_HALF>
__global__ void eo_copy_kernel(const double2* __restrict__ src, double2* __restrict__ dst, LatIdx q, int nrhs,
                               int par) {
  const int64_t Vh = q.V / 2;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (u >= Vh || r >= nrhs) return;
  const int64_t site = eo_site(q, u, par);
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    if (TO_HALF)
      dst[((size_t)r * 12 + j) * Vh + u] = src[((size_t)r * 12 + j) * q.V + site];
    else
      dst[((size_t)r * 12 + j) * q.V + site] = src[((size_t)r * 12 + j) * Vh + u];
  }
}

static dim3 eo_grid(int64_t V, int nrhs) { return dim3((unsigned)((V / 2 + 127) / 128), (unsigned)nrhs, 1); }

mglma_status eo_check(const mglma_gauge_s* G) {
  for (int m = 0; m < 4; ++m)
    if (G->g.L[m] % 2) return fail(MGLMA_ERR_INVALID, "even-odd: every lattice extent must be even");
  return MGLMA_OK;
}

mglma_status clover_inverse_ready(mglma_ctx ctx, mglma_gauge_s* G, cudaStream_t s) {
  if (G->Cinv64) return MGLMA_OK;
  MG_CHECK(eo_check(G));
  const int64_t V = G->g.V;
  MG_CUDA(cudaMalloc(&G->Cinv64, (size_t)V * 36 * sizeof(double2)));
  int* sing = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&sing, sizeof(int), s));
  MG_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
  {
    ProfScope ps(ctx, K_SETUP, s);
    clover_inverse_kernel<<<(unsigned)((2 * V + 127) / 128), 128, 0, s>>>(G->C64, G->Cinv64, V, sing);
  }
  MG_LAUNCH_CHECK();
  int h = 0;
  MG_CUDA(cudaMemcpyAsync(&h, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
  dfree(ctx, sing, s);
  MG_CUDA(cudaStreamSynchronize(s));
  if (h) return fail(MGLMA_ERR_NUMERIC, "even-odd: a clover block is singular");
  return MGLMA_OK;
}

// half-field work space of the Schur operator (two fields of nrhs RHS)
struct EoWork {
  mglma_ctx ctx = nullptr;
  cudaStream_t s = nullptr;
  Spinor t, w;
  ~EoWork() {
    if (ctx) {
      dfree(ctx, t.p, s);
      dfree(ctx, w.p, s);
    }
  }
  mglma_status setup(mglma_ctx c, cudaStream_t st, int nrhs, int64_t V) {
    ctx = c;
    s = st;
    MG_CHECK(alloc_spinor(ctx, t, MGLMA_FP64, nrhs, V / 2, s));
    MG_CHECK(alloc_spinor(ctx, w, MGLMA_FP64, nrhs, V / 2, s));
    return MGLMA_OK;
  }
};

static EoArgs eo_args(const mglma_gauge_s* G, int nrhs, int par) {
  EoArgs a;
  a.q = make_latidx(G->g.L);
  a.bc = (double)G->g.t_bc;
  a.nrhs = nrhs;
  a.par = par;
  return a;
}

// y_e = S x_e (dag: S^dag x_e; g5: gamma5 times the result), half fields of the
// even sites; the hops move through W.t and W.w
mglma_status schur64(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& x, Spinor& y, bool dag, bool g5,
                     EoWork& W, cudaStream_t s) {
  const int n = x.nrhs;
  const int64_t V = G->g.V;
  const dim3 g = eo_grid(V, n);
  // algorithmic traffic of one application: links (4 x 144 B) once per
  // hop pass, clover blocks (576 B) per clover pass, spinors read and written
  // once per pass -- about the bytes of one full application of D
  ProfScope ps(ctx, K_DSLASH64, s, (double)V * (1152.0 + 384.0 * n) * 1.0, 1896.0 * (double)V * n);
  const EoArgs ao = eo_args(G, n, 1), ae = eo_args(G, n, 0);
  // t_o = H_oe x_e ; w_o = A_oo^-1 t_o ; t_e = H_eo w_o ; y_e = A_ee x_e - t_e
  if (dag)
    eo_hop_kernel<true><<<g, 128, 0, s>>>((const double2*)x.p, (double2*)W.t.p, G->U64, ao);
  else
    eo_hop_kernel<false><<<g, 128, 0, s>>>((const double2*)x.p, (double2*)W.t.p, G->U64, ao);
  eo_clover_kernel<<<g, 128, 0, s>>>((const double2*)W.t.p, (double2*)W.w.p, G->Cinv64, nullptr, 0.0, 0, ao);
  if (dag)
    eo_hop_kernel<true><<<g, 128, 0, s>>>((const double2*)W.w.p, (double2*)W.t.p, G->U64, ae);
  else
    eo_hop_kernel<false><<<g, 128, 0, s>>>((const double2*)W.w.p, (double2*)W.t.p, G->U64, ae);
  eo_clover_kernel<<<g, 128, 0, s>>>((const double2*)x.p, (double2*)y.p, G->C64, (const double2*)W.t.p, -1.0,
                                     g5 ? 1 : 0, ae);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// b_e' = b_e - H_eo A_oo^-1 b_o from a full FP64 field b
static mglma_status eo_prepare64(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& b, Spinor& be, EoWork& W,
                                 cudaStream_t s) {
  const int n = b.nrhs;
  const LatIdx q = make_latidx(G->g.L);
  const dim3 g = eo_grid(G->g.V, n);
  ProfScope ps(ctx, K_PACK, s);
  eo_copy_kernel<true><<<g, 128, 0, s>>>((const double2*)b.p, (double2*)W.t.p, q, n, 1);
  eo_clover_kernel<<<g, 128, 0, s>>>((const double2*)W.t.p, (double2*)W.w.p, G->Cinv64, nullptr, 0.0, 0,
                                     eo_args(G, n, 1));
  eo_hop_kernel<false><<<g, 128, 0, s>>>((const double2*)W.w.p, (double2*)W.t.p, G->U64, eo_args(G, n, 0));
  eo_copy_kernel<true><<<g, 128, 0, s>>>((const double2*)b.p, (double2*)be.p, q, n, 0);
  MG_LAUNCH_CHECK();
  Vec vt = as_vec(W.t), vb = as_vec(be);
  return axpby(ctx, nullptr, CM1, vt, nullptr, C1, vb, s);
}

// x (full FP64) from x_e and b: x_o = A_oo^-1 (b_o - H_oe x_e)
static mglma_status eo_reconstruct64(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& b, const Spinor& xe,
                                     Spinor& x, EoWork& W, cudaStream_t s) {
  const int n = b.nrhs;
  const LatIdx q = make_latidx(G->g.L);
  const dim3 g = eo_grid(G->g.V, n);
  ProfScope ps(ctx, K_PACK, s);
  eo_hop_kernel<false><<<g, 128, 0, s>>>((const double2*)xe.p, (double2*)W.t.p, G->U64, eo_args(G, n, 1));
  eo_copy_kernel<true><<<g, 128, 0, s>>>((const double2*)b.p, (double2*)W.w.p, q, n, 1);
  MG_LAUNCH_CHECK();
  Vec vt = as_vec(W.t), vw = as_vec(W.w);
  MG_CHECK(axpby(ctx, nullptr, CM1, vt, nullptr, C1, vw, s));  // w = b_o - H_oe x_e
  eo_clover_kernel<<<g, 128, 0, s>>>((const double2*)W.w.p, (double2*)W.t.p, G->Cinv64, nullptr, 0.0, 0,
                                     eo_args(G, n, 1));
  eo_copy_kernel<false><<<g, 128, 0, s>>>((const double2*)W.t.p, (double2*)x.p, q, n, 1);
  eo_copy_kernel<false><<<g, 128, 0, s>>>((const double2*)xe.p, (double2*)x.p, q, n, 0);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// CG on S^dag S x_e = S^dag b_e' per RHS (its own scalars and mask), to
// ||b_e' - S x_e|| <= tol ||b_e'|| on the recursive residual; x_e starts at 0
static mglma_status cgne_schur64(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& be, Spinor& xe, double tol,
                                 int max_iter, int check_every, std::vector<int>& iters, EoWork& W, cudaStream_t s) {
  const int n = be.nrhs;
  const int64_t Vh = be.V;
  FreeList fl(ctx, s);
  Spinor r, z, p, w;
  for (Spinor* f : {&r, &z, &p, &w}) {
    MG_CHECK(alloc_spinor(ctx, *f, MGLMA_FP64, n, Vh, s));
    fl.add(f->p);
  }
  Scalars sc;
  MG_CHECK(sc.alloc(ctx, n, 5, 2, s));
  double *zz = sc.d, *zzn = sc.d + n, *ww = sc.d + 2 * n, *rr = sc.d + 3 * n, *bb = sc.d + 4 * n;
  double2 *alpha = sc.z, *beta = sc.z + n;
  Vec vb = as_vec(be), vx = as_vec(xe), vr = as_vec(r), vz = as_vec(z), vp = as_vec(p), vw = as_vec(w);
  MG_CHECK(zero_vec(ctx, vx, s));
  MG_CHECK(copy_vec(ctx, vb, vr, s));
  MG_CHECK(norm2(ctx, vb, bb, s));
  std::vector<double> hbb, hrr;
  MG_CHECK(read_doubles(bb, hbb, n, s));
  for (int i = 0; i < n; ++i)
    if (!(hbb[i] > 0)) sc.h_active[i] = 0;
  MG_CHECK(sc.push_active());
  MG_CHECK(schur64(ctx, G, r, z, true, false, W, s));  // z = S^dag r
  MG_CHECK(copy_vec(ctx, vz, vp, s));
  MG_CHECK(norm2(ctx, vz, zz, s));
  iters.assign(n, 0);
  for (int it = 1; it <= max_iter; ++it) {
    MG_CHECK(schur64(ctx, G, p, w, false, false, W, s));
    MG_CHECK(norm2(ctx, vw, ww, s));
    MG_CHECK(cg_scalars(ctx, zz, ww, alpha, sc.active, n, s));
    MG_CHECK(axpy2(ctx, alpha, vp, vx, vw, vr, s));
    MG_CHECK(schur64(ctx, G, r, z, true, false, W, s));
    MG_CHECK(norm2(ctx, vz, zzn, s));
    MG_CHECK(cg_beta(ctx, zzn, zz, beta, sc.active, n, s));
    MG_CHECK(axpby(ctx, nullptr, C1, vz, beta, C0, vp, s));
    for (int i = 0; i < n; ++i)
      if (sc.h_active[i]) iters[i]++;
    if (it % check_every != 0 && it < max_iter) continue;
    MG_CHECK(norm2(ctx, vr, rr, s));
    MG_CHECK(read_doubles(rr, hrr, n, s));
    bool any = false, changed = false;
    for (int i = 0; i < n; ++i) {
      if (!sc.h_active[i]) continue;
      const double rel = std::sqrt(hrr[i] / hbb[i]);
      if (!std::isfinite(rel)) return fail(MGLMA_ERR_NUMERIC, "cgne_eo: non-finite residual");
      if (rel <= tol) {
        sc.h_active[i] = 0;
        changed = true;
      } else {
        any = true;
      }
    }
    if (changed) MG_CHECK(sc.push_active());
    if (!any) break;
  }
  return MGLMA_OK;
}

// x (FP64 full, zero on entry) = D^-1 b: Schur CGNE + reconstruction, then FP64
// defect correction on the true residual of D until tol
mglma_status cgne_eo64(mglma_ctx ctx, mglma_gauge_s* G, const Spinor& b, Spinor& x, const SolveControl& ctl,
                       std::vector<RhsStat>& out, cudaStream_t s) {
  const int n = b.nrhs;
  const int64_t V = b.V;
  out.assign(n, RhsStat());
  MG_CHECK(clover_inverse_ready(ctx, G, s));
  FreeList fl(ctx, s);
  EoWork W;
  MG_CHECK(W.setup(ctx, s, n, V));
  Spinor r, e, be, xe;
  MG_CHECK(alloc_spinor(ctx, r, MGLMA_FP64, n, V, s));
  fl.add(r.p);
  MG_CHECK(alloc_spinor(ctx, e, MGLMA_FP64, n, V, s));
  fl.add(e.p);
  MG_CHECK(alloc_spinor(ctx, be, MGLMA_FP64, n, V / 2, s));
  fl.add(be.p);
  MG_CHECK(alloc_spinor(ctx, xe, MGLMA_FP64, n, V / 2, s));
  fl.add(xe.p);
  Scalars sc;
  MG_CHECK(sc.alloc(ctx, n, 2, 1, s));
  Vec vb = as_vec(b), vx = as_vec(x), vr = as_vec(r), ve = as_vec(e);
  MG_CHECK(norm2(ctx, vb, sc.d, s));
  std::vector<double> hbb, hrr;
  MG_CHECK(read_doubles(sc.d, hbb, n, s));
  MG_CHECK(zero_vec(ctx, vx, s));
  MG_CHECK(copy_vec(ctx, vb, vr, s));
  int total = 0;
  for (int cycle = 0;; ++cycle) {
    // the Schur system to a tenth of what is left of the target
    std::vector<int> it;
    MG_CHECK(eo_prepare64(ctx, G, r, be, W, s));
    MG_CHECK(cgne_schur64(ctx, G, be, xe, 0.1 * ctl.tol, ctl.max_iter - total, ctl.check_every, it, W, s));
    MG_CHECK(eo_reconstruct64(ctx, G, r, xe, e, W, s));
    int most = 0;
    for (int i = 0; i < n; ++i) {
      out[i].iterations += it[i];
      most = std::max(most, it[i]);
    }
    total += most;
    MG_CHECK(axpby(ctx, nullptr, C1, ve, nullptr, C1, vx, s));  // x += e
    MG_CHECK(dslash(ctx, G, x, r, false, false, s));           // r = b - D x
    MG_CHECK(axpby(ctx, nullptr, C1, vb, nullptr, CM1, vr, s));
    MG_CHECK(norm2(ctx, vr, sc.d + n, s));
    MG_CHECK(read_doubles(sc.d + n, hrr, n, s));
    bool all = true;
    for (int i = 0; i < n; ++i) {
      out[i].residual = hbb[i] > 0 ? std::sqrt(hrr[i] / hbb[i]) : 0.0;
      if (!std::isfinite(out[i].residual)) return fail(MGLMA_ERR_NUMERIC, "cgne_eo: non-finite residual");
      out[i].converged = out[i].residual <= ctl.tol;
      out[i].outer = cycle + 1;
      all = all && out[i].converged;
    }
    if (all) return MGLMA_OK;
    if (total >= ctl.max_iter || cycle >= 10) return fail(MGLMA_ERR_NOT_CONVERGED, "cgne_eo: iteration cap reached");
  }
}

// out = S in (op 4) or gamma5 S in (op 5) on the even sites of full canonical
// fields, zero on the odd sites (FP64)
mglma_status dirac_schur64(mglma_ctx ctx, mglma_gauge_s* G, int nrhs, const double* in_dev, double* out_dev, bool g5,
                           cudaStream_t s) {
  MG_CHECK(clover_inverse_ready(ctx, G, s));
  const int64_t V = G->g.V;
  FreeList fl(ctx, s);
  Spinor a, xe, ye;
  MG_CHECK(alloc_spinor(ctx, a, MGLMA_FP64, nrhs, V, s));
  fl.add(a.p);
  MG_CHECK(alloc_spinor(ctx, xe, MGLMA_FP64, nrhs, V / 2, s));
  fl.add(xe.p);
  MG_CHECK(alloc_spinor(ctx, ye, MGLMA_FP64, nrhs, V / 2, s));
  fl.add(ye.p);
  EoWork W;
  MG_CHECK(W.setup(ctx, s, nrhs, V));
  const LatIdx q = make_latidx(G->g.L);
  const dim3 g = eo_grid(V, nrhs);
  MG_CHECK(pack_spinor(ctx, in_dev, a, s));
  eo_copy_kernel<true><<<g, 128, 0, s>>>((const double2*)a.p, (double2*)xe.p, q, nrhs, 0);
  MG_LAUNCH_CHECK();
  MG_CHECK(schur64(ctx, G, xe, ye, false, g5, W, s));
  Vec va = as_vec(a);
  MG_CHECK(zero_vec(ctx, va, s));
  eo_copy_kernel<false><<<g, 128, 0, s>>>((const double2*)ye.p, (double2*)a.p, q, nrhs, 0);
  MG_LAUNCH_CHECK();
  return unpack_spinor(ctx, a, out_dev, s);
}

}  // namespace mglma
