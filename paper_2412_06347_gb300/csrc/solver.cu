// Krylov solvers for D x = b on batches of right-hand sides.
//
// Every RHS of a batch runs its own recurrence (no block-Krylov coupling): the
// kernels process all RHS of the batch in one launch, the per-RHS scalars
// stay on the device, and the host reads one vector of residual norms every
// `check_every` iterations to retire converged RHS.  So a RHS gives the same
// iterates alone or inside any batch.
//
// Plain method: CG on the normal equations D^dag D x = D^dag b in FP64 (the
// propagator S = D^-1 of Sec. 2 applied to b); converged RHS are frozen by a
// zero step length; when all recursive residuals pass the target the true
// FP64 residual b - D x is formed and any RHS above it restarts from there.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "internal.h"
#include "solver.h"
#include "subspace.h"

namespace mglma {

__global__ void cg_alpha_kernel(const double* zz, const double* ww, double2* alpha, const int* active, int n) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double a = (active[r] && ww[r] > 0) ? zz[r] / ww[r] : 0.0;
  alpha[r] = make_double2(a, 0.0);
}

__global__ void cg_beta_kernel(const double* zz_new, double* zz, double2* beta, const int* active, int n) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double b = (active[r] && zz[r] > 0) ? zz_new[r] / zz[r] : 0.0;
  beta[r] = make_double2(b, 0.0);
  zz[r] = zz_new[r];
}

__global__ void mr_alpha_kernel(const double2* num, const double* den, double2* a, int n) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double d = den[r];
  const double2 v = num[r];
  a[r] = d > 0 ? make_double2(v.x / d, v.y / d) : make_double2(0, 0);
}

mglma_status mr_alpha(mglma_ctx ctx, const double2* num, const double* den, double2* a, int n, cudaStream_t s) {
  ProfScope ps(ctx, K_SCALAR, s);
  mr_alpha_kernel<<<(n + 63) / 64, 64, 0, s>>>(num, den, a, n);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status cg_scalars(mglma_ctx ctx, const double* zz, const double* ww, double2* alpha, const int* active, int n,
                        cudaStream_t s) {
  ProfScope ps(ctx, K_SCALAR, s);
  cg_alpha_kernel<<<(n + 63) / 64, 64, 0, s>>>(zz, ww, alpha, active, n);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}
mglma_status cg_beta(mglma_ctx ctx, const double* zz_new, double* zz, double2* beta, const int* active, int n,
                     cudaStream_t s) {
  ProfScope ps(ctx, K_SCALAR, s);
  cg_beta_kernel<<<(n + 63) / 64, 64, 0, s>>>(zz_new, zz, beta, active, n);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// --------------------------------------------------------------- device scratch for scalars
__global__ void fill_int_kernel(int* p, int v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

mglma_status fill_int(int* p, int v, int n, cudaStream_t s) {
  fill_int_kernel<<<(n + 63) / 64, 64, 0, s>>>(p, v, n);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status Scalars::alloc(mglma_ctx c, int n, int count_d, int count_z, cudaStream_t st) {
  ctx = c;
  s = st;
  nrhs = n;
  MG_CHECK(dalloc(ctx, (void**)&d, sizeof(double) * (size_t)n * count_d, s));
  MG_CHECK(dalloc(ctx, (void**)&z, sizeof(double2) * (size_t)n * count_z, s));
  MG_CHECK(dalloc(ctx, (void**)&active, sizeof(int) * (size_t)n, s));
  h_active.assign(n, 1);
  fill_int_kernel<<<(n + 63) / 64, 64, 0, s>>>(active, 1, n);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}
Scalars::~Scalars() {
  if (ctx) {
    dfree(ctx, d, s);
    dfree(ctx, z, s);
    dfree(ctx, active, s);
  }
}
mglma_status Scalars::push_active() {
  MG_CUDA(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
  MG_CUDA(cudaStreamSynchronize(s));  // h_active may change right after
  return MGLMA_OK;
}

mglma_status read_doubles(const double* dev, std::vector<double>& host, int n, cudaStream_t s) {
  host.resize(n);
  MG_CUDA(cudaMemcpyAsync(host.data(), dev, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

mglma_status alloc_spinor(mglma_ctx ctx, Spinor& f, int prec, int nrhs, int64_t V, cudaStream_t s) {
  f.prec = prec;
  f.nrhs = nrhs;
  f.V = V;
  return dalloc(ctx, &f.p, f.bytes(), s);
}

// ============================================================ FP64 CGNE
mglma_status cgne64(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& b, Spinor& x, const SolveControl& ctl,
                    std::vector<RhsStat>& out, cudaStream_t s) {
  const int n = b.nrhs;
  const int64_t V = b.V;
  out.assign(n, RhsStat());
  FreeList fr(ctx, s);
  Spinor r, z, p, w;
  for (Spinor* f : {&r, &z, &p, &w}) {
    MG_CHECK(alloc_spinor(ctx, *f, MGLMA_FP64, n, V, s));
    fr.add(f->p);
  }
  Scalars sc;
  MG_CHECK(sc.alloc(ctx, n, 5, 2, s));
  double* zz = sc.d;
  double* zzn = sc.d + n;
  double* ww = sc.d + 2 * n;
  double* rr = sc.d + 3 * n;
  double* bb = sc.d + 4 * n;
  double2* alpha = sc.z;
  double2* beta = sc.z + n;
  Vec vb = as_vec(b), vx = as_vec(x), vr = as_vec(r), vz = as_vec(z), vp = as_vec(p), vw = as_vec(w);

  MG_CHECK(norm2(ctx, vb, bb, s));
  std::vector<double> hbb, hrr;
  MG_CHECK(read_doubles(bb, hbb, n, s));
  for (int i = 0; i < n; ++i)
    if (!(hbb[i] > 0)) {  // zero source: x stays as given (zero)
      sc.h_active[i] = 0;
      out[i].residual = 0;
      out[i].converged = true;
    }
  MG_CHECK(sc.push_active());

  // r = b - D x
  auto true_residual = [&]() -> mglma_status {
    MG_CHECK(dslash(ctx, G, x, w, false, false, s));
    MG_CHECK(copy_vec(ctx, vb, vr, s));
    MG_CHECK(axpby(ctx, nullptr, CM1, vw, nullptr, C1, vr, s));
    return MGLMA_OK;
  };
  // z = D^dag r ; p = z ; zz = |z|^2
  auto start = [&]() -> mglma_status {
    MG_CHECK(dslash(ctx, G, r, z, true, false, s));
    MG_CHECK(copy_vec(ctx, vz, vp, s));
    MG_CHECK(norm2(ctx, vz, zz, s));
    return MGLMA_OK;
  };
  MG_CHECK(true_residual());
  MG_CHECK(start());
  int iter = 0, restarts = 0;
  while (true) {
    MG_CHECK(dslash(ctx, G, p, w, false, false, s));
    MG_CHECK(norm2(ctx, vw, ww, s));
    MG_CHECK(cg_scalars(ctx, zz, ww, alpha, sc.active, n, s));
    MG_CHECK(axpy2(ctx, alpha, vp, vx, vw, vr, s));
    MG_CHECK(dslash(ctx, G, r, z, true, false, s));
    MG_CHECK(norm2(ctx, vz, zzn, s));
    MG_CHECK(cg_beta(ctx, zzn, zz, beta, sc.active, n, s));
    MG_CHECK(axpby(ctx, nullptr, C1, vz, beta, C0, vp, s));  // p = z + beta p
    MG_LAUNCH_CHECK();
    ++iter;
    for (int i = 0; i < n; ++i)
      if (sc.h_active[i]) out[i].iterations++;
    if (iter % ctl.check_every != 0 && iter < ctl.max_iter) continue;
    MG_CHECK(norm2(ctx, vr, rr, s));
    MG_CHECK(read_doubles(rr, hrr, n, s));
    bool any = false, changed = false;
    for (int i = 0; i < n; ++i) {
      if (!sc.h_active[i]) continue;
      const double rel = std::sqrt(hrr[i] / hbb[i]);
      if (!std::isfinite(rel)) return fail(MGLMA_ERR_NUMERIC, "cgne: non-finite residual");
      if (rel <= ctl.tol) {
        sc.h_active[i] = 0;
        changed = true;
      } else {
        any = true;
      }
    }
    if (changed) MG_CHECK(sc.push_active());
    if (any && iter < ctl.max_iter) continue;
    // every RHS passed on its recursive residual (or the cap hit): check the true one
    MG_CHECK(true_residual());
    MG_CHECK(norm2(ctx, vr, rr, s));
    MG_CHECK(read_doubles(rr, hrr, n, s));
    bool redo = false;
    for (int i = 0; i < n; ++i) {
      if (!(hbb[i] > 0)) continue;
      out[i].residual = std::sqrt(hrr[i] / hbb[i]);
      out[i].converged = out[i].residual <= ctl.tol;
      if (!out[i].converged) {
        sc.h_active[i] = 1;
        redo = true;
      }
    }
    if (!redo) return MGLMA_OK;
    if (iter >= ctl.max_iter || ++restarts > 20) return fail(MGLMA_ERR_NOT_CONVERGED, "cgne: iteration cap reached");
    MG_CHECK(sc.push_active());
    MG_CHECK(start());
  }
}

}  // namespace mglma

using namespace mglma;

MgParams mglma::mg_params(const mglma_solve_params& p) {
  MgParams mp;
  mp.tol = p.tol;
  mp.max_iter = p.max_iter;
  mp.gcr_m = p.gcr_m;
  mp.nu = p.nu;
  mp.inner_tol = p.inner_tol;
  mp.coarse_tol = p.coarse_tol;
  mp.coarse_max_iter = p.coarse_max_iter;
  mp.coarse_solver = p.coarse_solver;
  mp.graph = p.graph;
  return mp;
}

extern "C" {

void mglma_solve_params_default(mglma_solve_params* p, int method) {
  if (!p) return;
  p->method = method;
  p->tol = 1e-10;
  p->max_iter = method == MGLMA_SOLVER_MG ? 4000 : 100000;
  p->gcr_m = 4;
  p->nu = 7;
  p->inner_tol = 3e-6;
  p->coarse_tol = 0.02;
  // four cycles of 12 MINRES iterations: on 64x32^3 with 16 RHS a tighter
  // cap costs FGCR iterations and a looser one coarse iterations (measured
  // on GB300: 48 -> 1.74 s per 16-RHS solve, 60 -> 1.76 s, 108 -> 1.80 s)
  p->coarse_max_iter = 48;
  p->check_every = method == MGLMA_SOLVER_MG ? 1 : 20;
  p->max_batch = 0;
  p->coarse_solver = MGLMA_COARSE_MINRES_EO;
  p->autotune = method == MGLMA_SOLVER_MG ? 1 : 0;
  p->graph = method == MGLMA_SOLVER_MG ? 1 : 0;
}

mglma_status mglma_solve_batch(mglma_ctx ctx, mglma_gauge G, mglma_coarse C, const mglma_solve_params* prm,
                               int ngroups, const int* group_nrhs, const double* b, double* x, double* x_coarse,
                               mglma_solve_stats* stats, void* cuda_stream) {
  if (!ctx || !G || !prm || !group_nrhs || !b || !x) return fail(MGLMA_ERR_INVALID, "solve_batch: NULL argument");
  if (!G->ready) return fail(MGLMA_ERR_INVALID, "solve_batch: gauge field incomplete");
  MG_CHECK(check_gauge_device(ctx, G, "solve_batch"));
  if (prm->method != MGLMA_SOLVER_CGNE && prm->method != MGLMA_SOLVER_MG && prm->method != MGLMA_SOLVER_CGNE_EO)
    return fail(MGLMA_ERR_INVALID, "solve_batch: unknown method");
  if (prm->method == MGLMA_SOLVER_CGNE_EO)
    for (int m = 0; m < 4; ++m)
      if (G->g.L[m] % 2) return fail(MGLMA_ERR_INVALID, "solve_batch: even-odd needs every lattice extent even");
  if ((prm->method == MGLMA_SOLVER_MG || x_coarse) && !C)
    return fail(MGLMA_ERR_INVALID, "solve_batch: the MG method and the pieces need a coarse operator");
  if (C && C->sub->gauge != G) return fail(MGLMA_ERR_INVALID, "solve_batch: coarse operator of another gauge field");
  if (x_coarse && !C->sub->phi64) return fail(MGLMA_ERR_INVALID, "solve_batch: pieces need the FP64 basis");
  if (x_coarse && !C->A64) return fail(MGLMA_ERR_INVALID, "solve_batch: pieces need the FP64 coarse operator");
  if (!(prm->tol > 0) || prm->max_iter < 1 || prm->check_every < 1 ||
      (prm->method == MGLMA_SOLVER_MG && (prm->gcr_m < 1 || prm->gcr_m > 64 || prm->nu < 0 ||
                                          !(prm->inner_tol > 0) || !(prm->coarse_tol > 0) ||
                                          prm->coarse_max_iter < 1 ||
                                          (prm->coarse_solver != MGLMA_COARSE_GCR &&
                                           prm->coarse_solver != MGLMA_COARSE_MINRES &&
                                           prm->coarse_solver != MGLMA_COARSE_MINRES_EO))))
    return fail(MGLMA_ERR_INVALID, "solve_batch: bad parameters");
  int total = 0;
  for (int g = 0; g < ngroups; ++g) {
    if (group_nrhs[g] < 0) return fail(MGLMA_ERR_INVALID, "solve_batch: negative group size");
    total += group_nrhs[g];
  }
  if (total == 0) return MGLMA_OK;
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, cuda_stream);
  const int64_t V = G->g.V;
  const size_t per = (size_t)V * 24 * sizeof(double);
  Staged sb, sx, sxc;
  MG_CHECK(stage_in(ctx, b, per * total, s, sb));
  MG_CHECK(stage_out_alloc(ctx, x, per * total, s, sx));
  if (x_coarse) MG_CHECK(stage_out_alloc(ctx, x_coarse, per * total, s, sxc));
  // Ragged groups are merged into lockstep batches sized by the memory the
  // context can still use: free HBM plus the blocks its own pool holds cached
  // (a batch must not shrink because the library's cache grew).
  int cap = prm->max_batch > 0 ? prm->max_batch : 64;
  if (prm->max_batch <= 0) {
    size_t room = device_room(ctx, s);
    // the multigrid solve's double-float links and clover (2 x 36 float4 per
    // site), made on its first use, come out of the same room
    if (prm->method == MGLMA_SOLVER_MG && !(G->Udf && G->Cdf)) room -= std::min(room, (size_t)V * 1152);
    const size_t per_site = prm->method != MGLMA_SOLVER_MG ? 6 * 192 : 4 * 192 + (size_t)(7 + 2 * prm->gcr_m) * 96;
    const size_t per_rhs = per_site * (size_t)V;
    cap = (int)std::max<size_t>(1, std::min<size_t>(64, (size_t)(0.7 * (double)room) / per_rhs));
  }
  // equal lockstep batches: ceil(total / cap) batches of nearly equal size
  const int nbatch = (total + cap - 1) / cap;
  cap = (total + nbatch - 1) / nbatch;
  bool all_conv = true;
  for (int off = 0; off < total;) {
    const int n = std::min(cap, total - off);
    FreeList fl(ctx, s);
    Spinor B, X;
    MG_CHECK(alloc_spinor(ctx, B, MGLMA_FP64, n, V, s));
    fl.add(B.p);
    MG_CHECK(alloc_spinor(ctx, X, MGLMA_FP64, n, V, s));
    fl.add(X.p);
    MG_CHECK(pack_spinor(ctx, sb.dev + (size_t)off * V * 24, B, s));
    MG_CUDA(cudaMemsetAsync(X.p, 0, X.bytes(), s));
    if (prm->method == MGLMA_SOLVER_MG && prm->autotune) MG_CHECK(autotune_for_batch(ctx, G, C, n));
    std::vector<RhsStat> rs;
    mglma_status st;
    if (prm->method != MGLMA_SOLVER_MG) {
      SolveControl ctl;
      ctl.tol = prm->tol;
      ctl.max_iter = prm->max_iter;
      ctl.check_every = prm->check_every;
      st = prm->method == MGLMA_SOLVER_CGNE ? cgne64(ctx, G, B, X, ctl, rs, s) : cgne_eo64(ctx, G, B, X, ctl, rs, s);
    } else {
      const MgParams mp = mg_params(*prm);
      st = mg_solve(ctx, G, C, B, X, mp, rs, s);
    }
    if (st != MGLMA_OK && st != MGLMA_ERR_NOT_CONVERGED) return st;
    MG_CHECK(unpack_spinor(ctx, X, sx.dev + (size_t)off * V * 24, s));
    if (x_coarse) {
      // psi1 = T0 D1^-1 R0 b (FP64 transfers, coarse solve to tol)
      const size_t nc = (size_t)n * C->geo.V1 * C->n2;
      void *b1 = nullptr, *X1 = nullptr;
      MG_CHECK(dalloc(ctx, &b1, nc * sizeof(double2), s));
      fl.add(b1);
      MG_CHECK(dalloc(ctx, &X1, nc * sizeof(double2), s));
      fl.add(X1);
      MG_CHECK(restrict_fine(ctx, C->sub, B, b1, s));
      MG_CHECK(coarse_solve64(ctx, C, b1, X1, n, prm->tol * 0.1, s));
      MG_CHECK(prolong_coarse(ctx, C->sub, X1, X, false, s));
      MG_CHECK(unpack_spinor(ctx, X, sxc.dev + (size_t)off * V * 24, s));
    }
    for (int i = 0; i < n; ++i) {
      all_conv = all_conv && rs[i].converged;
      if (stats) {
        mglma_solve_stats& o = stats[off + i];
        o.iterations = rs[i].iterations;
        o.outer = rs[i].outer;
        o.coarse_iterations = rs[i].coarse_iterations;
        o.residual = rs[i].residual;
        o.converged = rs[i].converged ? 1 : 0;
        o.batch = n;
      }
    }
    off += n;
  }
  (void)ngroups;
  MG_CHECK(stage_out_finish(x, per * total, s, sx));
  if (x_coarse) MG_CHECK(stage_out_finish(x_coarse, per * total, s, sxc));
  MG_CUDA(cudaStreamSynchronize(s));
  if (!all_conv) return fail(MGLMA_ERR_NOT_CONVERGED, "solve_batch: some right-hand sides missed tol");
  return MGLMA_OK;
}

}  // extern "C"
