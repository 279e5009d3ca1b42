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
#include <cmath>
#include <functional>

#include "internal.h"
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

static Vec dir(const Vec& base, int j) {
  Vec v = base;
  v.p = (char*)base.p + (size_t)j * base.bytes();
  return v;
}

struct GcrResult {
  int iterations = 0;
  std::vector<int> per_rhs;  // iterations while active (when polled every step)
};

// Batched flexible GCR(m): x = A^-1 b per RHS to |r| <= tol |b| (or max_iter).
// M (nullable) is the right preconditioner.  poll_every > 0 reads the active
// mask on the host every that many iterations and stops when all converged.
static mglma_status gcr(mglma_ctx ctx, cudaStream_t s, const OpFn& A, const OpFn* M, const Vec& b, Vec& x, int m,
                        int max_iter, double tol, int poll_every, GcrResult& res) {
  const int n = b.nrhs;
  res = GcrResult();
  res.per_rhs.assign(n, 0);
  if (n == 0) return MGLMA_OK;
  FreeList fl(ctx, s);
  Vec Z = b, W = b, r = b;
  MG_CHECK(dalloc(ctx, &Z.p, b.bytes() * m, s));
  fl.add(Z.p);
  MG_CHECK(dalloc(ctx, &W.p, b.bytes() * m, s));
  fl.add(W.p);
  MG_CHECK(dalloc(ctx, &r.p, b.bytes(), s));
  fl.add(r.p);
  Scalars sc;
  MG_CHECK(sc.alloc(ctx, n, m + 2, 2 * m + 2, s));
  double* nw = sc.d;             // [m][n]
  double* rr = sc.d + m * n;     // [n]
  double* bb = sc.d + (m + 1) * n;
  double2* dots = sc.z;          // [m][n]
  double2* coef = sc.z + m * n;  // [m][n]
  double2* num = sc.z + 2 * m * n;
  double2* a = sc.z + (2 * m + 1) * n;
  const size_t stride = (size_t)n * b.n;  // reals between directions
  MG_CHECK(zero_vec(ctx, x, s));
  MG_CHECK(copy_vec(ctx, b, r, s));
  MG_CHECK(norm2(ctx, b, bb, s));
  const double tol2 = tol * tol;
  const int tb = 64, nb = (n + tb - 1) / tb;
  gcr_mask_kernel<<<nb, tb, 0, s>>>(bb, bb, 0.0, sc.active, n);  // zero sources never become active
  std::vector<int> hact(n, 1), prev(n, 1);
  if (poll_every == 1) {
    MG_CUDA(cudaMemcpyAsync(prev.data(), sc.active, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
  }
  int it = 0;
  while (it < max_iter) {
    const int k = it % m;
    Vec Zk = dir(Z, k), Wk = dir(W, k);
    if (M) {
      MG_CHECK((*M)(r, Zk));
    } else {
      MG_CHECK(copy_vec(ctx, r, Zk, s));
    }
    MG_CHECK(A(Zk, Wk));
    if (k > 0) {
      MG_CHECK(multi_cdot(ctx, W, stride, k, Wk, dots, s));
      {
        ProfScope ps(ctx, K_SCALAR, s);
        gcr_coef_kernel<<<(k * n + 63) / 64, 64, 0, s>>>(dots, nw, coef, k, n);
      }
      MG_CHECK(multi_axpy(ctx, W, stride, k, Wk, coef, s));
      MG_CHECK(multi_axpy(ctx, Z, stride, k, Zk, coef, s));
    }
    MG_CHECK(norm2_cdot(ctx, Wk, r, nw + (size_t)k * n, num, s));
    {
      ProfScope ps(ctx, K_SCALAR, s);
      gcr_alpha_kernel<<<nb, tb, 0, s>>>(num, nw + (size_t)k * n, sc.active, a, n);
    }
    MG_CHECK(axpy2_norm(ctx, a, Zk, x, Wk, r, rr, s));
    {
      ProfScope ps(ctx, K_SCALAR, s);
      gcr_mask_kernel<<<nb, tb, 0, s>>>(rr, bb, tol2, sc.active, n);
    }
    MG_LAUNCH_CHECK();
    ++it;
    if (poll_every > 0 && (it % poll_every == 0 || it == max_iter)) {
      MG_CUDA(cudaMemcpyAsync(hact.data(), sc.active, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
      MG_CUDA(cudaStreamSynchronize(s));
      bool any = false;
      for (int i = 0; i < n; ++i) {
        if (poll_every == 1 && prev[i]) res.per_rhs[i]++;  // active going into this iteration
        any = any || hact[i];
      }
      prev = hact;
      if (!any) break;
    }
  }
  res.iterations = it;
  if (poll_every != 1)
    for (int i = 0; i < n; ++i) res.per_rhs[i] = it;
  return MGLMA_OK;
}

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
  Vec b1, e1, sv, tv;
  Scalars sc;
  bool ready = false;
  ~TwoLevel() {
    dfree(ctx, b1.p, s);
    dfree(ctx, e1.p, s);
    dfree(ctx, sv.p, s);
    dfree(ctx, tv.p, s);
  }
  mglma_status setup(const Vec& r) {
    const int n = r.nrhs;
    b1.prec = e1.prec = MGLMA_FP32;
    b1.nrhs = e1.nrhs = n;
    b1.n = e1.n = (size_t)C->geo.V1 * C->n2 * 2;
    MG_CHECK(dalloc(ctx, &b1.p, b1.bytes(), s));
    MG_CHECK(dalloc(ctx, &e1.p, e1.bytes(), s));
    sv = r;
    tv = r;
    sv.p = tv.p = nullptr;
    MG_CHECK(dalloc(ctx, &sv.p, r.bytes(), s));
    MG_CHECK(dalloc(ctx, &tv.p, r.bytes(), s));
    MG_CHECK(sc.alloc(ctx, n, 1, 1, s));
    ready = true;
    return MGLMA_OK;
  }
  mglma_status operator()(const Vec& r, Vec& z) {
    if (!ready) MG_CHECK(setup(r));
    const int n = r.nrhs;
    const mglma_subspace_s* S = C->sub;
    const int64_t V = S->geo.V;
    Spinor rs = as_spinor(r, V), zs = as_spinor(z, V);
    MG_CHECK(restrict_fine(ctx, S, rs, b1.p, s));
    OpFn Ac = [&](const Vec& in, Vec& out) { return coarse_apply(ctx, C, in.p, out.p, in.nrhs, MGLMA_FP32, false, s); };
    GcrResult cr;
    MG_CHECK(gcr(ctx, s, Ac, nullptr, b1, e1, 16, p->coarse_max_iter, p->coarse_tol, 10, cr));
    coarse_iters += cr.iterations;
    MG_CHECK(prolong_coarse(ctx, S, e1.p, zs, false, s));
    if (p->nu > 0) {
      // s = r - D z ; nu MR steps on D e = s, accumulated into z
      Spinor ss = as_spinor(sv, V), ts = as_spinor(tv, V);
      MG_CHECK(dslash(ctx, G, zs, ts, false, false, s));
      MG_CHECK(copy_vec(ctx, r, sv, s));
      MG_CHECK(axpby(ctx, nullptr, CM1, tv, nullptr, C1, sv, s));
      for (int k = 0; k < p->nu; ++k) {
        MG_CHECK(dslash(ctx, G, ss, ts, false, false, s));
        MG_CHECK(cdot(ctx, tv, sv, sc.z, s));
        MG_CHECK(norm2(ctx, tv, sc.d, s));
        MG_CHECK(mr_alpha(ctx, sc.z, sc.d, sc.z, n, s));
        MG_CHECK(axpy2(ctx, sc.z, sv, z, tv, sv, s));
      }
    }
    return MGLMA_OK;
  }
};

// x (FP64, zero on entry) = D^-1 b to p.tol in the FP64 residual.
mglma_status mg_solve(mglma_ctx ctx, const mglma_gauge_s* G, const mglma_coarse_s* C, const Spinor& b, Spinor& x,
                      const MgParams& p, std::vector<RhsStat>& out, cudaStream_t s) {
  const int n = b.nrhs;
  const int64_t V = b.V;
  out.assign(n, RhsStat());
  FreeList fl(ctx, s);
  Spinor r, w, r32, e32;
  MG_CHECK(alloc_spinor(ctx, r, MGLMA_FP64, n, V, s));
  fl.add(r.p);
  MG_CHECK(alloc_spinor(ctx, w, MGLMA_FP64, n, V, s));
  fl.add(w.p);
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
  Vec vb = as_vec(b), vx = as_vec(x), vr = as_vec(r), vw = as_vec(w);
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
    GcrResult gr;
    MG_CHECK(gcr(ctx, s, A, &Kf, v32, e, p.gcr_m, p.max_iter - total_inner, p.inner_tol, 1, gr));
    total_inner += gr.iterations;
    for (int i = 0; i < n; ++i) {
      out[i].iterations += gr.per_rhs[i];
      if (!out[i].converged) out[i].outer++;
    }
    // x += |r| e ; r = b - D x (FP64)
    MG_CHECK(convert_spinor(ctx, e32, x, s, rn, true));
    MG_CHECK(dslash(ctx, G, x, w, false, false, s));
    MG_CHECK(copy_vec(ctx, vb, vr, s));
    MG_CHECK(axpby(ctx, nullptr, CM1, vw, nullptr, C1, vr, s));
  }
  for (int i = 0; i < n; ++i) out[i].coarse_iterations = K.coarse_iters;
  return coarse_tc_check(const_cast<mglma_coarse_s*>(C), s);
}

// X (FP64 coarse, [n][V1][n2]) = D1^-1 b1 to tol by FP64 defect correction
// around FP32 coarse GCR.
mglma_status coarse_solve64(mglma_ctx ctx, const mglma_coarse_s* C, const void* b1, void* X, int n, double tol,
                            cudaStream_t s) {
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
  OpFn Ac = [&](const Vec& in, Vec& out) { return coarse_apply(ctx, C, in.p, out.p, in.nrhs, MGLMA_FP32, false, s); };
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
    MG_CHECK(coarse_apply(ctx, C, vx.p, vw.p, n, MGLMA_FP64, false, s));
    MG_CHECK(copy_vec(ctx, vb, vr, s));
    MG_CHECK(axpby(ctx, nullptr, CM1, vw, nullptr, C1, vr, s));
  }
  return fail(MGLMA_ERR_NOT_CONVERGED, "coarse solve: FP64 defect correction did not reach tol");
}

}  // namespace mglma
