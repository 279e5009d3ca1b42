// Solver plumbing shared by solver.cu, multigrid.cu and capi.cu.
#pragma once
#include <vector>

#include "internal.h"

struct mglma_coarse_s;

namespace mglma {

struct SolveControl {
  double tol = 1e-10;    // target ||b - D x|| / ||b|| (FP64 true residual)
  int max_iter = 20000;  // iteration cap
  int check_every = 10;  // host polls residual norms every this many iterations
};

struct RhsStat {
  int iterations = 0;
  int outer = 0;
  long long coarse_iterations = 0;
  double residual = -1;
  bool converged = false;
};

// per-RHS scalars on the device: `d` holds count_d doubles per RHS, `z`
// count_z complex per RHS, `active` the convergence mask (1 = iterating)
struct Scalars {
  mglma_ctx ctx = nullptr;
  cudaStream_t s = nullptr;
  int nrhs = 0;
  double* d = nullptr;
  double2* z = nullptr;
  int* active = nullptr;
  std::vector<int> h_active;
  mglma_status alloc(mglma_ctx c, int n, int count_d, int count_z, cudaStream_t st);
  mglma_status push_active();
  ~Scalars();
};

// frees a list of pool allocations at scope exit (stream ordered)
struct FreeList {
  mglma_ctx c;
  cudaStream_t s;
  std::vector<void*> v;
  FreeList(mglma_ctx c_, cudaStream_t s_) : c(c_), s(s_) {}
  void add(void* p) { v.push_back(p); }
  ~FreeList() {
    for (void* q : v) dfree(c, q, s);
  }
};

mglma_status fill_int(int* p, int v, int n, cudaStream_t s);
mglma_status read_doubles(const double* dev, std::vector<double>& host, int n, cudaStream_t s);
mglma_status alloc_spinor(mglma_ctx ctx, Spinor& f, int prec, int nrhs, int64_t V, cudaStream_t s);

constexpr double2 C1 = {1.0, 0.0};
constexpr double2 CM1 = {-1.0, 0.0};
constexpr double2 C0 = {0.0, 0.0};

// CG step lengths: alpha = active ? zz / ww : 0 ; beta = active ? zz_new / zz : 0, zz <- zz_new
mglma_status cg_scalars(mglma_ctx, const double* zz, const double* ww, double2* alpha, const int* active, int n,
                        cudaStream_t s);
mglma_status cg_beta(mglma_ctx, const double* zz_new, double* zz, double2* beta, const int* active, int n,
                     cudaStream_t s);
// a[r] = <w, r>_r / |w|_r^2 (complex, in place allowed: a may alias num)
mglma_status mr_alpha(mglma_ctx ctx, const double2* num, const double* den, double2* a, int n, cudaStream_t s);

struct MgParams {
  double tol = 1e-10;
  int max_iter = 2000;
  int gcr_m = 4;
  int nu = 7;
  double inner_tol = 3e-6;
  double coarse_tol = 0.02;
  int coarse_max_iter = 108;
  int coarse_solver = MGLMA_COARSE_MINRES;
  int graph = 1;  // FGCR iterations as captured graphs
};

// the MG fields of the public parameter block
MgParams mg_params(const mglma_solve_params& p);

mglma_status mg_solve(mglma_ctx ctx, const mglma_gauge_s* G, const mglma_coarse_s* C, const Spinor& b, Spinor& x,
                      const MgParams& p, std::vector<RhsStat>& out, cudaStream_t s);
mglma_status coarse_solve64(mglma_ctx ctx, const mglma_coarse_s* C, const void* b1, void* X, int n, double tol,
                            cudaStream_t s);

mglma_status cgne64(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& b, Spinor& x, const SolveControl& ctl,
                    std::vector<RhsStat>& out, cudaStream_t s);
// even-odd (evenodd.cu): FP64 CGNE on the Schur complement S = A_ee - H_eo
// A_oo^-1 H_oe with reconstruction and FP64 defect correction on D
mglma_status cgne_eo64(mglma_ctx ctx, mglma_gauge_s* G, const Spinor& b, Spinor& x, const SolveControl& ctl,
                       std::vector<RhsStat>& out, cudaStream_t s);
// out = S in (g5: gamma5 S in) on the even sites of canonical device fields,
// zero on the odd sites (FP64)
mglma_status dirac_schur64(mglma_ctx ctx, mglma_gauge_s* G, int nrhs, const double* in_dev, double* out_dev, bool g5,
                           cudaStream_t s);

}  // namespace mglma
