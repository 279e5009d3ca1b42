// Internal definitions shared by the CUDA translation units of libmglma.
//
// Device layouts (all fields live in HBM; sites in the canonical lexicographic
// order ((x0*L1 + x1)*L2 + x2)*L3 + x3):
//   fine spinor batch, FP32 : [rhs][6 chunks][V] float4   (24 reals per site)
//   fine spinor batch, FP64 : [rhs][12 chunks][V] double2
//     chunk j of a site holds reals 4j..4j+3 (FP32) / 2j..2j+1 (FP64) of the
//     site vector, real index k = 2*(spin*3 + colour) + re/im.
//   gauge, FP64             : [mu][9][V] double2, full 3x3 (row-major)
//   gauge, FP32             : [mu][3][V] float4, rows 0 and 1 only
//                             (reconstruct-12: row2 = conj(row0 x row1))
//   clover, FP64            : [2 chiralities][18][V] double2
//   clover, FP32            : [2 chiralities][9][V] float4
//     each chirality block is a Hermitian 6x6 matrix on (spin mod 2)*3 +
//     colour, packed as 6 real diagonal entries then the 15 upper off-diagonal
//     entries (i<j, row-major) as (re, im) pairs: 36 reals.
//   coarse field            : [rhs][V1][2 Nv] complex (float2 / double2),
//                             dof index alpha*Nv + c
//   block basis, coarse operator: see subspace.h / subspace.cu / coarse.cu
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mglma.h"

namespace mglma {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
mglma_status fail(mglma_status st, const std::string& msg);

// "file.cu:line" of a check, for error messages
inline std::string src_line(const char* file, int line) {
  const char* b = file;
  for (const char* p = file; *p; ++p)
    if (*p == '/') b = p + 1;
  return std::string(b) + ":" + std::to_string(line);
}

// A failed runtime call is reported with its text and source line; the
// runtime's last-error slot is cleared so that a handled failure is not
// reported again by a later launch check.
#define MG_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      (void)cudaGetLastError();                                                    \
      return ::mglma::fail(MGLMA_ERR_CUDA, std::string(#call) + " (" +             \
                                               ::mglma::src_line(__FILE__, __LINE__) + \
                                               "): " + cudaGetErrorString(e_));    \
    }                                                                              \
  } while (0)

#define MG_CHECK(expr)                                                             \
  do {                                                                             \
    mglma_status s_ = (expr);                                                      \
    if (s_ != MGLMA_OK) return s_;                                                 \
  } while (0)

#define MG_LAUNCH_CHECK() MG_CUDA(cudaGetLastError())

// ---------------------------------------------------------------- geometry
struct Geom {
  int L[4];
  int64_t V;
  int t_bc;  // -1 antiperiodic, +1 periodic fermion hops across x0 = L0-1 <-> 0
};

inline Geom make_geom(const int L[4], int t_bc) {
  Geom g;
  for (int m = 0; m < 4; ++m) g.L[m] = L[m];
  g.V = (int64_t)L[0] * L[1] * L[2] * L[3];
  g.t_bc = t_bc;
  return g;
}

// ---------------------------------------------------------------- handles
struct KernelStat {
  std::string name;
  long long launches = 0;
  double ms = 0.0;
  double bytes = 0.0;  // algorithmic bytes of the timed launches
  double flops = 0.0;  // algorithmic flops of the timed launches
};

}  // namespace mglma

#include <map>
#include <tuple>

struct mglma_ctx_s {
  int device = 0;
  // per-stream scratch of the reductions: partial sums and tickets
  struct RedScratch {
    double2* part = nullptr;
    unsigned* count = nullptr;
    size_t part_cap = 0;
    int count_cap = 0;
  };
  std::map<cudaStream_t, RedScratch> red;
  // autotuned tile choices: (kernel, RHS bucket, lattice volume) -> (choice,
  // ms); volume 0 applies to every lattice (mglma_autotune_set)
  std::map<std::tuple<int, int, int64_t>, std::pair<int, double>> tune;
  std::string tune_cache;  // file the table is saved to after automatic tuning ("" = none)
  cudaStream_t stream = nullptr;  // default stream of the context
  cudaMemPool_t pool = nullptr;
  int sm_count = 0;
  // optional per-kernel timing (CUDA events around launches)
  bool profile = false;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
    double bytes, flops;
  };
  std::vector<Pending> pending;
  // while a CUDA graph is captured with profiling on, launch brackets become
  // external event-record nodes listed here (resolved after each replay)
  std::vector<Pending>* capture_events = nullptr;
  std::vector<cudaEvent_t> event_cache;
  bool coarse_level = false;  // see CoarseLevelScope
  mglma::KernelStat stats[16];
};

struct mglma_gauge_s {
  mglma_ctx ctx = nullptr;
  mglma::Geom g;
  double kappa = 0, csw = 0, m0 = 0;
  double2* U64 = nullptr;  // [4][9][V]
  float4* U32 = nullptr;   // [4][3][V]
  double2* C64 = nullptr;  // [2][18][V]
  float4* C32 = nullptr;   // [2][9][V]
  double2* Cinv64 = nullptr;  // [2][18][V] inverse clover blocks (even-odd, formed on first use)
  float4* Udf = nullptr;      // [4][9][V] U64 split into double-float (re.hi, re.lo, im.hi, im.lo), first use
  float4* Cdf = nullptr;      // [2][18][V] C64 split likewise (two reals per float4), first use
  int slabs_loaded = 0;   // time slices received
  std::vector<char> slab_seen;
  bool ready = false;
  double unitarity_dev = 0;  // max |U U^dag - 1| seen at load
};

namespace mglma {

// tile-choice keys of the autotuner
enum TuneKernel { TUNE_DSLASH32_NR = 0, TUNE_COARSE_NT = 1 };
inline int rhs_bucket(int n) {
  int b = 1;
  while (b < n && b < 64) b *= 2;
  return b;
}
// the tuned choice for this lattice volume, else the one set for every
// lattice, else dflt
inline int tuned(const mglma_ctx_s* ctx, int kernel, int nrhs, int64_t volume, int dflt) {
  auto it = ctx->tune.find(std::make_tuple(kernel, rhs_bucket(nrhs), volume));
  if (it == ctx->tune.end()) it = ctx->tune.find(std::make_tuple(kernel, rhs_bucket(nrhs), (int64_t)0));
  return it == ctx->tune.end() ? dflt : it->second.first;
}
inline bool has_tuned(const mglma_ctx_s* ctx, int kernel, int nrhs, int64_t volume) {
  return ctx->tune.count(std::make_tuple(kernel, rhs_bucket(nrhs), volume)) > 0;
}
// FP32 stencil tile codes: NR RHS per thread (1, 2, 4) and RW RHS tiles per
// CTA (1, 2, 4), code = NR + 16 (RW - 1); codes 1, 2, 4 are RW = 1.  Codes
// 64 + NRT (NRT = 4, 8, 16) select the staged-tile kernel: 32 sites x NRT
// RHS per CTA with links and clover staged in shared memory.
inline int dslash32_tile_code(int nr, int rw) { return nr + 16 * (rw - 1); }
inline int dslash32_tile_nr(int code) { return code & 15; }
inline int dslash32_tile_rw(int code) { return 1 + (code >> 4); }
inline bool dslash32_tile_staged(int code) { return code == 68 || code == 72 || code == 80; }
inline int dslash32_tile_nrt(int code) { return code - 64; }
inline bool dslash32_tile_valid(int code) {
  if (dslash32_tile_staged(code)) return true;
  const int nr = dslash32_tile_nr(code), rw = dslash32_tile_rw(code);
  return code > 0 && code < 64 && (nr == 1 || nr == 2 || nr == 4) && (rw == 1 || rw == 2 || rw == 4) &&
         (nr < 4 || rw == 1);
}
int dslash32_default_tile(int nrhs);

// kernel-statistics kinds (timing is optional, see mglma_profile)
enum KernelKind {
  K_DSLASH64 = 0,
  K_DSLASH32 = 1,
  K_BLAS = 2,
  K_REDUCE = 3,
  K_RESTRICT = 4,
  K_PROLONG = 5,
  K_COARSE = 6,
  K_PACK = 7,
  K_SETUP = 8,
  K_SCALAR = 9,
  K_CBLAS = 10,    // BLAS-1 on coarse fields (inside a coarse solve)
  K_CREDUCE = 11,  // reductions on coarse fields
  K_CONTRACT = 12, // time-slice contractions
  K_NKINDS = 13
};
// While alive, BLAS and reduction launches on the context count as coarse-level
// work in the per-kernel statistics.
struct CoarseLevelScope {
  mglma_ctx ctx;
  bool prev;
  explicit CoarseLevelScope(mglma_ctx c);
  ~CoarseLevelScope();
};
const char* kernel_kind_name(int k);

// Event bracket around one launch when profiling is on.
struct ProfScope {
  mglma_ctx ctx;
  int kind;
  cudaStream_t s;
  double bytes, flops;
  cudaEvent_t a = nullptr, b = nullptr;
  bool captured = false;
  ProfScope(mglma_ctx c, int k, cudaStream_t st, double bytes_ = 0, double flops_ = 0);
  ~ProfScope();
};

// tile shapes of this (lattice, RHS bucket) tuned unless already known (tune.cu)
mglma_status autotune_for_batch(mglma_ctx ctx, mglma_gauge_s* G, struct ::mglma_coarse_s* C, int nrhs);

// ---------------------------------------------------------------- memory
mglma_status dalloc(mglma_ctx ctx, void** p, size_t bytes, cudaStream_t s);
void dfree(mglma_ctx ctx, void* p, cudaStream_t s);
bool is_device_pointer(const void* p);
// Bytes the context can still allocate: the device's free memory plus the
// blocks its pool holds cached but unused (waits for stream s first, so
// stream-ordered frees have returned to the pool).
size_t device_room(mglma_ctx ctx, cudaStream_t s);
// MGLMA_ERR_INVALID unless the gauge field was loaded on ctx's device.
mglma_status check_gauge_device(mglma_ctx ctx, const mglma_gauge_s* G, const char* who);

// host-or-device staging of one canonical buffer (capi.cu)
struct Staged {
  mglma_ctx ctx = nullptr;
  cudaStream_t s = nullptr;
  double* dev = nullptr;
  bool owned = false;
  ~Staged() {
    if (owned) dfree(ctx, dev, s);
  }
};
mglma_status stage_in(mglma_ctx ctx, const double* p, size_t bytes, cudaStream_t s, Staged& st);
mglma_status stage_out_alloc(mglma_ctx ctx, double* p, size_t bytes, cudaStream_t s, Staged& st);
mglma_status stage_out_finish(double* p, size_t bytes, cudaStream_t s, Staged& st);
cudaStream_t pick_stream(mglma_ctx ctx, void* s);

// ---------------------------------------------------------------- fine fields
// Internal spinor batch (see layout at top).
struct Spinor {
  void* p = nullptr;
  int prec = MGLMA_FP32;  // MGLMA_FP64 or MGLMA_FP32; MGLMA_BF16 for the MR smoother's fields
  int nrhs = 0;
  int64_t V = 0;
  size_t rhs_reals() const { return (size_t)24 * V; }
  size_t bytes() const { return rhs_reals() * nrhs * (prec == MGLMA_FP64 ? 8 : prec == MGLMA_BF16 ? 2 : 4); }
};

// conversions canonical complex128 (device) <-> internal
mglma_status pack_spinor(mglma_ctx, const double* canon, Spinor& dst, cudaStream_t s);
mglma_status unpack_spinor(mglma_ctx, const Spinor& src, double* canon, cudaStream_t s);
// dst = scale_r * src (+ dst when accumulate); precisions may differ; scale
// (device, per RHS) NULL means 1
mglma_status convert_spinor(mglma_ctx, const Spinor& src, Spinor& dst, cudaStream_t s, const double* scale = nullptr,
                            bool accumulate = false);

// fine operator application: out = op(in), op in {D, D^dag, gamma5 D, gamma5 D^dag}
mglma_status dslash(mglma_ctx, const mglma_gauge_s* G, const Spinor& in, Spinor& out, bool dagger,
                    bool gamma5_out, cudaStream_t s);
// One fused MR smoothing step (the (1,1) stencil tile; t, tn, sk FP32 or all
// BF16, z FP32): with u = D t,
// tn = t - alpha u, sk <- sk - alpha t, z <- z + alpha sk (alpha per RHS, the
// previous step's), and per RHS nrm = |tn|^2, dot = <tn, sk_new>, reduced as
// in dslash_dot.  The four fields must differ.  dslash_mr_fused says whether
// the tuned stencil tile for nrhs RHS has this form (else the step runs as
// dslash_dot plus a vector update).
bool dslash_mr_fused(mglma_ctx, const mglma_gauge_s* G, int nrhs);
// FGCR direction image out = D in (FP32, the (1,1) tile) with its dots in the
// same pass: k = 0 -> nw[r] = |out|^2, num[r] = <out, res>; k = 1..3 ->
// dots[j n + r] = <W_j, out> for the earlier images W_j = W0 + j wslot reals;
// part: dslash_gcr_part_doubles(V, nrhs) doubles of scratch
size_t dslash_gcr_part_doubles(int64_t V, int nrhs);
mglma_status dslash_gcr(mglma_ctx, const mglma_gauge_s* G, const Spinor& in, Spinor& out, int k, const void* W0,
                        size_t wslot_reals, const void* res, double* part, double* nw, double2* num, double2* dots,
                        cudaStream_t s);
// z += alpha s (per-RHS alpha) for BF16 s and FP32 z: the last MR step
mglma_status mr_zupdate(mglma_ctx, const double2* alpha, const Spinor& sk, Spinor& z, cudaStream_t s);
mglma_status dslash_mr_step(mglma_ctx, const mglma_gauge_s* G, const Spinor& t, Spinor& tn, Spinor& sk, Spinor& z,
                            const double2* alpha, double* part, double* nrm, double2* dot, cudaStream_t s);
// out = b - D in (FP32; the residual of the preconditioner's coarse correction
// formed in the stencil's epilogue); out must not alias in or b
// r -= scale[rhs] D e per RHS: e FP32, r FP64, D applied in double-float
// arithmetic (about 2^-47 relative to the terms) on the FP64 links and clover
// split once into double-float words (kept on the gauge handle)
mglma_status dslash_resid_df(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& e, Spinor& r, const double* scale,
                             cudaStream_t s);
mglma_status dslash_resid(mglma_ctx, const mglma_gauge_s* G, const Spinor& in, const Spinor& b, Spinor& out,
                          cudaStream_t s);
// FP32 t = D in with, per RHS, nrm = |t|^2 and dot = <t, in> = sum conj(t) in
// reduced in the same pass (FP32 per warp of 32 sites, then FP64 partials per
// 32-site tile in `part`, at least dslash_dot_part_doubles(V, nrhs) doubles,
// summed in a fixed order).
mglma_status dslash_dot(mglma_ctx, const mglma_gauge_s* G, const Spinor& in, Spinor& out, double* part, double* nrm,
                        double2* dot, cudaStream_t s);
size_t dslash_dot_part_doubles(int64_t V, int nrhs);
// single hop-slot pieces of D in FP64, used to assemble the coarse operator:
// slot d < 8: the hop term of slot d at sites whose hop leaves their block
// (zero elsewhere); slot 8: clover term plus every hop that stays in the block.
mglma_status dslash_slot64_batch(mglma_ctx, const mglma_gauge_s* G, const int block[4], const Spinor& in,
                                 Spinor& out, int slot, cudaStream_t s);


// ---------------------------------------------------------------- BLAS-1 (multi-RHS)
// Every scalar is per RHS and lives in device memory.  All vectors are rhs-major
// blocks of n reals (n = 24 V for fine fields, 4 Nv V1 for coarse fields).
struct Vec {
  void* p = nullptr;
  int prec = MGLMA_FP32;
  int nrhs = 0;
  size_t n = 0;  // reals per RHS (multiple of 4)
  size_t bytes() const { return n * (size_t)nrhs * (prec == MGLMA_FP64 ? 8 : prec == MGLMA_BF16 ? 2 : 4); }
};
inline Vec as_vec(const Spinor& s) {
  Vec v;
  v.p = s.p;
  v.prec = s.prec;
  v.nrhs = s.nrhs;
  v.n = s.rhs_reals();
  return v;
}

// y = a x + b y (complex a, b per RHS from device arrays; a NULL uses a_def
// for every RHS, b NULL uses b_def); sign scales a
mglma_status axpby(mglma_ctx, const double2* a, double2 a_def, const Vec& x, const double2* b, double2 b_def,
                   Vec& y, cudaStream_t s, double sign = 1.0);
mglma_status caxpy(mglma_ctx, const double2* a, const Vec& x, Vec& y, cudaStream_t s, double sign = 1.0);
// x += a p ; r -= a w
mglma_status axpy2(mglma_ctx, const double2* a, const Vec& p, Vec& x, const Vec& w, Vec& r, cudaStream_t s);
// r -= a w with rr = |r|^2 per RHS (FP32)
mglma_status axpy_norm(mglma_ctx, const double2* a, const Vec& w, Vec& r, double* rr, cudaStream_t s);
// multi_axpy on FP32 fields with nrm = |y_new|^2 and dot = <y_new, w> per RHS
// in the same pass
mglma_status multi_axpy_nd(mglma_ctx, const Vec& x0, size_t jstride_reals, int k, Vec& y, const double2* c,
                           const Vec* x0b, Vec* yb, const Vec& w, double* nrm, double2* dot, cudaStream_t s);
// y -= sum_{j<k} c[j*nrhs + r] x_j  where x_j starts jstride reals after x_{j-1}
// (x0b, yb optional: a second set updated with the same coefficients)
mglma_status multi_axpy(mglma_ctx, const Vec& x0, size_t jstride_reals, int k, Vec& y, const double2* c,
                        cudaStream_t s, const Vec* x0b = nullptr, Vec* yb = nullptr);
mglma_status copy_vec(mglma_ctx, const Vec& x, Vec& y, cudaStream_t s);
mglma_status zero_vec(mglma_ctx, Vec& y, cudaStream_t s);
// out[r] = <x_r, y_r> = sum conj(x) y (FP64 accumulation, deterministic)
mglma_status cdot(mglma_ctx, const Vec& x, const Vec& y, double2* out, cudaStream_t s);
// out[j*nrhs + r] = <x_j,r, y_r> for j < k
mglma_status multi_cdot(mglma_ctx, const Vec& x0, size_t jstride_reals, int k, const Vec& y, double2* out,
                        cudaStream_t s);
// out[r] = |x_r|^2
mglma_status norm2(mglma_ctx, const Vec& x, double* out, cudaStream_t s);
// allocates the stream's reduction scratch (must happen before a graph capture)
mglma_status red_scratch_ready(mglma_ctx, cudaStream_t s);
// accumulates the launch times of a replayed graph's event brackets
void resolve_graph_events(mglma_ctx ctx, const std::vector<mglma_ctx_s::Pending>& ev);
// nrm[r] = |x_r|^2 and dot[r] = <x_r, y_r> in one pass
mglma_status norm2_cdot(mglma_ctx, const Vec& x, const Vec& y, double* nrm, double2* dot, cudaStream_t s);
// x += a p ; r -= a w ; rr[r] = |r_r|^2 in one pass
mglma_status axpy2_norm(mglma_ctx, const double2* a, const Vec& p, Vec& x, const Vec& w, Vec& r, double* rr,
                        cudaStream_t s);
// MINRES: z -= Re(dot_r) v + beta_r u, zz[r] = |z_r|^2 (RHS with active[r] == 0
// are left alone, zz = 0)
// st (nullable): also runs the MINRES scalar step of each RHS (minres.cuh)
// in the kernel's last block; zz must then be st's MR_BN2 slot
mglma_status lanczos_norm(mglma_ctx, const double2* dot, const double* beta, int* active, const Vec& v,
                          const Vec& u, Vec& z, double* zz, cudaStream_t s, double* st = nullptr, double tol = 0,
                          int cap = 0);
// MINRES: wn = c0 v + c1 w1 + c2 w2 ; x += c3 wn ; z *= c4 for RHS with c5 != 0,
// c_j[r] = cf[j * stride + r] (real, device)
mglma_status minres_update(mglma_ctx, const double* cf, int stride, const Vec& v, const Vec& w1, const Vec& w2,
                           Vec& wn, Vec& x, Vec& z, cudaStream_t s);
// y = scale_r gamma5hat x on coarse fields of n2 dofs per site (scale device, per RHS)
mglma_status coarse_g5_scale(mglma_ctx, const Vec& x, Vec& y, const double* scale, int n2, cudaStream_t s);

}  // namespace mglma
