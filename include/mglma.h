/* mglma -- GB300 (sm_103a) hot path of multigrid low-mode averaging.
 *
 * C ABI of libmglma.so.  The operations follow arXiv:2412.06347 (Gruber,
 * Harris, Krstic Marinkovic, "Multigrid low-mode averaging"); each entry
 * point names the passage that defines what it computes.
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice: x = (x0, x1, x2, x3), x0 is time, extents L[0..3]; the canonical
 *   site index is ((x0*L1 + x1)*L2 + x2)*L3 + x3; V = L0 L1 L2 L3.
 * Canonical spinor batch: complex128, interleaved (re, im), index order
 *   [rhs][site][spin 4][colour 3]; 24 doubles per site per RHS.
 * Canonical links: complex128 [site][mu 4][row 3][col 3]; U_mu(x) sits on the
 *   link x -> x + mu.  Links are periodic.
 * Gamma matrices: chiral basis, gamma5 = diag(1, 1, -1, -1); chirality
 *   alpha = 0 is spins {0, 1}, alpha = 1 is spins {2, 3}.
 * Dirac operator (the paper uses O(a)-improved Wilson fermions, Tab.
 *   ensembles, without printing D):
 *     D psi(x) = A(x) psi(x) - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                         + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)]
 *     A(x) = 4 + m0 + c_sw (i/4) sum_{mu nu} sigma_{mu nu} Fhat_{mu nu}(x),
 *     m0 = 1/(2 kappa) - 4, Fhat from the four clover leaves; a fermion hop
 *     across the time boundary is multiplied by t_bc.  This is D itself, not
 *     2 kappa D.
 * Blocks (Sec. 3, Eqs. block_decomp, block_def): sides b[mu] dividing L[mu];
 *   block y_mu = x_mu / b_mu, block index and site-in-block index
 *   lexicographic like the site index.
 * Coarse fields: complex128 [rhs][coarse site][2 Nv], dof alpha*Nv + c.
 * Coarse operator export: complex128 [9 slots][V1][2Nv][2Nv]; slot d < 4 is
 *   the +mu neighbour, 4..7 the -mu neighbour, 8 the block itself.
 *
 * Pointers: every double* argument may be host memory (pageable or pinned)
 *   or device memory of the context's device; the library detects which.
 *   Host inputs are copied in and host outputs copied out before the call
 *   returns.  Device buffers are read/written in stream order on the given
 *   stream (NULL = the context's own stream) and must stay valid until that
 *   stream reaches the call's work.  The caller owns all buffers it passes;
 *   the library owns every handle until the matching *_free.
 * Errors: every call returns an mglma_status; nothing throws across the ABI.
 *   mglma_last_error() returns a thread-local message for the last failure.
 */
#ifndef MGLMA_H
#define MGLMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mglma_ctx_s* mglma_ctx;
typedef struct mglma_gauge_s* mglma_gauge;
typedef struct mglma_subspace_s* mglma_subspace;
typedef struct mglma_coarse_s* mglma_coarse;

typedef enum {
  MGLMA_OK = 0,
  MGLMA_ERR_INVALID = 1,       /* bad argument (sizes, NULL, blocking)          */
  MGLMA_ERR_OOM = 2,           /* device allocation failed                      */
  MGLMA_ERR_CUDA = 3,          /* a CUDA runtime call failed                    */
  MGLMA_ERR_RANK = 4,          /* a block basis vector is linearly dependent    */
  MGLMA_ERR_NOT_CONVERGED = 5, /* iteration cap reached; best iterate returned  */
  MGLMA_ERR_NUMERIC = 6,       /* non-finite value met                          */
  MGLMA_ERR_TIMEOUT = 7,       /* a bounded device wait gave up                 */
  MGLMA_ERR_REJECTED = 8       /* admission refused (serving)                   */
} mglma_status;

typedef enum { MGLMA_FP64 = 0, MGLMA_FP32 = 1, MGLMA_BF16 = 2, MGLMA_FP16 = 3 } mglma_prec;

typedef enum {
  MGLMA_OP_D = 0,        /* D                 */
  MGLMA_OP_DDAG = 1,     /* D^dag = g5 D g5   */
  MGLMA_OP_Q = 2,        /* Q = gamma5 D (Sec. 2) */
  MGLMA_OP_DDAGD = 3,    /* D^dag D           */
  MGLMA_OP_SCHUR = 4,    /* S = A_ee - H_eo A_oo^-1 H_oe, the even-odd
                            preconditioned operator on the even sites
                            (x0 + x1 + x2 + x3 even); coarse: D_ee - D_eo D_oo^-1 D_oe */
  MGLMA_OP_SCHUR_Q = 5   /* gamma5 S (coarse: g5hat S_ee), Hermitian */
} mglma_op;

typedef struct {
  int L[4];
  int t_bc; /* -1 antiperiodic (default), +1 periodic */
} mglma_lattice;

/* ---------------------------------------------------------------- context */
/* Creates a context on CUDA device `device` (own stream and memory pool). */
mglma_status mglma_create(int device, mglma_ctx* out);
void mglma_destroy(mglma_ctx ctx);
const char* mglma_last_error(void);
/* Library version string. */
const char* mglma_version(void);

/* Per-kernel timing with CUDA events on the launching stream (off by
 * default).  enable = 1 starts collecting, 0 stops; reset clears. */
mglma_status mglma_profile(mglma_ctx ctx, int enable, int reset);
/* Fetches the accumulated launches, milliseconds, algorithmic bytes and
 * algorithmic flops of kernel class `name` ("dslash64", "dslash32", "blas",
 * "reduce", "restrict", "prolong", "coarse", "pack", "setup", "scalar",
 * "cblas", "creduce", "contract"; "cblas" and "creduce" are BLAS-1 and
 * reductions on coarse fields inside coarse solves, "blas" and "reduce" the
 * fine-level ones).  Algorithmic
 * bytes count every operand read once and every result written once (for
 * the stencil: links, clover, input and output spinors).  Waits for the
 * recorded events.  Any output pointer may be NULL. */
mglma_status mglma_profile_get(mglma_ctx ctx, const char* name, long long* launches, double* ms, double* bytes,
                               double* flops);

/* ---------------------------------------------------------------- gauge field */
/* Loads links and builds everything the operator needs: reconstruct-12 FP32
 * and full FP64 copies of U, the clover term A(x) with the mass folded in,
 * both chirality blocks (O(a)-improved Wilson-clover action, Tab. ensembles).
 * links: canonical complex128 links of time slices t_begin .. t_begin +
 *   t_count - 1 (host or device).  Pass *inout = NULL on the first slab; the
 *   handle is created and returned.  The clover term is built when the last
 *   missing time slice arrives; only then can the handle be used.
 * Links must be SU(3) to 1e-10 (rows orthonormal, det 1): reconstruct-12
 *   relies on it; larger deviations give MGLMA_ERR_INVALID. */
mglma_status mglma_gauge_load(mglma_ctx ctx, const mglma_lattice* lat, const double* links, int64_t t_begin,
                              int64_t t_count, double kappa, double csw, mglma_gauge* inout);
/* Generates the synthetic gauge field of the benchmark configurations on the
 * device and loads it as mglma_gauge_load would: link (x, mu) is
 * P_SU3(exp(i eps H)) with H = sum_a h_a lambda_a / 2, h_a ~ N(0, 1) the
 * Gaussians 8 n .. 8 n + 7 (n = 4 x + mu) of the SplitMix64 counter stream
 * (seed, tag 1), Box-Muller pairs; exp by an order-18 Taylor series, then
 * row Gram-Schmidt and row2 = conj(row0 x row1).  This is an input
 * generator, not part of the paper's method: it reproduces the library's
 * Python input generator to rounding (CUDA's log / sin / cos), so that
 * lattices too large to generate on the host (96x48^3, 128x64^3) can be set
 * up.  Works in time slabs of at most 512 MB; *out receives a new handle. */
mglma_status mglma_gauge_random(mglma_ctx ctx, const mglma_lattice* lat, double eps, uint64_t seed, double kappa,
                                double csw, mglma_gauge* out);
void mglma_gauge_free(mglma_gauge g);
/* Lattice extents and V of a gauge handle. */
mglma_status mglma_gauge_info(mglma_gauge g, int L[4], int64_t* volume);

/* Applies op to nrhs canonical spinors: out = op(in).  compute selects the
 * arithmetic: MGLMA_FP64 (FP64 links and clover) or MGLMA_FP32 (FP32
 * reconstruct-12 links, FP32 clover, inputs rounded to FP32).  The definition
 * of D is the one stated at the top of this header (Sec. 2: Q = gamma5 D).
 * MGLMA_OP_SCHUR / _SCHUR_Q (FP64 only, every extent even): the even-odd
 * operator S (or gamma5 S) reads the even sites of in and writes the even
 * sites of out, zero on the odd ones; the first call on a gauge field forms
 * the inverse clover blocks (two Hermitian 6x6 per site, FP64). */
mglma_status mglma_dirac_apply(mglma_ctx ctx, mglma_gauge g, mglma_op op, int nrhs, const double* in, double* out,
                               mglma_prec compute, void* cuda_stream);

/* Allocation-free variant of mglma_dirac_apply.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need the operator -- code running while a CUDA
 * graph is being captured, code called from inside an allocator hook, or a
 * process whose HBM is already fully reserved by another caching allocator.
 * It computes exactly what mglma_dirac_apply computes, but its two
 * internal-layout work fields live in one file-scope device array of 32 MiB
 * that the library holds on every GPU that loads it, until the process
 * exits; the call makes no cudaMalloc/cudaFree and no allocating library call.
 *   in, out: DEVICE pointers to nrhs canonical spinors (host pointers are
 *     rejected with MGLMA_ERR_INVALID: staging them would need memory).
 *   Limit: 2 x nrhs x V x 24 x (8 for FP64, 4 for FP32) bytes <= 32 MiB,
 *     i.e. nrhs x V <= 87381 (FP64) or 174762 (FP32); larger requests return
 *     MGLMA_ERR_INVALID with the sizes in the message.
 *   The first call on a device looks up the array's device address once
 *     (cudaGetSymbolAddress with that device current); make that first call
 *     before any stream capture.
 *   Every call shares the one array and leaves its last contents there;
 *     each call overwrites both work fields completely before reading them,
 *     so no clearing is needed.  Calls that overlap on the GPU (different
 *     streams, or different host threads) race on the array: serialise them. */
mglma_status mglma_dirac_apply_noalloc(mglma_ctx ctx, mglma_gauge g, mglma_op op, int nrhs, const double* in,
                                       double* out, mglma_prec compute, void* cuda_stream);

/* ---------------------------------------------------------------- block basis (Sec. 3, Sec. 4) */
/* Builds the chirality-split block basis of Eq. mg_basis:
 *   1. nv Gaussian start vectors drawn on the device from the counter-based
 *      generator (SplitMix64 keyed by (seed, tag 3), Box-Muller pairs);
 *   2. n_smooth minimal-residual steps on D v = 0 in FP64 (the paper uses
 *      exact low modes of Q and notes inexact ones work the same way);
 *   3. P_alpha theta_{B_y} v_c for every block y (sides block[4], each
 *      dividing L) and chirality alpha, orthonormalised per (block, alpha) --
 *      the unique factor with positive real R that Gram-Schmidt gives -- in
 *      FP64.
 * store: the copy the FP32 solvers read: MGLMA_FP64 or MGLMA_FP32 (FP32
 *   basis), or MGLMA_FP16 (one FP32 scale per (block, alpha, c)).  The FP64
 *   basis is always kept (FP64 R0/T0, coarse build, export).
 * Returns MGLMA_ERR_RANK when a vector's remaining norm falls below 1e-6 of
 * its starting norm inside a block (the paper assumes full rank, App.
 * chirality). */
mglma_status mglma_subspace_build(mglma_ctx ctx, mglma_gauge g, const int block[4], int nv, int n_smooth,
                                  uint64_t seed, mglma_prec store, mglma_subspace* out);
/* The same with the full set-up recipe: after the n_smooth MR steps each
 * vector takes n_cg conjugate-gradient steps on the normal equations of
 * D x = 0 (in cg_prec arithmetic, FP64 or FP32), which filters it towards the
 * low right singular vectors of D -- the low modes of Q (App. chirality) that
 * the paper's basis is built from.  mglma_subspace_build is this call with
 * n_cg = 0. */
/* lean_group > 0 selects the memory-lean set-up for large lattices: the
 * test vectors are stored in FP32 and relaxed lean_group at a time (MR and
 * CG in FP32, so cg_prec is ignored), the per-(block, chirality)
 * orthonormalisation runs in FP64 on chunks of blocks, and only the store
 * copy (MGLMA_FP32 or MGLMA_FP16) is kept -- no FP64 basis.  Peak device
 * memory is about 96 nv + 384 lean_group bytes per site, plus the stored
 * copy (48 nv for FP16, 96 nv for FP32) and a 1 GiB chunk buffer, instead of
 * about 670 nv.  FP64 R0 / T0 and the coarse build then read the stored
 * copy in FP64 arithmetic; the propagator pieces (which need the FP64 basis)
 * are refused.  0 = the standard FP64 set-up. */
typedef struct {
  int block[4];
  int nv;
  int n_smooth;
  int n_cg;
  int cg_prec;
  uint64_t seed;
  int store;
  int lean_group;
} mglma_subspace_params;
mglma_status mglma_subspace_create(mglma_ctx ctx, mglma_gauge g, const mglma_subspace_params* params,
                                   mglma_subspace* out);
/* Same from caller-provided test vectors (e.g. exact low modes, Sec. 3):
 * vecs = nv canonical spinors (host or device). */
mglma_status mglma_subspace_load(mglma_ctx ctx, mglma_gauge g, const int block[4], int nv, const double* vecs,
                                 mglma_prec store, mglma_subspace* out);
void mglma_subspace_free(mglma_subspace s);
mglma_status mglma_subspace_info(mglma_subspace s, int* nv, int Lb[4], int64_t* coarse_volume);
/* Exports the FP64 basis as complex128 [V1][2][nv][|B|][4][3] (spins of the
 * other chirality are zero); sites of a block in site-in-block order.  A lean
 * subspace exports its stored FP32 / FP16 copy (scale applied). */
mglma_status mglma_subspace_export(mglma_subspace s, double* phi);
/* R0 (Eq. res_mg): out[rhs][y][alpha nv + c] = sum_{x in B_y} phi^dag psi(x).
 * in: nrhs canonical spinors; out: nrhs canonical coarse fields.  compute:
 * MGLMA_FP64, MGLMA_FP32, or MGLMA_BF16 = the tensor-core path (tcgen05,
 * FP32 fields rounded to BF16, BF16 image of the basis, FP32 accumulation;
 * relative error of order 1e-3) for nv % 8 == 0, nv <= 32 and blocks of 64,
 * 128, ... 512 sites; MGLMA_ERR_INVALID otherwise, MGLMA_ERR_TIMEOUT if a
 * bounded wait of the kernel gave up. */
mglma_status mglma_restrict(mglma_ctx ctx, mglma_subspace s, int nrhs, const double* in, double* out,
                            mglma_prec compute, void* cuda_stream);
/* T0 (Eq. pro_mg): out(x) = sum_{alpha c} in[y(x)][alpha nv + c] phi(x).
 * in: nrhs canonical coarse fields; out: nrhs canonical spinors.  compute:
 * MGLMA_FP64, MGLMA_FP32, or MGLMA_BF16 = the tensor-core path (coarse
 * fields and the basis image in BF16, FP32 accumulation and output) for
 * nv % 8 == 0, nv <= 32 and blocks of 128, 256, 384 or 512 sites;
 * MGLMA_ERR_INVALID otherwise, MGLMA_ERR_TIMEOUT if a bounded wait of the
 * kernel gave up. */
mglma_status mglma_prolong(mglma_ctx ctx, mglma_subspace s, int nrhs, const double* in, double* out,
                           mglma_prec compute, void* cuda_stream);

/* ---------------------------------------------------------------- coarse operator (Sec. 2, Fig. A) */
/* Builds D1 = R0 D T0 in FP64 as the nine-slot stencil of dense
 * (2nv x 2nv) blocks; store selects the copy used by the solvers' coarse
 * applications: MGLMA_BF16 (FP32 accumulation), MGLMA_FP32 or MGLMA_FP64.
 * The FP64 operator is kept (export, FP64 coarse residuals) until
 * mglma_coarse_release_fp64.  With a lean subspace the operator is R0 D T0
 * of the stored FP32 / FP16 basis, computed in FP64 arithmetic. */
mglma_status mglma_coarse_build(mglma_ctx ctx, mglma_gauge g, mglma_subspace s, mglma_prec store,
                                mglma_coarse* out);
void mglma_coarse_free(mglma_coarse c);
/* Frees the FP64 copy of D1 when a low-precision copy exists (store BF16 or
 * FP32), e.g. to keep large lattices resident for serving; FP64 coarse
 * applications, export and the propagator pieces are refused afterwards.
 * When every coarse extent is even, the even-odd self-block inverses are
 * formed first (kept as their BF16 tensor-core image when the operator has
 * one, else in FP64). */
mglma_status mglma_coarse_release_fp64(mglma_coarse c);
mglma_status mglma_coarse_info(mglma_coarse c, int* nv, int Lb[4], int64_t* coarse_volume);
/* Exports the FP64 stencil as complex128 [9][V1][2nv][2nv]. */
mglma_status mglma_coarse_export(mglma_coarse c, double* dhat);
/* out = op(D1) in for nrhs canonical coarse fields; compute MGLMA_FP64 uses
 * the FP64 operator, MGLMA_FP32 the stored low-precision copy.  op:
 *   MGLMA_OP_D     D1
 *   MGLMA_OP_DDAG  D1^dag, applied as g5hat D1 g5hat (g5hat = +1 on the
 *                  alpha = 0 dofs, -1 on alpha = 1): D1 inherits
 *                  gamma5-hermiticity from D because the basis is split by
 *                  chirality (Sec. 2, App. chirality)
 *   MGLMA_OP_Q     Q1 = g5hat D1, the Hermitian coarse operator of Sec. 2
 *   MGLMA_OP_SCHUR / MGLMA_OP_SCHUR_Q
 *                  S_ee = D_ee - D_eo D_oo^-1 D_oe (or g5hat S_ee) of the
 *                  even-odd decomposition (sites of even y0 + y1 + y2 + y3):
 *                  reads the even sites of in, writes the even sites of out
 *                  and zero on the odd ones.  Every coarse extent must be
 *                  even; the first such call forms the self-block inverses
 *                  from the FP64 operator (which must be held).
 * MGLMA_OP_DDAGD is rejected with MGLMA_ERR_INVALID. */
mglma_status mglma_coarse_apply(mglma_ctx ctx, mglma_coarse c, mglma_op op, int nrhs, const double* in, double* out,
                                mglma_prec compute, void* cuda_stream);

/* ---------------------------------------------------------------- deeper levels (Sec. "Multigrid decompositions") */
/* Builds the operator of the next level of the nested block hierarchy,
 * D_{l+1} = R_l D_l T_l, from the level-l operator `parent` (a handle of
 * mglma_coarse_build for l = 1, or of this call).  For l >= 1 the paper's
 * restrictor of a coarse field psi_l on the level-l grid is
 *   (R_l psi_l)_{alpha c}(y) = sqrt(V_{l+1} / V_l) sum_{z in B_y} psi_{l, alpha c}(z)
 * (blocks of side block[mu] in level-l sites, each dividing the parent's
 * grid extent), and T_l = R_l^dag; the Hermitian Q_{l+1} = R_l Q_l T_l of the
 * paper equals g5hat D_{l+1} because R_l acts per (alpha, c).  D_{l+1} is
 * again a nine-slot stencil of (2nv x 2nv) blocks on the grid L_l / block
 * (same slot rules as D1 when an extent is 1 or 2) and every coarse call
 * (apply, export, info, free) accepts it; store as in mglma_coarse_build.
 * The parent's FP64 operator must still be held; the new handle refers to
 * the parent (free the children first).  A grid of one site is the LMA
 * limit of the hierarchy. */
mglma_status mglma_coarse_build_next(mglma_ctx ctx, mglma_coarse parent, const int block[4], mglma_prec store,
                                     mglma_coarse* out);
/* R_l and T_l between the grid of level l (the parent of `level`) and that
 * of `level` (level l+1 >= 2): in / out are nrhs canonical coarse fields of
 * the respective grids (complex128 [rhs][site][2nv], host or device), FP64
 * arithmetic.  MGLMA_ERR_INVALID for a level-1 handle (use mglma_restrict /
 * mglma_prolong there). */
mglma_status mglma_coarse_restrict(mglma_ctx ctx, mglma_coarse level, int nrhs, const double* in, double* out,
                                   void* cuda_stream);
mglma_status mglma_coarse_prolong(mglma_ctx ctx, mglma_coarse level, int nrhs, const double* in, double* out,
                                  void* cuda_stream);
/* The coarse-level pieces of the telescoping decomposition S = S_0 + ... +
 * S_{N-1} (Sec. "Multigrid decompositions", Eq. mglma:decomp) for nrhs
 * sources b: psi[l-1] = calT_l D_l^-1 calR_l b for l = 1 .. nlevels with
 * calR_l = R_{l-1} ... R_0 and calT_l = T_0 ... T_{l-1} (App. chirality:
 * calT_l Q_l^-1 calR_l gamma5 = calT_l D_l^-1 calR_l).  levels[0] is a
 * level-1 operator of g's basis and levels[k] the mglma_coarse_build_next
 * child of levels[k-1]; each D_l^-1 is solved to relative residual tol by
 * FP64 defect correction around FP32 GCR on that level's stored operator.
 * With x = D^-1 b from mglma_solve_batch: S_0 b = x - psi[0], S_l b =
 * psi[l-1] - psi[l], S_{N-1} b = psi[N-2] (N = nlevels + 1 levels in all).
 *   b: nrhs canonical spinors; psi: nlevels x nrhs canonical spinors
 *   ([level][rhs][site][spin][colour]); host or device. */
mglma_status mglma_pieces(mglma_ctx ctx, mglma_gauge g, const mglma_coarse* levels, int nlevels, int nrhs,
                          const double* b, double* psi, double tol, void* cuda_stream);

/* ---------------------------------------------------------------- exact coarsest level (Sec. "Exact estimator on the coarsest grid") */
/* Coarse matrices of gamma5 gamma_k with an open fine time index (Eq.
 * coarse:gamma):  Gam_k(x0) = calR gamma5 gamma_k P_{x0} calT on the grid of
 * `level` (calR, calT the compound transfers from the fine lattice), k = 1,
 * 2, 3.  They are block-diagonal over coarse sites: out receives complex128
 * [L0][V_c][2nv][2nv], block y of slice x0 (zero when block y does not meet
 * the fine time slice x0), host or device.  Level 1 computes them from the
 * basis (phi_i^dag gamma5 gamma_k phi_j summed over the block's sites on the
 * slice); deeper levels sum them over a block times V_{l+1} / V_l. */
mglma_status mglma_coarse_gamma5_gamma(mglma_ctx ctx, mglma_coarse level, int k, double* out);
/* Q_c^-1 of the Hermitian coarse operator Q_c = g5hat D_c of `level` as a
 * dense complex128 n x n matrix (n = V_c 2nv <= 16384, row index
 * site * 2nv + dof), formed in FP64 by Gauss-Jordan elimination with partial
 * pivoting on the device (n^3 complex multiply-adds; the level's FP64
 * operator must be held).  MGLMA_ERR_NUMERIC if Q_c is singular. */
mglma_status mglma_coarse_dense_inverse(mglma_ctx ctx, mglma_coarse level, double* out);
/* The exact estimator of the coarsest level's correlator (Eq. G_LL:exact):
 *   corr[x0][y0] = -(1 / (3 L1 L2 L3)) sum_{k=1}^{3} tr{Gam_k(y0) Q_c^-1 Gam_k(x0) Q_c^-1}
 *   G[t]         = (1 / L0) sum_{y0} corr[(t + y0) mod L0][y0]   (Eq. timetrans)
 * complex128, corr [L0][L0] and G [L0] (either may be NULL), host or device.
 * This is C_ll of the level's coarse propagator calT D_c^-1 calR (App.
 * chirality), averaged over the whole lattice with no noise; Q_c^-1 as in
 * mglma_coarse_dense_inverse (n <= 16384, at most 80 dofs per site).  Sums
 * run in a fixed order. */
mglma_status mglma_exact_correlator(mglma_ctx ctx, mglma_coarse level, double* corr, double* G);

/* ---------------------------------------------------------------- sources (Sec. 5) */
typedef enum { MGLMA_SOURCE_Z2 = 0, MGLMA_SOURCE_Z4 = 1, MGLMA_SOURCE_POINT = 2 } mglma_source_kind;
/* Writes nrhs canonical sources to out (host or device):
 *   Z2: every real component +-1 (imaginary 0); Z4: (+-1 +- i)/sqrt(2), the
 *     noise the paper's stochastic estimator uses.  Component (spin s,
 *     colour c) of RHS r at site x takes draw n = ((first + r) V + x) 12 +
 *     3 s + c of the counter-based stream key = mix64(mix64(seed) ^ 2)
 *     (mix64 = SplitMix64 output function): bit 63 of mix64(key + n) is the
 *     real sign, bit 62 the imaginary sign.
 *   POINT: a unit vector at site point_sites[r], spin-colour point_sc[r]
 *     (host arrays of nrhs entries).
 * t_slice >= 0 keeps only the time slice x0 = t_slice (time dilution,
 * Sec. 5); -1 keeps the whole lattice. */
mglma_status mglma_sources(mglma_ctx ctx, const mglma_lattice* lat, int kind, int nrhs, uint64_t seed,
                           int64_t first, const int64_t* point_sites, const int* point_sc, int t_slice, double* out,
                           void* cuda_stream);

/* ---------------------------------------------------------------- contractions (Sec. 5) */
/* Time-slice contraction of the stochastic estimator, Eq. C_stoch2: for each
 * RHS r and time slice x0,
 *   out[r][x0] = -(1 / (3 L1 L2 L3)) sum_{k=1}^{3} sum_{x in slice x0}
 *                < a[r][k-1](x), gamma5 gamma_k b[r](x) >
 * with <u, v> = sum over spin and colour of conj(u) v.  For a noise source
 * eta on slice y0, a[r][k-1] = S_j gamma5 gamma_k^dag eta and b[r] = S_i eta
 * give G_ij(x0, y0) (gamma_k is Hermitian in the chiral basis, so the
 * sources are mglma_gamma5_gamma of eta).
 *   a: nrhs x 3 canonical spinors ([r][k-1][site][spin][colour]);
 *   b: nrhs canonical spinors; out: nrhs x L0 complex128 ([r][x0]).
 * Host or device pointers.  Sums in FP64 in a fixed order (one CTA per RHS
 * and time slice), so the result does not depend on the batch. */
mglma_status mglma_contract(mglma_ctx ctx, const mglma_lattice* lat, int nrhs, const double* a, const double* b,
                            double* out, void* cuda_stream);
/* out = gamma5 gamma_k in for nrhs canonical spinors, k = 1, 2, 3 (chiral
 * basis: gamma5 gamma_k = [[0, -i sigma_k], [-i sigma_k, 0]]); the sources
 * of the a fields of mglma_contract.  in and out must differ. */
mglma_status mglma_gamma5_gamma(mglma_ctx ctx, const mglma_lattice* lat, int k, int nrhs, const double* in,
                                double* out, void* cuda_stream);

/* ---------------------------------------------------------------- solves (Sec. 2, Sec. 5) */
typedef enum {
  MGLMA_SOLVER_CGNE = 0,    /* FP64 CG on D^dag D x = D^dag b: the plain method */
  MGLMA_SOLVER_MG = 1,      /* FP64 defect correction around FP32 flexible GCR
                               preconditioned by the coarse-grid correction
                               T0 D1^-1 R0 plus MR smoothing */
  MGLMA_SOLVER_CGNE_EO = 2  /* the plain method on the even-odd preconditioned
                               operator: FP64 CG on S^dag S x_e = S^dag b_e' with
                               S = A_ee - H_eo A_oo^-1 H_oe (A the clover term,
                               H the hops), b_e' = b_e - H_eo A_oo^-1 b_o, then
                               x_o = A_oo^-1 (b_o - H_oe x_e) and FP64 defect
                               correction on the true residual of D; every
                               lattice extent must be even */
} mglma_solver;

/* Solver of the coarse system inside the MG preconditioner. */
typedef enum {
  MGLMA_COARSE_GCR = 0,       /* restarted GCR(16) on D1 */
  MGLMA_COARSE_MINRES = 1,    /* MINRES on the Hermitian Q1 = g5hat D1 (Sec. 2),
                                 solving Q1 e = g5hat b: a three-term Lanczos
                                 recurrence, no restarts, about a third of the
                                 vector traffic of GCR per iteration */
  MGLMA_COARSE_MINRES_EO = 2  /* MINRES on g5hat S_ee, the even-odd (Schur)
                                 preconditioned coarse operator S_ee = D_ee -
                                 D_eo D_oo^-1 D_oe on the even coarse sites, the
                                 odd sites by back-substitution (the paper's
                                 coarse solves use the even-odd preconditioned
                                 coarse operator, Sec. "Comparison of the
                                 cost"); the default.  It runs on the BF16
                                 tensor-core operator; without one, on a coarse
                                 grid with an odd extent, or when the set-up
                                 cannot be formed (FP64 operator released before
                                 it was), it runs as MGLMA_COARSE_MINRES.  The self-block inverses
                                 are formed from the FP64 operator on first use
                                 (or by mglma_coarse_release_fp64, before it
                                 frees the FP64 operator) */
} mglma_coarse_solver;

typedef struct {
  int method;           /* mglma_solver */
  double tol;           /* target FP64 ||b - D x|| / ||b|| (e.g. 1e-10) */
  int max_iter;         /* cap on iterations (CGNE) / inner FGCR iterations (MG) */
  int gcr_m;            /* FGCR restart length (MG) */
  int nu;               /* MR smoothing steps after the coarse correction (MG) */
  double inner_tol;     /* relative reduction asked of each FP32 cycle (MG) */
  double coarse_tol;    /* relative tolerance of the preconditioner's coarse solve */
  int coarse_max_iter;  /* cap on coarse iterations per preconditioner call */
  int check_every;      /* host polls residual norms every this many iterations */
  int max_batch;        /* RHS solved together (0: as many as 70 % of the memory the
                           context can use allows -- free HBM plus its pool's idle
                           cached blocks -- at most 64, split into equal batches) */
  int coarse_solver;    /* mglma_coarse_solver (MG) */
  int autotune;         /* MG: 1 = the first lockstep batch of each (lattice, RHS
                           bucket) tunes the stencil and coarse tile shapes
                           (mglma_autotune) before it runs; 0 = use the table as
                           it stands (defaults where empty) */
  int graph;            /* MG: 1 = every FGCR iteration after the first runs as one
                           CUDA graph -- fine stencil, restriction, the coarse
                           MINRES loop as a device-side conditional node that
                           stops when every RHS converged or the cycle cap is
                           reached, prolongation, MR smoothing, orthogonalisation
                           and update -- with one host read of the convergence
                           mask per iteration (not while mglma_profile is on);
                           0 = launches issued from the host */
} mglma_solve_params;

typedef struct {
  int iterations;              /* CGNE iterations / FGCR iterations summed over cycles */
  int outer;                   /* FP64 defect-correction cycles (MG) */
  long long coarse_iterations; /* coarse-solver iterations (MG) */
  double residual;             /* final FP64 ||b - D x|| / ||b|| */
  int converged;               /* 1 if residual <= tol */
  int batch;                   /* RHS in the lockstep batch this RHS was solved in
                                  (mglma_solve_batch); 0 from mglma_serve */
} mglma_solve_stats;

/* Fills *p with the library defaults for `method`: tol 1e-10; MG: gcr_m 4,
 * nu 7, inner_tol 3e-6, coarse_tol 0.02, coarse_max_iter 48 (whole cycles
 * of 12 MINRES iterations), coarse_solver MINRES_EO, check_every 1, max_batch 0,
 * autotune 1, graph 1; CGNE: max_iter 100000, check_every 20, autotune 0,
 * graph 0. */
void mglma_solve_params_default(mglma_solve_params* p, int method);

/* Solves D x = b (x = S b, the propagator of Sec. 2 applied to b) for
 * ngroups groups of right-hand sides; group g holds group_nrhs[g] canonical
 * spinors, the groups stored back to back in b and x.  Uneven groups are
 * merged: all RHS run as lockstep batches of up to max_batch RHS (one launch
 * of every kernel covers the whole batch).  Every RHS follows its own
 * recurrence with its own scalars and convergence mask, so its result does
 * not depend on the batch it is in.  coarse may be NULL for MGLMA_SOLVER_CGNE.
 * x_coarse (nullable): also returns the coarse-space piece
 *   psi1 = T0 D1^-1 R0 b (S1 b of Sec. 2 via App. chirality), with D1^-1
 *   solved to tol by FP64 defect correction; S0 b = x - psi1.
 * stats (nullable): one entry per RHS.
 * Returns MGLMA_ERR_NOT_CONVERGED (best iterate in x) if any RHS misses tol. */
mglma_status mglma_solve_batch(mglma_ctx ctx, mglma_gauge g, mglma_coarse coarse, const mglma_solve_params* params,
                               int ngroups, const int* group_nrhs, const double* b, double* x, double* x_coarse,
                               mglma_solve_stats* stats, void* cuda_stream);

/* ---------------------------------------------------------------- serving */
/* A resident lattice the server solves on: gauge field and its coarse
 * operator (the coarse operator's basis must belong to the same gauge). */
typedef struct {
  mglma_gauge gauge;
  mglma_coarse coarse;
} mglma_serve_lattice;

/* One solve request: nrhs canonical sources b for lattice `lattice`,
 * solutions written to x (each host or device).  arrival is the time on the
 * serving clock (seconds since mglma_serve started) at which the request was
 * made; latency is measured from it. */
typedef struct {
  int lattice;
  int nrhs;
  const double* b;
  double* x;
  double arrival;
  int64_t id;
} mglma_request;

/* Called by the server to pull requests: fill *out and return 1 when a
 * request with arrival <= now exists, return 0 when none has arrived yet, -1
 * when the stream has ended. */
typedef int (*mglma_request_fn)(void* user, double now, mglma_request* out);
/* Called once per request when all its RHS are done (or it was rejected):
 * status, latency (completion - arrival, seconds) and one stats entry per
 * RHS.  x holds the solutions when status is MGLMA_OK. */
typedef void (*mglma_done_fn)(void* user, const mglma_request* req, mglma_status status, double latency,
                              const mglma_solve_stats* per_rhs);

typedef struct {
  int nlattices;                        /* 1..8 */
  const mglma_serve_lattice* lattices;
  int max_slots;                        /* RHS in flight per lattice, upper bound */
  double hbm_fraction;                  /* share of the HBM free at start the slots may take;
                                           lattices split it in proportion to their volume */
  mglma_solve_params params;            /* MGLMA_SOLVER_MG parameters (tol, gcr_m, nu, ...) */
} mglma_serve_config;

typedef struct {
  long long requests, rhs, rejected;
  double wall_s, solves_per_s;          /* RHS completed per second of serving */
  double p50_s, p99_s, mean_s, max_s;   /* request latency, arrival to completion */
  int slots[8];                         /* slots granted per lattice */
  double slot_bytes[8];                 /* device bytes per slot */
} mglma_serve_stats;

/* Serves a stream of solve requests with continuous batching.  Per lattice
 * the server sizes a set of RHS slots from free HBM (admission by memory),
 * keeps gauge, basis and coarse operator resident, and runs the mixed
 * multigrid solve of mglma_solve_batch on all occupied slots together.
 * Requests are admitted RHS by RHS as slots free up (a request larger than
 * the slot count is spread over time); a RHS joins and leaves at restart
 * boundaries of the inner FGCR, so requests that arrive while others run
 * share the same kernel launches, and every RHS follows the recurrence it
 * would follow alone.  Host sources and solutions pass one RHS at a time
 * through a staging spinor per lattice.  Lattices are served in turn, one
 * restart cycle each.  Malformed requests come back with MGLMA_ERR_INVALID. */
mglma_status mglma_serve(mglma_ctx ctx, const mglma_serve_config* cfg, mglma_request_fn next, mglma_done_fn done,
                         void* user, mglma_serve_stats* out);

/* ---------------------------------------------------------------- autotuning */
/* Times the candidate RHS tile widths for nrhs right-hand sides with CUDA
 * events and keeps the fastest in the context, per lattice volume (used by
 * every later call on a lattice of that volume with an RHS count in the same
 * power-of-two bucket):
 *   kernel 0: tile shape of the FP32 stencil, needs g: NR right-hand sides
 *     per thread (1, 2, 4) and RW RHS tiles per 128-thread CTA (1, 2, 4;
 *     a CTA then covers 128 / RW sites), coded NR + 16 (RW - 1) (NR = 4 only
 *     with RW = 1); or the staged-tile kernel, 32 sites x NRT RHS per CTA
 *     with each site's links and clover staged once in shared memory, coded
 *     64 + NRT (NRT = 4, 8, 16);
 *   kernel 1: RHS per tile of the tensor-core coarse stencil (8, 16, 32), needs c.
 * g or c may be NULL to skip that kernel. */
mglma_status mglma_autotune(mglma_ctx ctx, mglma_gauge g, mglma_coarse c, int nrhs);
/* Sets the choice for kernel / the RHS bucket of nrhs by hand (codes as
 * above); MGLMA_ERR_INVALID for an unknown kernel or choice. */
mglma_status mglma_autotune_set(mglma_ctx ctx, int kernel, int nrhs, int choice);
/* The tuned choice (0 if none) and its time in ms for kernel / nrhs. */
mglma_status mglma_autotune_get(mglma_ctx ctx, int kernel, int nrhs, int* choice, double* ms);
/* Text cache of the tuned table, one line per entry (GPU name, kernel, RHS
 * bucket, lattice volume -- 0 for entries set by mglma_autotune_set --,
 * choice, ms); entries of other GPUs are ignored on load.  When the
 * environment variable MGLMA_TUNE_CACHE names a file, mglma_create loads it
 * (if it exists) and the solver saves the table there after each automatic
 * tuning. */
mglma_status mglma_autotune_save(mglma_ctx ctx, const char* path);
mglma_status mglma_autotune_load(mglma_ctx ctx, const char* path);

/* Debug export of the integer tables the kernels compute on the fly:
 * nbr[V][8] (hop slots +0..+3, -0..-3) and block_of_site[V] for the given
 * block sides (block may be NULL to skip it).  Host pointers. */
mglma_status mglma_debug_tables(mglma_gauge g, const int block[4], int32_t* nbr, int32_t* block_of_site);

#ifdef __cplusplus
}
#endif
#endif /* MGLMA_H */
