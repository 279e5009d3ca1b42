// Block basis handle and coarse-operator handle (shared by subspace.cu,
// coarse.cu, multigrid solver and C ABI).
#pragma once
#include "internal.h"

namespace mglma {

struct BlockGeo {
  int L[4], b[4], Lb[4];
  int64_t V, V1;
  int nB;
};
BlockGeo make_blockgeo(const int L[4], const int b[4]);

}  // namespace mglma

struct mglma_subspace_s {
  mglma_ctx ctx = nullptr;
  mglma_gauge gauge = nullptr;
  int nv = 0;
  int store = MGLMA_FP32;
  mglma::BlockGeo geo;
  double2* phi64 = nullptr;  // [V1][2Nv][6][nB]
  float4* phi32 = nullptr;   // [V1][2Nv][3][nB]
  uint2* phi16 = nullptr;    // [V1][2Nv][3][nB], halves
  float* scale16 = nullptr;  // [V1][2Nv]
  bool lean = false;         // built without an FP64 copy (phi64 stays NULL)
  uint16_t* rt_img = nullptr;  // cache: BF16 image of the basis for the tensor-core R0 (transfer_tc.cu), built on first use
  uint16_t* pt_img = nullptr;  // cache: BF16 image of the basis for the tensor-core T0, built on first use
  int* rt_err = nullptr;       // the error flag of both tensor-core transfer kernels
};

struct mglma_coarse_s {
  mglma_ctx ctx = nullptr;
  mglma_subspace sub = nullptr;
  int nv = 0, n2 = 0;
  int store = MGLMA_BF16;
  mglma::BlockGeo geo;
  double2* A64 = nullptr;        // [V1][9][n2 (j)][n2 (i)] column-major blocks, FP64 master (optional)
  float2* A32 = nullptr;         // same layout, FP32
  __nv_bfloat162* A16 = nullptr; // same layout, BF16 (re, im)
  uint16_t* Aimg = nullptr;      // BF16 tensor-core image, see coarse_tc.cu
  int* tc_err = nullptr;         // device error flag of the tensor-core kernel
  double2* tc_dpart = nullptr;   // per-CTA partials of the epilogue dot ([CTA][RHS])
  unsigned* tc_dcount = nullptr; // its ticket
  // level of the hierarchy: 1 for D1 = R0 D T0 (geo: fine lattice -> block
  // grid); l >= 2 for D_l = R_{l-1} D_{l-1} T_{l-1}, built by aggregation
  // from `parent` (geo: level l-1 grid -> level l grid, geo.V = V_{l-1},
  // geo.V1 = V_l; sub is the level-1 basis of the chain)
  int level = 1;
  const mglma_coarse_s* parent = nullptr;
  // even-odd preconditioning (coarse_eo.cu), built on first use: inverses of
  // the self blocks D_yy (FP64, layout of one slot of A64) and their BF16
  // tensor-core image (one slot per site)
  double2* Sinv64 = nullptr;
  uint16_t* Sinv_img = nullptr;
  // D_oo^-1 D_oe: per odd site (half-lattice index u) the eight hop slots
  // multiplied by the inverse self block, as a BF16 tensor-core image
  // ([u][8 slots]); with it S_ee takes two tensor-core launches
  uint16_t* Ahat_img = nullptr;
};

namespace mglma {

mglma_status restrict_fine(mglma_ctx ctx, const mglma_subspace_s* S, const Spinor& in, void* out_coarse,
                           cudaStream_t s);
mglma_status prolong_coarse(mglma_ctx ctx, const mglma_subspace_s* S, const void* in_coarse, Spinor& out,
                            bool accumulate, cudaStream_t s);
// n_smooth MR steps on D v = 0 in the precision of v
mglma_status mr_smooth(mglma_ctx ctx, const mglma_gauge_s* G, Spinor& v, int n_smooth, cudaStream_t s);

// coarse fields: internal [rhs][V1][n2] float2 (FP32) or double2 (FP64)
mglma_status coarse_to_canonical(mglma_ctx ctx, const void* c, int prec, size_t ncplx, double* canon,
                                 cudaStream_t s);
mglma_status coarse_from_canonical(mglma_ctx ctx, const double* canon, size_t ncplx, void* c, int prec,
                                   cudaStream_t s);
// dst = scale_r src (+ dst when accumulate) on coarse fields of `per` complex per RHS
mglma_status coarse_scale_convert(mglma_ctx ctx, const void* src, int sprec, void* dst, int dprec,
                                  const double* scale, size_t per, int nrhs, bool accumulate, cudaStream_t s);
// tensor-core path (coarse_tc.cu)
bool coarse_tc_supported(int n2);
mglma_status coarse_tc_image(mglma_ctx ctx, mglma_coarse_s* C, cudaStream_t s);
// scratch: B images of X (coarse_tc_scratch_bytes); NULL or too small ->
// allocated for the call (refused inside a graph capture)
mglma_status coarse_apply_tc(mglma_ctx ctx, const mglma_coarse_s* C, const float2* X, float2* Y, int nrhs,
                             int mode, void* scratch, size_t scratch_bytes, cudaStream_t s);
size_t coarse_tc_scratch_bytes(const mglma_coarse_s* C, int nrhs);
int coarse_tc_default_nt(int nrhs);
mglma_status coarse_tc_check(mglma_coarse_s* C, cudaStream_t s);
// Y = Dhat X for nrhs coarse fields; prec of X/Y: FP64 (FP64 operator) or FP32
// (FP32 or BF16 operator as stored).  mode bit 0 applies gamma5hat to X, bit 1
// to Y: 0 Dhat, 2 Qhat = gamma5hat Dhat, 3 gamma5hat Dhat gamma5hat = Dhat^dag
// (gamma5hat-hermiticity, inherited from D by the chirality-split basis).
constexpr int CMODE_D = 0, CMODE_Q = 2, CMODE_DDAG = 3;
// scratch (optional): work space of the tensor-core path, see coarse_apply_tc
mglma_status coarse_apply(mglma_ctx ctx, const mglma_coarse_s* Cc, const void* X, void* Y, int nrhs, int prec,
                          int mode, cudaStream_t s, void* scratch = nullptr, size_t scratch_bytes = 0);
// ---- even-odd (Schur) preconditioning of the coarse operator (coarse_eo.cu)
// Needs every coarse extent even (then every hop joins opposite parities).
// Half-lattice fields: [rhs][V1 / 2][n2], site y of a parity at index y >> 1.
mglma_status coarse_eo_setup(mglma_ctx ctx, mglma_coarse_s* C, cudaStream_t s);
// Y_e = S_ee X_e (mode bit 1: gamma5hat S_ee, the Hermitian form) with
// S_ee = D_ee - D_eo D_oo^-1 D_oe; FP32 fields use the tensor cores when the
// operator has its BF16 image, FP64 fields the FP64 operator
// whether coarse_schur_apply can return <X_r, Y_r> per RHS (dot_out) from
// its last launch: FP32 on the tensor cores, one RHS tile
bool coarse_schur_dot_ok(mglma_ctx ctx, const mglma_coarse_s* C, int nrhs, int prec);
// x_imaged (with dot_out only): the scratch's first half already holds the
// image of X_e (coarse_x_image_half / minres_update_image)
mglma_status coarse_schur_apply(mglma_ctx ctx, const mglma_coarse_s* C, const void* Xe, void* Ye, int nrhs, int prec,
                                int mode, void* scratch, size_t scratch_bytes, cudaStream_t s,
                                double2* dot_out = nullptr, bool x_imaged = false);
// b_e' = b_e - D_eo D_oo^-1 b_o from a full field b; x (full) from x_e and b:
// x_o = D_oo^-1 (b_o - D_oe x_e)
mglma_status coarse_eo_prepare(mglma_ctx ctx, const mglma_coarse_s* C, const void* b, void* be, int nrhs, int prec,
                               void* scratch, size_t scratch_bytes, cudaStream_t s);
mglma_status coarse_eo_reconstruct(mglma_ctx ctx, const mglma_coarse_s* C, const void* b, const void* xe, void* x,
                                   int nrhs, int prec, void* scratch, size_t scratch_bytes, cudaStream_t s);
// Y (full field) = S_ee X on the even sites, zero on the odd ones (the C ABI's
// MGLMA_OP_SCHUR / _Q); forms the even-odd set-up on first use
mglma_status coarse_schur_full(mglma_ctx ctx, mglma_coarse_s* C, const void* X, void* Y, int nrhs, int prec,
                               int mode, cudaStream_t s);
// R0 on the tensor cores (transfer_tc.cu): FP32 fine fields in, FP32 coarse
// [rhs][V1][2Nv] out, BF16 operands (basis imaged on first use); needs
// Nv % 8 == 0, Nv <= 32, 64 | |B| <= 512.  restrict_tc_check reports a
// bounded wait that gave up.
bool restrict_tc_supported(const mglma_subspace_s* S);
mglma_status restrict_tc(mglma_ctx ctx, mglma_subspace_s* S, const Spinor& in, void* out, cudaStream_t s);
mglma_status restrict_tc_check(const mglma_subspace_s* S, cudaStream_t s);
// T0 on the tensor cores: FP32 coarse [rhs][V1][2Nv] in, FP32 fine fields
// out (overwritten), BF16 operands; needs Nv % 8 == 0, Nv <= 32,
// 128 | |B| <= 512.  Its timeouts are reported by restrict_tc_check too.
bool prolong_tc_supported(const mglma_subspace_s* S);
mglma_status prolong_tc(mglma_ctx ctx, mglma_subspace_s* S, const void* in_coarse, Spinor& out, cudaStream_t s);
// scratch the FP32 (tensor-core) even-odd calls need for nrhs RHS
size_t coarse_eo_scratch_bytes(const mglma_coarse_s* C, int nrhs);
// one tensor-core launch on half-lattice fields (coarse_tc.cu): Y = sign *
// sum over slots d_lo..d_hi, hop slots reading Xhop, the self slot reading
// Xself (with the self-block image Aself when given), for the sites of
// parity par; mode bit 0 applies gamma5hat to both inputs, bit 1 to Y.  The
// B images go to scratch (hop input) and scratch + one half image (self
// input); self_image (nullable) is an image of the self input an earlier
// launch with the same RHS count and mode bit 0 left, used instead of writing
// one; Ahop (nullable) replaces the hop slots with an eight-slot image
// indexed by the half-lattice index of the output site; dot_out (nullable,
// one RHS tile only) receives <dotX_r, Y_r> per RHS, taken in the epilogue;
// hop_imaged: the scratch's first half already holds the image of Xhop (mode
// bit 0 clear), so no image pass runs for it
mglma_status coarse_tc_eo_launch(mglma_ctx ctx, const mglma_coarse_s* C, const float2* Xhop, const float2* Xself,
                                 float2* Y, int nrhs, int mode, int par, int d_lo, int d_hi, const uint16_t* Aself,
                                 float sign, void* scratch, cudaStream_t s, const void* self_image = nullptr,
                                 const uint16_t* Ahop = nullptr, const float2* dotX = nullptr,
                                 double2* dot_out = nullptr, bool hop_imaged = false);
// RHS tile width of the tensor-core coarse launches for nrhs RHS
int coarse_tc_nt(mglma_ctx ctx, const mglma_coarse_s* C, int nrhs);
// the B-operand image (no gamma5hat) of a FP32 half-lattice field X into
// image (the first half of the even-odd scratch), as the Schur apply's first
// launch would write it
mglma_status coarse_x_image_half(mglma_ctx ctx, const mglma_coarse_s* C, const void* X, int nrhs, void* image,
                                 cudaStream_t s);
// minres_update on FP32 half-lattice fields that also writes the image of
// the scaled z (the next Lanczos vector) into image, as coarse_x_image_half
mglma_status minres_update_image(mglma_ctx ctx, const mglma_coarse_s* C, const double* cf, int stride, const Vec& v,
                                 const Vec& w1, const Vec& w2, Vec& wn, Vec& x, Vec& z, void* image, cudaStream_t s);
size_t coarse_tc_half_image_bytes(const mglma_coarse_s* C, int nrhs);
mglma_status coarse_tc_image_blocks(mglma_ctx ctx, const double2* A64, int64_t V1, int n2, int nslots,
                                    uint16_t** img, cudaStream_t s);

// Gam_k on level 1 (Eq. coarse:gamma with an open time index): out[y][t][i][j],
// t < b[0] the block's local time slice, FP64
mglma_status coarse_gamma_level1(mglma_ctx ctx, const mglma_subspace_s* S, int k, double2* out, cudaStream_t s);
// the copy the FP32 solvers read (FP32, BF16 tensor-core image or BF16 plain)
// from the FP64 master A64
mglma_status coarse_store_copies(mglma_ctx ctx, mglma_coarse_s* Cc, int store, cudaStream_t s);
// inner-level transfers between the grids of Cc->parent (level l-1) and Cc
// (level l), FP64 or FP32 internal coarse fields [rhs][V][n2]:
//   restrict: out(y) = sqrt(V_l / V_{l-1}) sum_{z in B_y} in(z)
//   prolong:  out(z) = sqrt(V_l / V_{l-1}) in(y(z)) (+ out when accumulate)
mglma_status restrict_level(mglma_ctx ctx, const mglma_coarse_s* Cc, const void* in, void* out, int nrhs, int prec,
                            cudaStream_t s);
mglma_status prolong_level(mglma_ctx ctx, const mglma_coarse_s* Cc, const void* in, void* out, int nrhs, int prec,
                           bool accumulate, cudaStream_t s);

}  // namespace mglma
