// Time-slice contractions of the stochastic estimator (Sec. 5, Eq. C_stoch2)
// and the gamma5 gamma_k sources they need.
//
// For one noise source eta on time slice y0 the estimator of the isovector
// vector correlator between levels i and j is
//   G_ij(x0, y0) = -(1 / (3 L^3)) sum_{k=1}^{3} sum_{x in slice x0}
//                  < (S_j gamma5 gamma_k^dag eta)(x), gamma5 gamma_k (S_i eta)(x) >
// (<u, v> = sum over spin and colour of conj(u) v).  mglma_contract takes the
// solved fields a_k = S_j gamma5 gamma_k^dag eta (k = 1, 2, 3) and
// b = S_i eta and returns G for every x0; mglma_gamma5_gamma makes the
// sources gamma5 gamma_k eta (gamma_k is Hermitian in the chiral basis).
//
// Chiral basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] and
// gamma5 = diag(1, 1, -1, -1), so gamma5 gamma_k = [[0, -i sigma_k],
// [-i sigma_k, 0]]: the upper spin pair of gamma5 gamma_k b is -i sigma_k
// times the lower pair of b, and vice versa.
//
// One CTA per (RHS, time slice) walks the slice's sites in a fixed order and
// sums in FP64 with a fixed tree, so results do not depend on timing or on
// how RHS are batched.  Each site reads four canonical spinors once (HBM
// bound at about 768 B per site per RHS).
#include <string>

#include "internal.h"

namespace mglma {

// w = -i sigma_k (u0, u1) for one colour
__device__ __forceinline__ void minus_i_sigma(int k, double2 u0, double2 u1, double2& w0, double2& w1) {
  // -i (x + i y) = y - i x
  auto mi = [](double2 z) { return make_double2(z.y, -z.x); };
  if (k == 1) {  // sigma_1 (u0, u1) = (u1, u0)
    w0 = mi(u1);
    w1 = mi(u0);
  } else if (k == 2) {  // sigma_2 (u0, u1) = (-i u1, i u0); -i sigma_2 = (-u1, u0)
    w0 = make_double2(-u1.x, -u1.y);
    w1 = u0;
  } else {  // sigma_3 (u0, u1) = (u0, -u1)
    w0 = mi(u0);
    w1 = make_double2(-mi(u1).x, -mi(u1).y);
  }
}

// psi[spin][colour] of one site of a canonical spinor: 12 double2
__device__ __forceinline__ void load_site(const double2* __restrict__ f, double2 v[12]) {
#pragma unroll
  for (int i = 0; i < 12; ++i) v[i] = __ldg(f + i);
}

// out[r][x0] = -(1/(3 L^3)) sum_k sum_{x in x0} <a[r][k-1](x), gamma5 gamma_k b[r](x)>
__global__ void __launch_bounds__(256) contract_kernel(const double2* __restrict__ a, const double2* __restrict__ b,
                                                       int64_t V, int64_t slice, double scale,
                                                       double2* __restrict__ out) {
  const int x0 = blockIdx.x, r = blockIdx.y, L0 = gridDim.x;
  double sr = 0.0, si = 0.0;
  for (int64_t s = threadIdx.x; s < slice; s += 256) {
    const int64_t site = (int64_t)x0 * slice + s;
    double2 bv[12];
    load_site(b + ((size_t)r * V + site) * 12, bv);
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
      double2 av[12];
      load_site(a + (((size_t)r * 3 + (k - 1)) * V + site) * 12, av);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double2 g[4];
        minus_i_sigma(k, bv[6 + c], bv[9 + c], g[0], g[1]);  // upper = -i sigma_k b_lower
        minus_i_sigma(k, bv[c], bv[3 + c], g[2], g[3]);      // lower = -i sigma_k b_upper
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          const double2 u = av[3 * sp + c], w = g[sp];
          sr += u.x * w.x + u.y * w.y;
          si += u.x * w.y - u.y * w.x;
        }
      }
    }
  }
  __shared__ double shr[256], shi[256];
  shr[threadIdx.x] = sr;
  shi[threadIdx.x] = si;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      shr[threadIdx.x] += shr[threadIdx.x + h];
      shi[threadIdx.x] += shi[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(size_t)r * L0 + x0] = make_double2(scale * shr[0], scale * shi[0]);
}

// out = gamma5 gamma_k in, canonical spinors, one thread per (site, colour)
__global__ void gamma5_gamma_kernel(const double2* __restrict__ in, double2* __restrict__ out, int64_t n, int k) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (rhs * V + site) * 3 + c
  if (t >= n) return;
  const int64_t sv = t / 3;
  const int c = (int)(t % 3);
  const double2* p = in + sv * 12;
  double2* q = out + sv * 12;
  double2 w0, w1, w2, w3;
  minus_i_sigma(k, p[6 + c], p[9 + c], w0, w1);
  minus_i_sigma(k, p[c], p[3 + c], w2, w3);
  q[c] = w0;
  q[3 + c] = w1;
  q[6 + c] = w2;
  q[9 + c] = w3;
}

static mglma_status lattice_volume(const mglma_lattice* lat, int64_t* V, const char* who) {
  *V = 1;
  for (int m = 0; m < 4; ++m) {
    if (lat->L[m] < 1 || lat->L[m] > 4096) return fail(MGLMA_ERR_INVALID, std::string(who) + ": bad extent");
    *V *= lat->L[m];
  }
  return MGLMA_OK;
}

}  // namespace mglma

using namespace mglma;

extern "C" mglma_status mglma_contract(mglma_ctx ctx, const mglma_lattice* lat, int nrhs, const double* a,
                                       const double* b, double* out, void* cuda_stream) {
  if (!ctx || !lat || !a || !b || !out) return fail(MGLMA_ERR_INVALID, "contract: NULL argument");
  if (nrhs < 0) return fail(MGLMA_ERR_INVALID, "contract: nrhs < 0");
  int64_t V = 0;
  MG_CHECK(lattice_volume(lat, &V, "contract"));
  if (nrhs == 0) return MGLMA_OK;
  if (nrhs > 65535) return fail(MGLMA_ERR_INVALID, "contract: at most 65535 RHS per call");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, cuda_stream);
  const int64_t slice = V / lat->L[0];
  const size_t bb = (size_t)nrhs * V * 24 * sizeof(double);
  const size_t ob = (size_t)nrhs * lat->L[0] * 2 * sizeof(double);
  Staged ia, ib, o;
  MG_CHECK(stage_in(ctx, a, 3 * bb, s, ia));
  MG_CHECK(stage_in(ctx, b, bb, s, ib));
  MG_CHECK(stage_out_alloc(ctx, out, ob, s, o));
  {
    // algorithmic traffic: four spinors per site and RHS read once
    ProfScope ps(ctx, K_CONTRACT, s, 4.0 * (double)bb, 144.0 * (double)V * nrhs);
    contract_kernel<<<dim3((unsigned)lat->L[0], (unsigned)nrhs, 1), 256, 0, s>>>(
        (const double2*)ia.dev, (const double2*)ib.dev, V, slice, -1.0 / (3.0 * (double)slice), (double2*)o.dev);
  }
  MG_LAUNCH_CHECK();
  MG_CHECK(stage_out_finish(out, ob, s, o));
  return MGLMA_OK;
}

extern "C" mglma_status mglma_gamma5_gamma(mglma_ctx ctx, const mglma_lattice* lat, int k, int nrhs,
                                           const double* in, double* out, void* cuda_stream) {
  if (!ctx || !lat || !in || !out) return fail(MGLMA_ERR_INVALID, "gamma5_gamma: NULL argument");
  if (k < 1 || k > 3) return fail(MGLMA_ERR_INVALID, "gamma5_gamma: k must be 1, 2 or 3");
  if (nrhs < 0) return fail(MGLMA_ERR_INVALID, "gamma5_gamma: nrhs < 0");
  if (in == out) return fail(MGLMA_ERR_INVALID, "gamma5_gamma: in and out must differ");
  int64_t V = 0;
  MG_CHECK(lattice_volume(lat, &V, "gamma5_gamma"));
  if (nrhs == 0) return MGLMA_OK;
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, cuda_stream);
  const size_t bytes = (size_t)nrhs * V * 24 * sizeof(double);
  Staged i, o;
  MG_CHECK(stage_in(ctx, in, bytes, s, i));
  MG_CHECK(stage_out_alloc(ctx, out, bytes, s, o));
  const int64_t n = (int64_t)nrhs * V * 3;
  {
    ProfScope ps(ctx, K_PACK, s, 2.0 * (double)bytes);
    gamma5_gamma_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2*)i.dev, (double2*)o.dev, n, k);
  }
  MG_LAUNCH_CHECK();
  MG_CHECK(stage_out_finish(out, bytes, s, o));
  return MGLMA_OK;
}
