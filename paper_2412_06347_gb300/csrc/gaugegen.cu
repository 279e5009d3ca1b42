// Random SU(3) gauge fields generated on the device: the synthetic input
// recipe of the library's Python input generators, drawn from the same
// counter-based streams, so that lattices of tens of millions of sites (the
// 3 and 4 fm boxes) need no host-side generation or host->device copy.
//
// Link (site x, direction mu) is U = P_SU3(exp(i eps H)), H = sum_a h_a
// lambda_a / 2 with Gell-Mann matrices lambda_a and h_a ~ N(0, 1) the
// Gaussians 8 n .. 8 n + 7 of stream (seed, 1), n = 4 x + mu.  A stream is
// keyed by mix64(mix64(seed) ^ tag) and its k-th draw is mix64(key + k)
// (SplitMix64, Steele, Lea and Flood 2014); Gaussians come in Box-Muller
// pairs from uniforms ((z >> 11) + 1/2) 2^-53.  exp is an order-18 Taylor
// series in Horner form; the projection normalises row 0, orthogonalises and
// normalises row 1, and sets row 2 = conj(row0 x row1).  The transcendental
// functions are CUDA's, so links agree with the host generator to rounding
// (about 1e-16), not bit for bit.
#include <algorithm>
#include <string>

#include "internal.h"

namespace mglma {

__device__ __forceinline__ uint64_t gg_mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double gg_u53(uint64_t z) { return ((double)(z >> 11) + 0.5) * 0x1.0p-53; }

struct Z3 {
  double re[3][3], im[3][3];
};

// canonical links [site][mu][row][col] complex128 for sites site0 .. site0 + nsites - 1
__global__ void gauge_random_kernel(double2* __restrict__ out, int64_t site0, int64_t nsites, uint64_t key,
                                    double eps) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // local link index
  if (t >= nsites * 4) return;
  const uint64_t n = (uint64_t)(site0 * 4 + t);
  double h[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint64_t d = 8 * n + 2 * k;
    const double u1 = gg_u53(gg_mix64(key + d)), u2 = gg_u53(gg_mix64(key + d + 1));
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    h[2 * k] = r * cs;
    h[2 * k + 1] = r * sn;
  }
  // X = i eps H with H = sum_a h_a lambda_a / 2 (Hermitian, traceless)
  const double r3 = 1.0 / sqrt(3.0);
  double Hr[3][3], Hi[3][3];
  Hr[0][0] = 0.5 * (h[2] + h[7] * r3);
  Hr[1][1] = 0.5 * (-h[2] + h[7] * r3);
  Hr[2][2] = 0.5 * (-2.0 * h[7] * r3);
  Hi[0][0] = Hi[1][1] = Hi[2][2] = 0.0;
  Hr[0][1] = Hr[1][0] = 0.5 * h[0];
  Hi[0][1] = -0.5 * h[1];
  Hi[1][0] = 0.5 * h[1];
  Hr[0][2] = Hr[2][0] = 0.5 * h[3];
  Hi[0][2] = -0.5 * h[4];
  Hi[2][0] = 0.5 * h[4];
  Hr[1][2] = Hr[2][1] = 0.5 * h[5];
  Hi[1][2] = -0.5 * h[6];
  Hi[2][1] = 0.5 * h[6];
  Z3 X;  // i eps H
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      X.re[a][b] = -eps * Hi[a][b];
      X.im[a][b] = eps * Hr[a][b];
    }
  Z3 U;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      U.re[a][b] = a == b ? 1.0 : 0.0;
      U.im[a][b] = 0.0;
    }
  for (int k = 18; k >= 1; --k) {  // U <- X U / k + 1
    Z3 T;
    const double inv = 1.0 / (double)k;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double sr = 0.0, si = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sr += X.re[a][c] * U.re[c][b] - X.im[a][c] * U.im[c][b];
          si += X.re[a][c] * U.im[c][b] + X.im[a][c] * U.re[c][b];
        }
        T.re[a][b] = sr * inv + (a == b ? 1.0 : 0.0);
        T.im[a][b] = si * inv;
      }
    U = T;
  }
  // projection onto SU(3)
  double n0 = 0.0;
#pragma unroll
  for (int b = 0; b < 3; ++b) n0 += U.re[0][b] * U.re[0][b] + U.im[0][b] * U.im[0][b];
  n0 = 1.0 / sqrt(n0);
  double r0r[3], r0i[3], r1r[3], r1i[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    r0r[b] = U.re[0][b] * n0;
    r0i[b] = U.im[0][b] * n0;
  }
  double pr = 0.0, pi = 0.0;  // <r0, row1> = sum conj(r0) row1
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    pr += r0r[b] * U.re[1][b] + r0i[b] * U.im[1][b];
    pi += r0r[b] * U.im[1][b] - r0i[b] * U.re[1][b];
  }
  double n1 = 0.0;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    r1r[b] = U.re[1][b] - (pr * r0r[b] - pi * r0i[b]);
    r1i[b] = U.im[1][b] - (pr * r0i[b] + pi * r0r[b]);
    n1 += r1r[b] * r1r[b] + r1i[b] * r1i[b];
  }
  n1 = 1.0 / sqrt(n1);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    r1r[b] *= n1;
    r1i[b] *= n1;
  }
  double2* o = out + (size_t)t * 9;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    o[b] = make_double2(r0r[b], r0i[b]);
    o[3 + b] = make_double2(r1r[b], r1i[b]);
  }
  // row 2 = conj(r0 x r1): (r0 x r1)_b = r0_{b+1} r1_{b+2} - r0_{b+2} r1_{b+1}
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int p = (b + 1) % 3, q = (b + 2) % 3;
    const double cr = (r0r[p] * r1r[q] - r0i[p] * r1i[q]) - (r0r[q] * r1r[p] - r0i[q] * r1i[p]);
    const double ci = (r0r[p] * r1i[q] + r0i[p] * r1r[q]) - (r0r[q] * r1i[p] + r0i[q] * r1r[p]);
    o[6 + b] = make_double2(cr, -ci);
  }
}

static uint64_t gg_key(uint64_t seed, uint64_t tag) {
  auto h = [](uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  return h(h(seed) ^ tag);
}

}  // namespace mglma

using namespace mglma;

extern "C" mglma_status mglma_gauge_random(mglma_ctx ctx, const mglma_lattice* lat, double eps, uint64_t seed,
                                           double kappa, double csw, mglma_gauge* out) {
  if (!ctx || !lat || !out) return fail(MGLMA_ERR_INVALID, "mglma_gauge_random: NULL argument");
  if (!(eps >= 0)) return fail(MGLMA_ERR_INVALID, "mglma_gauge_random: eps must be >= 0");
  for (int m = 0; m < 4; ++m)
    if (lat->L[m] < 1 || lat->L[m] > 4096) return fail(MGLMA_ERR_INVALID, "mglma_gauge_random: bad extent");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const int64_t slice = (int64_t)lat->L[1] * lat->L[2] * lat->L[3];
  // time slabs of at most ~512 MB of canonical links (576 B per site)
  const int64_t per_slab = std::max<int64_t>(1, ((int64_t)512 << 20) / (slice * 576));
  const int64_t tc_max = std::min<int64_t>(lat->L[0], per_slab);
  double2* buf = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&buf, (size_t)tc_max * slice * 36 * sizeof(double2), s));
  const uint64_t key = gg_key(seed, 1);
  mglma_gauge G = nullptr;
  mglma_status st = MGLMA_OK;
  for (int64_t t0 = 0; t0 < lat->L[0] && st == MGLMA_OK; t0 += tc_max) {
    const int64_t tc = std::min<int64_t>(tc_max, lat->L[0] - t0);
    const int64_t nl = tc * slice * 4;
    {
      ProfScope ps(ctx, K_SETUP, s);
      gauge_random_kernel<<<(unsigned)((nl + 127) / 128), 128, 0, s>>>(buf, t0 * slice, tc * slice, key, eps);
    }
    if (cudaGetLastError() != cudaSuccess) {
      st = fail(MGLMA_ERR_CUDA, "mglma_gauge_random: launch failed");
      break;
    }
    st = mglma_gauge_load(ctx, lat, (const double*)buf, t0, tc, kappa, csw, &G);
  }
  dfree(ctx, buf, s);
  cudaStreamSynchronize(s);
  cudaMemPoolTrimTo(ctx->pool, 0);
  if (st != MGLMA_OK) {
    mglma_gauge_free(G);
    return st;
  }
  *out = G;
  return MGLMA_OK;
}
