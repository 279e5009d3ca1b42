// Block basis of the multigrid low-mode construction and the transfer
// operators R0 / T0.
//
// Sec. 3 / Sec. 4, Eq. mg_basis: the fields P_alpha theta_{B_y} v_c
// (alpha = 0, 1 chiralities, c < Nv test vectors, y a block of the regular
// decomposition, Eq. block_def) are orthonormalised inside each block and
// chirality; R0 (Eq. res_mg) and T0 (Eq. pro_mg) project onto and expand from
// that basis.
//
// Test vectors (the paper uses exact low modes and notes that inexact ones
// work the same way): Nv Gaussian starts drawn on the device from the
// counter-based generator (SplitMix64 + Box-Muller, the same definition the
// Python input generators use), then n_smooth minimal-residual steps on
// D v = 0 in FP64, all Nv vectors as one multi-RHS batch.
//
// Orthonormalisation: the Q factor with positive real diagonal R of the
// (6|B| x Nv) matrix of one block and chirality is unique; Gram-Schmidt is one
// way to reach it.  On the GPU it is reached by CholeskyQR2 (Gram matrix,
// Cholesky, U R^-1, all twice) in FP64, which streams each block's vectors a
// fixed number of times instead of O(Nv^2) times.
//
// Basis layouts (per block y, dof j = alpha*Nv + c, site-in-block k, and the
// six (spin mod 2, colour) components q of chirality alpha):
//   FP64 : double2 [V1][2Nv][6][|B|]
//   FP32 : float4  [V1][2Nv][3][|B|]          (2 complex per float4)
//   FP16 : uint2   [V1][2Nv][3][|B|] (2 complex as 4 halves) with one FP32
//          scale per (y, j): value = half * scale
#include <algorithm>
#include <cmath>
#include <mutex>

#include "cplx.cuh"
#include "internal.h"
#include "solver.h"
#include "subspace.h"

namespace mglma {

// ------------------------------------------------------------ geometry
BlockGeo make_blockgeo(const int L[4], const int b[4]) {
  BlockGeo g;
  g.V = 1;
  g.V1 = 1;
  g.nB = 1;
  for (int m = 0; m < 4; ++m) {
    g.L[m] = L[m];
    g.b[m] = b[m];
    g.Lb[m] = L[m] / b[m];
    g.V *= L[m];
    g.V1 *= g.Lb[m];
    g.nB *= b[m];
  }
  return g;
}

__device__ __forceinline__ int64_t block_site(const BlockGeo& g, int64_t y, int k) {
  int yc[4], kc[4];
  int64_t t = y;
  for (int m = 3; m >= 0; --m) {
    yc[m] = (int)(t % g.Lb[m]);
    t /= g.Lb[m];
  }
  int u = k;
  for (int m = 3; m >= 0; --m) {
    kc[m] = u % g.b[m];
    u /= g.b[m];
  }
  int64_t s = 0;
  for (int m = 0; m < 4; ++m) s = s * g.L[m] + (int64_t)yc[m] * g.b[m] + kc[m];
  return s;
}

// ------------------------------------------------------------ random starts
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u53(uint64_t z) { return ((double)(z >> 11) + 0.5) * 0x1.0p-53; }

// Gaussian start vectors in the internal FP64 layout; complex component k of
// vector c at site s uses Gaussian pair n = (c V + s) 12 + k of stream (seed, 3).
__global__ void random_starts_kernel(double2* __restrict__ out, int64_t V, int nv, uint64_t key) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (s >= V || c >= nv) return;
  for (int k = 0; k < 12; ++k) {
    const uint64_t n = ((uint64_t)c * V + s) * 12 + k;
    const double u1 = u53(mix64(key + 2 * n)), u2 = u53(mix64(key + 2 * n + 1));
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[((size_t)c * 12 + k) * V + s] = make_double2(r * cs, r * sn);
  }
}

// The same Gaussians rounded to FP32 in the FP32 internal layout, for the
// vectors c0 .. c0 + ng - 1 (lean set-up).
__global__ void random_starts32_kernel(float4* __restrict__ out, int64_t V, int ng, int c0, uint64_t key) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (s >= V || c >= ng) return;
  for (int k2 = 0; k2 < 6; ++k2) {
    float v[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t n = ((uint64_t)(c0 + c) * V + s) * 12 + 2 * k2 + h;
      const double u1 = u53(mix64(key + 2 * n)), u2 = u53(mix64(key + 2 * n + 1));
      const double r = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      v[2 * h] = (float)(r * cs);
      v[2 * h + 1] = (float)(r * sn);
    }
    out[((size_t)c * 6 + k2) * V + s] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// ------------------------------------------------------------ basis IO
template <typename B>
struct BIO;

template <>
struct BIO<double> {  // double2 [y][j][6][nB]
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, const float*, size_t yj, int nB, int k, Cx<R> o[6]) {
    const double2* p = reinterpret_cast<const double2*>(base) + yj * 6 * nB + k;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      double2 v = __ldg(p + q * nB);
      o[q] = cx((R)v.x, (R)v.y);
    }
  }
};
template <>
struct BIO<float> {  // float4 [y][j][3][nB]
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, const float*, size_t yj, int nB, int k, Cx<R> o[6]) {
    const float4* p = reinterpret_cast<const float4*>(base) + yj * 3 * nB + k;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float4 v = __ldg(p + q * nB);
      o[2 * q] = cx((R)v.x, (R)v.y);
      o[2 * q + 1] = cx((R)v.z, (R)v.w);
    }
  }
};
template <>
struct BIO<__half> {  // uint2 (4 halves) [y][j][3][nB], scale per (y, j)
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, const float* scale, size_t yj, int nB, int k,
                                              Cx<R> o[6]) {
    const uint2* p = reinterpret_cast<const uint2*>(base) + yj * 3 * nB + k;
    const float sc = __ldg(scale + yj);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      uint2 v = __ldg(p + q * nB);
      __half2 a = *reinterpret_cast<__half2*>(&v.x), b = *reinterpret_cast<__half2*>(&v.y);
      float2 fa = __half22float2(a), fb = __half22float2(b);
      o[2 * q] = cx((R)(fa.x * sc), (R)(fa.y * sc));
      o[2 * q + 1] = cx((R)(fb.x * sc), (R)(fb.y * sc));
    }
  }
};

// fine spinor component q (0..11) of RHS r at a site, internal layout
template <typename R>
__device__ __forceinline__ Cx<R> fine_get(const void* f, int64_t V, int r, int64_t site, int q);
template <>
__device__ __forceinline__ Cx<float> fine_get<float>(const void* f, int64_t V, int r, int64_t site, int q) {
  const float2* p = reinterpret_cast<const float2*>(reinterpret_cast<const float4*>(f) + ((size_t)r * 6 + q / 2) * V + site);
  float2 v = p[q & 1];
  return cx(v.x, v.y);
}
template <>
__device__ __forceinline__ Cx<double> fine_get<double>(const void* f, int64_t V, int r, int64_t site, int q) {
  double2 v = reinterpret_cast<const double2*>(f)[((size_t)r * 12 + q) * V + site];
  return cx(v.x, v.y);
}

// ------------------------------------------------------------ R0: restrict
// out[r][y][j] = sum_{k in B_y} sum_q conj(phi_{y j}(k)_q) psi_r(site(y,k))_{6 alpha(j) + q}
// One CTA per (block, RHS tile): the block's spinors are staged in shared
// memory (component-major, conflict-free), each warp owns a set of dofs j,
// lanes stride over the sites reading the basis coalesced, and a warp-shuffle
// reduction finishes each inner product.
constexpr int RP_THREADS = 256;
constexpr int RP_CHUNK = 128;  // sites per shared-memory chunk

template <typename R, typename B, int NRT, int JW>
__global__ void __launch_bounds__(RP_THREADS) restrict_kernel(const void* __restrict__ fine, int nrhs,
                                                              const void* __restrict__ basis,
                                                              const float* __restrict__ scale, BlockGeo g, int n2,
                                                              Cx<R>* __restrict__ out) {
  extern __shared__ unsigned char smraw[];
  Cx<R>* sm = reinterpret_cast<Cx<R>*>(smraw);  // [NRT][12][RP_CHUNK]
  // RHS tiles fastest: the CTAs of one block run together and share its basis in L2
  const int ntile = (nrhs + NRT - 1) / NRT;
  const int64_t y = blockIdx.x / ntile;
  const int r0 = (int)(blockIdx.x % ntile) * NRT;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  constexpr int NW = RP_THREADS / 32;
  constexpr int MAXJ = JW;  // dofs per warp
  Cx<R> acc[MAXJ][NRT];
#pragma unroll
  for (int a = 0; a < MAXJ; ++a)
#pragma unroll
    for (int r = 0; r < NRT; ++r) acc[a][r] = cx<R>(0, 0);

  __shared__ int64_t site_of[RP_CHUNK];
  const int nv = n2 / 2;
  for (int k0 = 0; k0 < g.nB; k0 += RP_CHUNK) {
    const int ck = min(RP_CHUNK, g.nB - k0);
    __syncthreads();
    for (int kk = threadIdx.x; kk < ck; kk += RP_THREADS) site_of[kk] = block_site(g, y, k0 + kk);
    __syncthreads();
    if constexpr (sizeof(R) == 4) {  // 16-byte loads: two complex components per load
      for (int idx = threadIdx.x; idx < NRT * 6 * ck; idx += RP_THREADS) {
        const int kk = idx % ck, c = (idx / ck) % 6, r = idx / (ck * 6);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r0 + r < nrhs) v = __ldg(reinterpret_cast<const float4*>(fine) + ((size_t)(r0 + r) * 6 + c) * g.V + site_of[kk]);
        sm[(r * 12 + 2 * c) * RP_CHUNK + kk] = cx<R>(v.x, v.y);
        sm[(r * 12 + 2 * c + 1) * RP_CHUNK + kk] = cx<R>(v.z, v.w);
      }
    } else {
      for (int idx = threadIdx.x; idx < NRT * 12 * ck; idx += RP_THREADS) {
        const int kk = idx % ck, q = (idx / ck) % 12, r = idx / (ck * 12);
        Cx<R> v = cx<R>(0, 0);
        if (r0 + r < nrhs) v = fine_get<R>(fine, g.V, r0 + r, site_of[kk], q);
        sm[(r * 12 + q) * RP_CHUNK + kk] = v;
      }
    }
    __syncthreads();
    // per site of the lane and chirality: the spinor components once into
    // registers, then every dof of this warp with that chirality
    for (int kk = lane; kk < ck; kk += 32) {
#pragma unroll
      for (int al = 0; al < 2; ++al) {
        Cx<R> ps[NRT][6];
#pragma unroll
        for (int r = 0; r < NRT; ++r)
#pragma unroll
          for (int q = 0; q < 6; ++q) ps[r][q] = sm[(r * 12 + 6 * al + q) * RP_CHUNK + kk];
#pragma unroll
        for (int a = 0; a < MAXJ; ++a) {
          const int j = warp + a * NW;
          if (j >= n2 || (j >= nv) != (al == 1)) continue;
          Cx<R> ph[6];
          BIO<B>::template load<R>(basis, scale, (size_t)y * n2 + j, g.nB, k0 + kk, ph);
#pragma unroll
          for (int r = 0; r < NRT; ++r)
#pragma unroll
            for (int q = 0; q < 6; ++q) cfma_conj(acc[a][r], ph[q], ps[r][q]);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < MAXJ; ++a) {
    const int j = warp + a * NW;
    if (j >= n2) break;
#pragma unroll
    for (int r = 0; r < NRT; ++r) {
      Cx<R> v = acc[a][r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v.re += __shfl_down_sync(0xffffffffu, v.re, o);
        v.im += __shfl_down_sync(0xffffffffu, v.im, o);
      }
      if (lane == 0 && r0 + r < nrhs) out[((size_t)(r0 + r) * g.V1 + y) * n2 + j] = v;
    }
  }
}

// ------------------------------------------------------------ T0: prolong
// fine_r(site(y,k))_{6 alpha + q} (+)= sum_j coarse[r][y][j] phi_{y j}(k)_q
template <typename R, typename B, int NRT>
__global__ void __launch_bounds__(RP_THREADS) prolong_kernel(const Cx<R>* __restrict__ coarse, int nrhs,
                                                             const void* __restrict__ basis,
                                                             const float* __restrict__ scale, BlockGeo g, int n2,
                                                             void* __restrict__ fine, int accumulate) {
  extern __shared__ unsigned char smraw[];
  Cx<R>* cs = reinterpret_cast<Cx<R>*>(smraw);  // [NRT][n2]
  const int ntile = (nrhs + NRT - 1) / NRT;
  const int64_t y = blockIdx.x / ntile;
  const int r0 = (int)(blockIdx.x % ntile) * NRT;
  for (int idx = threadIdx.x; idx < NRT * n2; idx += RP_THREADS) {
    const int j = idx % n2, r = idx / n2;
    cs[idx] = (r0 + r < nrhs) ? coarse[((size_t)(r0 + r) * g.V1 + y) * n2 + j] : cx<R>(0, 0);
  }
  __syncthreads();
  const int nv = n2 / 2;
  for (int k = threadIdx.x; k < g.nB; k += RP_THREADS) {
    Cx<R> acc[NRT][12];
#pragma unroll
    for (int r = 0; r < NRT; ++r)
#pragma unroll
      for (int q = 0; q < 12; ++q) acc[r][q] = cx<R>(0, 0);
    for (int j = 0; j < n2; ++j) {
      Cx<R> ph[6];
      BIO<B>::template load<R>(basis, scale, (size_t)y * n2 + j, g.nB, k, ph);
      const int qa = j < nv ? 0 : 6;
#pragma unroll
      for (int r = 0; r < NRT; ++r) {
        const Cx<R> c = cs[r * n2 + j];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          // only the chirality of j is touched; select by branch-free index
          if (qa == 0)
            cfma(acc[r][q], c, ph[q]);
          else
            cfma(acc[r][6 + q], c, ph[q]);
        }
      }
    }
    const int64_t site = block_site(g, y, k);
#pragma unroll
    for (int r = 0; r < NRT; ++r) {
      if (r0 + r >= nrhs) break;
      if (sizeof(R) == 4) {
        float4* p = reinterpret_cast<float4*>(fine) + (size_t)(r0 + r) * 6 * g.V + site;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          float4 v = make_float4(acc[r][2 * c].re, acc[r][2 * c].im, acc[r][2 * c + 1].re, acc[r][2 * c + 1].im);
          if (accumulate) {
            float4 o = p[c * g.V];
            v.x += o.x;
            v.y += o.y;
            v.z += o.z;
            v.w += o.w;
          }
          p[c * g.V] = v;
        }
      } else {
        double2* p = reinterpret_cast<double2*>(fine) + (size_t)(r0 + r) * 12 * g.V + site;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          double2 v = make_double2(acc[r][c].re, acc[r][c].im);
          if (accumulate) {
            double2 o = p[c * g.V];
            v.x += o.x;
            v.y += o.y;
          }
          p[c * g.V] = v;
        }
      }
    }
  }
}

// ------------------------------------------------------------ chirality split into the basis buffer
// phi64[y][alpha Nv + c][q][k] = component (2 alpha + q/3, q%3) of v_c at site(y,k)
__global__ void split_kernel(const double2* __restrict__ vecs, int nv, BlockGeo g, double2* __restrict__ phi) {
  const int64_t y = blockIdx.x;
  const int j = blockIdx.y;  // 0 .. 2nv-1
  const int alpha = j / nv, c = j % nv;
  for (int k = threadIdx.x; k < g.nB; k += blockDim.x) {
    const int64_t site = block_site(g, y, k);
#pragma unroll
    for (int q = 0; q < 6; ++q)
      phi[(((size_t)y * 2 * nv + j) * 6 + q) * g.nB + k] = vecs[((size_t)c * 12 + 6 * alpha + q) * g.V + site];
  }
}

// The same from FP32 vectors ([c][6 float4 chunks][V]) for blocks y0 + blockIdx.x,
// written to a chunk buffer that starts at block y0.
__global__ void split32_kernel(const float4* __restrict__ vecs, int nv, BlockGeo g, int64_t y0,
                               double2* __restrict__ phi) {
  const int64_t yl = blockIdx.x;
  const int j = blockIdx.y;
  const int alpha = j / nv, c = j % nv;
  for (int k = threadIdx.x; k < g.nB; k += blockDim.x) {
    const int64_t site = block_site(g, y0 + yl, k);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int cidx = 6 * alpha + q;  // complex component (spin, colour)
      const float4 v = vecs[((size_t)c * 6 + cidx / 2) * g.V + site];
      phi[(((size_t)yl * 2 * nv + j) * 6 + q) * g.nB + k] =
          (cidx & 1) ? make_double2(v.z, v.w) : make_double2(v.x, v.y);
    }
  }
}

// stored FP32 / FP16 basis -> FP64 layout (export of a lean subspace)
template <typename B>
__global__ void basis_widen_kernel(const void* __restrict__ src, const float* __restrict__ scale,
                                   double2* __restrict__ p64, size_t nyj, int nB) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nyj * nB
  if (i >= nyj * nB) return;
  const size_t yj = i / nB;
  const int k = (int)(i % nB);
  Cx<double> o[6];
  BIO<B>::template load<double>(src, scale, yj, nB, k, o);
#pragma unroll
  for (int q = 0; q < 6; ++q) p64[(yj * 6 + q) * nB + k] = make_double2(o[q].re, o[q].im);
}

// ------------------------------------------------------------ CholeskyQR2 per (block, chirality)
constexpr int GS_THREADS = 256;
constexpr int GS_TR = 32;  // rows per shared tile

// U: the Nv columns j = alpha Nv + c of block y, rows (q, k): element at
// phi[((y*2nv + j)*6 + q)*nB + k].  Overwritten by the orthonormal factor.
__global__ void __launch_bounds__(GS_THREADS) cholqr2_kernel(double2* __restrict__ phi, int nv, BlockGeo g,
                                                             double rank_tol, int* __restrict__ rank_flag) {
  extern __shared__ unsigned char smraw[];
  double2* G = reinterpret_cast<double2*>(smraw);  // [nv][nv]
  double2* Ri = G + nv * nv;                         // [nv][nv] upper-triangular R^-1
  double2* T = Ri + nv * nv;                         // [GS_TR][nv] row tile
  __shared__ int bad;
  const int64_t y = blockIdx.x;
  const int alpha = blockIdx.y;
  const int nrows = 6 * g.nB;
  double2* U = phi + ((size_t)y * 2 * nv + (size_t)alpha * nv) * 6 * g.nB;  // column j at U + j*6nB
  const size_t cstride = (size_t)6 * g.nB;

  for (int pass = 0; pass < 2; ++pass) {
    // ---- Gram matrix G = U^dag U (upper triangle, accumulated in shared memory)
    for (int e = threadIdx.x; e < nv * nv; e += GS_THREADS) G[e] = make_double2(0, 0);
    if (threadIdx.x == 0) bad = 0;
    const int nent = nv * (nv + 1) / 2;
    for (int r0 = 0; r0 < nrows; r0 += GS_TR) {
      const int tr = min(GS_TR, nrows - r0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < tr * nv; idx += GS_THREADS) {
        const int rr = idx % tr, j = idx / tr;
        T[rr * nv + j] = U[j * cstride + r0 + rr];
      }
      __syncthreads();
      for (int e = threadIdx.x; e < nent; e += GS_THREADS) {
        // entry e -> (i, j), i <= j, row-major over the upper triangle
        int i = 0, rem = e;
        while (rem >= nv - i) {
          rem -= nv - i;
          ++i;
        }
        const int j = i + rem;
        double2 s = G[i * nv + j];
        for (int rr = 0; rr < tr; ++rr) {
          const double2 a = T[rr * nv + i], b = T[rr * nv + j];
          s.x += a.x * b.x + a.y * b.y;
          s.y += a.x * b.y - a.y * b.x;
        }
        G[i * nv + j] = s;
      }
    }
    __syncthreads();
    // ---- Cholesky G = R^dag R (R upper, positive real diagonal), then R^-1
    if (threadIdx.x == 0) {
      for (int c = 0; c < nv; ++c) {
        double d = G[c * nv + c].x;
        const double d0 = d;
        for (int i = 0; i < c; ++i) d -= G[i * nv + c].x * G[i * nv + c].x + G[i * nv + c].y * G[i * nv + c].y;
        if (!(d > rank_tol * rank_tol * d0) || !(d0 > 0)) {
          bad = 1;
          d = d0 > 0 ? d0 : 1.0;
        }
        const double rc = sqrt(d);
        G[c * nv + c] = make_double2(rc, 0);
        for (int j = c + 1; j < nv; ++j) {
          double2 s = G[c * nv + j];
          for (int i = 0; i < c; ++i) {
            const double2 a = G[i * nv + c], b = G[i * nv + j];  // conj(R_ic) R_ij
            s.x -= a.x * b.x + a.y * b.y;
            s.y -= a.x * b.y - a.y * b.x;
          }
          G[c * nv + j] = make_double2(s.x / rc, s.y / rc);
        }
      }
      // R^-1 (upper): column by column back substitution
      for (int j = 0; j < nv; ++j) {
        for (int i = nv - 1; i >= 0; --i) {
          double2 s = make_double2(i == j ? 1.0 : 0.0, 0.0);
          for (int l = i + 1; l <= j; ++l) {
            const double2 a = G[i * nv + l], b = Ri[l * nv + j];
            s.x -= a.x * b.x - a.y * b.y;
            s.y -= a.x * b.y + a.y * b.x;
          }
          const double rd = G[i * nv + i].x;
          Ri[i * nv + j] = i > j ? make_double2(0, 0) : make_double2(s.x / rd, s.y / rd);
        }
      }
      if (bad && pass == 0) atomicOr(rank_flag, 1);
    }
    __syncthreads();
    // ---- U <- U R^-1, tile by tile
    for (int r0 = 0; r0 < nrows; r0 += GS_TR) {
      const int tr = min(GS_TR, nrows - r0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < tr * nv; idx += GS_THREADS) {
        const int rr = idx % tr, j = idx / tr;
        T[rr * nv + j] = U[j * cstride + r0 + rr];
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < tr * nv; idx += GS_THREADS) {
        const int rr = idx % tr, j = idx / tr;
        double2 s = make_double2(0, 0);
        for (int i = 0; i <= j; ++i) {
          const double2 a = T[rr * nv + i], b = Ri[i * nv + j];
          s.x += a.x * b.x - a.y * b.y;
          s.y += a.x * b.y + a.y * b.x;
        }
        U[j * cstride + r0 + rr] = s;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ precision conversion of the basis
__global__ void basis_to32_kernel(const double2* __restrict__ p64, float4* __restrict__ p32, size_t nyj, int nB) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nyj * 3 * nB
  if (i >= nyj * 3 * nB) return;
  const size_t yj = i / (3 * (size_t)nB);
  const int q = (int)((i / nB) % 3), k = (int)(i % nB);
  const double2 a = p64[(yj * 6 + 2 * q) * nB + k], b = p64[(yj * 6 + 2 * q + 1) * nB + k];
  p32[i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// scale[yj] = max |component| of vector (y, j); then quantise to FP16
__global__ void basis_scale_kernel(const double2* __restrict__ p64, float* __restrict__ scale, int nB) {
  const size_t yj = blockIdx.x;
  double m = 0;
  for (int i = threadIdx.x; i < 6 * nB; i += blockDim.x) {
    const double2 v = p64[yj * 6 * nB + i];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double wm[32];
  if (threadIdx.x % 32 == 0) wm[threadIdx.x / 32] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t = fmax(t, wm[w]);
    scale[yj] = t > 0 ? (float)t : 1.0f;
  }
}

__global__ void basis_to16_kernel(const double2* __restrict__ p64, const float* __restrict__ scale,
                                  uint2* __restrict__ p16, size_t nyj, int nB) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nyj * 3 * nB) return;
  const size_t yj = i / (3 * (size_t)nB);
  const int q = (int)((i / nB) % 3), k = (int)(i % nB);
  const float inv = 1.0f / scale[yj];
  const double2 a = p64[(yj * 6 + 2 * q) * nB + k], b = p64[(yj * 6 + 2 * q + 1) * nB + k];
  __half2 ha = __floats2half2_rn((float)a.x * inv, (float)a.y * inv);
  __half2 hb = __floats2half2_rn((float)b.x * inv, (float)b.y * inv);
  uint2 o;
  o.x = *reinterpret_cast<unsigned*>(&ha);
  o.y = *reinterpret_cast<unsigned*>(&hb);
  p16[i] = o;
}

// canonical export: [V1][2][Nv][nB][4][3] complex128 (other chirality zero)
__global__ void basis_export_kernel(const double2* __restrict__ p64, double2* __restrict__ out, int nv, int nB,
                                    size_t nyj) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over nyj * nB
  if (i >= nyj * nB) return;
  const size_t yj = i / nB;
  const int k = (int)(i % nB);
  const int alpha = (int)((yj % (2 * nv)) / nv);
  double2* o = out + i * 12;
#pragma unroll
  for (int q = 0; q < 12; ++q) o[q] = make_double2(0, 0);
#pragma unroll
  for (int q = 0; q < 6; ++q) o[6 * alpha + q] = p64[(yj * 6 + q) * nB + k];
}

// ------------------------------------------------------------ R0 / T0 at many RHS (FP32 fields)
// One CTA per (block, tile of 16 RHS), so the block's basis is read once for
// all of them.  Both kernels walk the block's sites in chunks staged in
// shared memory by cp.async into two buffers: the next chunk is in flight
// while the current one is consumed.  The FP16 basis is staged as it is
// stored (converted at use) and its per-(block, dof) scale multiplies the R0
// result and the T0 coefficients instead of every element.  Rows are padded
// so that the consumers' loads of consecutive sites fall in different banks.
//   R0: each thread owns a 4 dof x 4 RHS tile of the outputs over a share of
//       each chunk's sites (split K); the shares are summed in a fixed order.
//   T0: each thread owns one site of the chunk, one chirality and four RHS
//       (6 x 4 complex accumulators) and runs over that chirality's Nv dofs.
// Needs Nv % 4 == 0 and 2 Nv <= 64.
constexpr int T16_KC = 16;     // sites per chunk (R0)
constexpr int T16_MAXT = 384;  // R0 threads per CTA (at most)
constexpr int T16_TKC = 32;    // sites per chunk (T0)

__device__ __forceinline__ uint32_t t16_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <int BYTES>
__device__ __forceinline__ void t16_cp(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(t16_smem(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void t16_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void t16_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// one complex basis element as staged: FP16 pair (4 B) or FP32 pair (8 B)
template <typename B>
struct T16El;
template <>
struct T16El<__half> {
  static constexpr int bytes = 4;
  __device__ __forceinline__ static Cx<float> get(const void* p) {
    uint32_t u = *reinterpret_cast<const uint32_t*>(p);
    const float2 f = __half22float2(*reinterpret_cast<__half2*>(&u));
    return cx(f.x, f.y);
  }
};
template <>
struct T16El<float> {
  static constexpr int bytes = 8;
  __device__ __forceinline__ static Cx<float> get(const void* p) {
    const float2 f = *reinterpret_cast<const float2*>(p);
    return cx(f.x, f.y);
  }
};
template <typename B>
__device__ __forceinline__ float basis_scale(const float* scale, size_t yj) {
  return sizeof(B) == 2 ? __ldg(scale + yj) : 1.f;
}

// bytes of one staged R0 chunk row (site kk): phi [q][jg][a] elements, then
// psi [c][h][rg] float4, each padded by 16 B
template <typename B>
__host__ __device__ constexpr int r16_phi_row(int n2) { return 6 * n2 * T16El<B>::bytes + 16; }
constexpr int R16_PSI_ROW = 12 * 2 * 4 * 16 + 16;
template <typename B>
__host__ __device__ constexpr size_t r16_buf(int n2) { return (size_t)T16_KC * (r16_phi_row<B>(n2) + R16_PSI_ROW); }

template <typename B>
__global__ void __launch_bounds__(T16_MAXT) restrict16_kernel(const float4* __restrict__ fine, int nrhs,
                                                              const void* __restrict__ basis,
                                                              const float* __restrict__ scale, BlockGeo g, int nv,
                                                              float2* __restrict__ out) {
  extern __shared__ float4 sm16[];
  constexpr int EB = T16El<B>::bytes;
  const int n2 = 2 * nv, ng = n2 / 4;
  const int prow = r16_phi_row<B>(n2);
  const size_t buf = r16_buf<B>(n2);
  uint8_t* base = reinterpret_cast<uint8_t*>(sm16);
  int64_t* site_of = reinterpret_cast<int64_t*>(base + 2 * buf);  // [nB]
  const int ntile = (nrhs + 15) / 16;
  const int64_t y = blockIdx.x / ntile;
  const int r0 = (int)(blockIdx.x % ntile) * 16;
  const int ntt = 4 * ng;  // output tiles (dof group, RHS group)
  const int KS = blockDim.x / ntt;
  const int tid = threadIdx.x;
  const int tt = tid % ntt, ks = tid / ntt;
  const int jg = tt % ng, rg = tt / ng;
  const int al = (4 * jg) / nv;
  for (int k = tid; k < g.nB; k += blockDim.x) site_of[k] = block_site(g, y, k);
  __syncthreads();
  const size_t esz = sizeof(B) == 2 ? 8 : 16;  // stored bytes of two complex components
  // stage chunk k0 into buffer b (cp.async; RHS beyond nrhs read as zero)
  auto stage = [&](int k0, int b) {
    const int ck = min(T16_KC, g.nB - k0);
    uint8_t* bb = base + (size_t)b * buf;
    for (int idx = tid; idx < n2 * 3 * ck; idx += blockDim.x) {
      const int kk = idx % ck, c = (idx / ck) % 3, j = idx / (ck * 3);
      const uint8_t* src = reinterpret_cast<const uint8_t*>(basis) + (((size_t)y * n2 + j) * 3 + c) * g.nB * esz +
                           (size_t)(k0 + kk) * esz;
      uint8_t* row = bb + (size_t)kk * (prow + R16_PSI_ROW);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        t16_cp<EB>(row + (((2 * c + h) * ng + j / 4) * 4 + j % 4) * EB, src + h * EB);
    }
    for (int idx = tid; idx < 16 * 6 * ck; idx += blockDim.x) {
      const int kk = idx % ck, c = (idx / ck) % 6, r = idx / (ck * 6);
      uint8_t* row = bb + (size_t)kk * (prow + R16_PSI_ROW) + prow;
      float2* d0 = reinterpret_cast<float2*>(row + (((2 * c) * 2 + (r % 4) / 2) * 4 + r / 4) * 16 + (r % 2) * 8);
      float2* d1 = reinterpret_cast<float2*>(row + (((2 * c + 1) * 2 + (r % 4) / 2) * 4 + r / 4) * 16 + (r % 2) * 8);
      if (r0 + r < nrhs) {
        const float4* src = fine + ((size_t)(r0 + r) * 6 + c) * g.V + site_of[k0 + kk];
        t16_cp<8>(d0, src);
        t16_cp<8>(d1, reinterpret_cast<const uint8_t*>(src) + 8);
      } else {
        *d0 = make_float2(0.f, 0.f);
        *d1 = make_float2(0.f, 0.f);
      }
    }
    t16_commit();
  };
  Cx<float> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = cx(0.f, 0.f);
  stage(0, 0);
  int b = 0;
  for (int k0 = 0; k0 < g.nB; k0 += T16_KC, b ^= 1) {
    const int ck = min(T16_KC, g.nB - k0);
    t16_wait();
    __syncthreads();  // chunk k0 landed in buffer b; buffer b ^ 1 is free
    if (k0 + T16_KC < g.nB) stage(k0 + T16_KC, b ^ 1);
    const uint8_t* bb = base + (size_t)b * buf;
    if (ks < KS) {
      for (int kk = ks; kk < ck; kk += KS) {
        const uint8_t* prw = bb + (size_t)kk * (prow + R16_PSI_ROW);
        const float4* srw = reinterpret_cast<const float4*>(prw + prow);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint8_t* pe = prw + ((q * ng + jg) * 4) * EB;
          const Cx<float> ph[4] = {T16El<B>::get(pe), T16El<B>::get(pe + EB), T16El<B>::get(pe + 2 * EB),
                                   T16El<B>::get(pe + 3 * EB)};
          const float4 sa = srw[((6 * al + q) * 2 + 0) * 4 + rg], sb = srw[((6 * al + q) * 2 + 1) * 4 + rg];
          const Cx<float> ps[4] = {cx(sa.x, sa.y), cx(sa.z, sa.w), cx(sb.x, sb.y), cx(sb.z, sb.w)};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c2 = 0; c2 < 4; ++c2) cfma_conj(acc[a][c2], ph[a], ps[c2]);
        }
      }
    }
  }
  // sum the K shares in a fixed order
  __syncthreads();
  float2* red = reinterpret_cast<float2*>(sm16);  // [ks][tt][16]
  if (ks < KS)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2)
        red[((size_t)ks * ntt + tt) * 16 + a * 4 + c2] = make_float2(acc[a][c2].re, acc[a][c2].im);
  __syncthreads();
  for (int o = tid; o < n2 * 16; o += blockDim.x) {
    const int j = o % n2, r = o / n2;
    if (r0 + r >= nrhs) continue;
    const int t2 = (r / 4) * ng + j / 4, e = (j % 4) * 4 + r % 4;
    float sx = 0.f, sy = 0.f;
    for (int k = 0; k < KS; ++k) {
      const float2 v = red[((size_t)k * ntt + t2) * 16 + e];
      sx += v.x;
      sy += v.y;
    }
    const float sc = basis_scale<B>(scale, (size_t)y * n2 + j);
    out[((size_t)(r0 + r) * g.V1 + y) * n2 + j] = make_float2(sc * sx, sc * sy);
  }
}

// bytes of one staged T0 chunk row (site kk): the basis [j][q] elements, padded
// by two elements (consecutive sites' rows two banks apart for FP16, four for
// FP32; rows stay aligned for the 8- or 16-byte copies)
template <typename B>
__host__ __device__ constexpr int p16_row(int n2) { return 6 * n2 * T16El<B>::bytes + 2 * T16El<B>::bytes; }

template <typename B>
__global__ void __launch_bounds__(256) prolong16_kernel(const float2* __restrict__ coarse, int nrhs,
                                                        const void* __restrict__ basis,
                                                        const float* __restrict__ scale, BlockGeo g, int nv,
                                                        float4* __restrict__ fine, int accumulate) {
  extern __shared__ float4 sm16[];
  constexpr int EB = T16El<B>::bytes;
  __shared__ float4 cs[64 * 2 * 4];  // [j][h][rg] = scale_j (c_{4rg+2h}, c_{4rg+2h+1}), n2 <= 64
  const int n2 = 2 * nv;
  const int prow = p16_row<B>(n2);
  const size_t buf = (size_t)T16_TKC * prow;
  uint8_t* base = reinterpret_cast<uint8_t*>(sm16);
  const int ntile = (nrhs + 15) / 16;
  const int64_t y = blockIdx.x / ntile;
  const int r0 = (int)(blockIdx.x % ntile) * 16;
  const int tid = threadIdx.x;
  const size_t esz = sizeof(B) == 2 ? 8 : 16;
  auto stage = [&](int k0, int b) {
    const int ck = min(T16_TKC, g.nB - k0);
    uint8_t* bb = base + (size_t)b * buf;
    for (int idx = tid; idx < n2 * 3 * ck; idx += blockDim.x) {
      const int kk = idx % ck, c = (idx / ck) % 3, j = idx / (ck * 3);
      const uint8_t* src = reinterpret_cast<const uint8_t*>(basis) + (((size_t)y * n2 + j) * 3 + c) * g.nB * esz +
                           (size_t)(k0 + kk) * esz;
      t16_cp<2 * EB>(bb + (size_t)kk * prow + (j * 6 + 2 * c) * EB, src);
    }
    t16_commit();
  };
  stage(0, 0);
  for (int idx = tid; idx < n2 * 16; idx += blockDim.x) {
    const int j = idx % n2, r = idx / n2;
    const float sc = basis_scale<B>(scale, (size_t)y * n2 + j);
    float2 v = r0 + r < nrhs ? coarse[((size_t)(r0 + r) * g.V1 + y) * n2 + j] : make_float2(0.f, 0.f);
    v.x *= sc;
    v.y *= sc;
    reinterpret_cast<float2*>(cs)[((j * 2 + (r % 4) / 2) * 4 + r / 4) * 2 + (r % 2)] = v;
  }
  // work item of a chunk: (site kk fastest, chirality, RHS group of four)
  const int kk = tid % T16_TKC, al = (tid / T16_TKC) % 2, rg = tid / (2 * T16_TKC);
  int b = 0;
  for (int k0 = 0; k0 < g.nB; k0 += T16_TKC, b ^= 1) {
    const int ck = min(T16_TKC, g.nB - k0);
    t16_wait();
    __syncthreads();  // chunk k0 landed in buffer b (and cs is ready); buffer b ^ 1 is free
    if (k0 + T16_TKC < g.nB) stage(k0 + T16_TKC, b ^ 1);
    if (kk >= ck || r0 + 4 * rg >= nrhs) continue;
    const uint8_t* row = base + (size_t)b * buf + (size_t)kk * prow;
    Cx<float> acc[6][4];
#pragma unroll
    for (int q = 0; q < 6; ++q)
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2) acc[q][c2] = cx(0.f, 0.f);
    for (int jj = 0; jj < nv; ++jj) {
      const int j = al * nv + jj;
      const uint8_t* pe = row + (size_t)j * 6 * EB;
      Cx<float> ph[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) ph[q] = T16El<B>::get(pe + q * EB);
      const float4 ca = cs[(j * 2 + 0) * 4 + rg], cb = cs[(j * 2 + 1) * 4 + rg];
      const Cx<float> cv[4] = {cx(ca.x, ca.y), cx(ca.z, ca.w), cx(cb.x, cb.y), cx(cb.z, cb.w)};
#pragma unroll
      for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) cfma(acc[q][c2], cv[c2], ph[q]);
    }
    const int64_t site = block_site(g, y, k0 + kk);
#pragma unroll
    for (int c2 = 0; c2 < 4; ++c2) {
      const int r = r0 + 4 * rg + c2;
      if (r >= nrhs) break;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float4* p = fine + ((size_t)r * 6 + 3 * al + c) * g.V + site;
        float4 v = make_float4(acc[2 * c][c2].re, acc[2 * c][c2].im, acc[2 * c + 1][c2].re, acc[2 * c + 1][c2].im);
        if (accumulate) {
          const float4 o = *p;
          v.x += o.x;
          v.y += o.y;
          v.z += o.z;
          v.w += o.w;
        }
        *p = v;
      }
    }
  }
  t16_wait();
}

// ============================================================ host side
static int subspace_smem_restrict(int nrt, int rbytes) { return nrt * 12 * RP_CHUNK * 2 * rbytes; }

template <typename R, typename B, int NRT, int JW>
static mglma_status launch_restrict_jw(const mglma_subspace_s* S, const void* fine, int nrhs, const void* basis,
                                       void* out, cudaStream_t s) {
  const BlockGeo g = S->geo;
  const int smem = subspace_smem_restrict(NRT, sizeof(R));
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(restrict_kernel<R, B, NRT, JW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr_set = true;
  }
  const unsigned grid = (unsigned)(g.V1 * ((nrhs + NRT - 1) / NRT));
  restrict_kernel<R, B, NRT, JW><<<grid, RP_THREADS, smem, s>>>(fine, nrhs, basis, S->scale16, g, 2 * S->nv,
                                                                reinterpret_cast<Cx<R>*>(out));
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// dofs per warp: ceil(2 Nv / 8) rounded up to an instantiated width
template <typename R, typename B, int NRT>
static mglma_status launch_restrict(const mglma_subspace_s* S, const void* fine, int nrhs, const void* basis,
                                    void* out, cudaStream_t s) {
  const int jw = (2 * S->nv + 7) / 8;
  if (jw <= 1) return launch_restrict_jw<R, B, NRT, 1>(S, fine, nrhs, basis, out, s);
  if (jw <= 2) return launch_restrict_jw<R, B, NRT, 2>(S, fine, nrhs, basis, out, s);
  if (jw <= 3) return launch_restrict_jw<R, B, NRT, 3>(S, fine, nrhs, basis, out, s);
  if (jw <= 4) return launch_restrict_jw<R, B, NRT, 4>(S, fine, nrhs, basis, out, s);
  if (jw <= 6) return launch_restrict_jw<R, B, NRT, 6>(S, fine, nrhs, basis, out, s);
  if (jw <= 8) return launch_restrict_jw<R, B, NRT, 8>(S, fine, nrhs, basis, out, s);
  if (jw <= 12) return launch_restrict_jw<R, B, NRT, 12>(S, fine, nrhs, basis, out, s);
  return launch_restrict_jw<R, B, NRT, 16>(S, fine, nrhs, basis, out, s);
}

template <typename R, typename B, int NRT>
static mglma_status launch_prolong(const mglma_subspace_s* S, const void* coarse, int nrhs, const void* basis,
                                   void* fine, bool acc, cudaStream_t s) {
  const BlockGeo g = S->geo;
  const int smem = NRT * 2 * S->nv * 2 * (int)sizeof(R);
  const unsigned grid = (unsigned)(g.V1 * ((nrhs + NRT - 1) / NRT));
  prolong_kernel<R, B, NRT><<<grid, RP_THREADS, smem, s>>>(reinterpret_cast<const Cx<R>*>(coarse), nrhs, basis,
                                                           S->scale16, g, 2 * S->nv, fine, acc ? 1 : 0);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// algorithmic traffic of R0 / T0: the basis once (2Nv x 6 complex per site
// in its storage precision) plus the fine and coarse fields once per RHS
static double transfer_bytes(const mglma_subspace_s* S, int prec, int nrhs) {
  const double V = (double)S->geo.V, V1 = (double)S->geo.V1, n2 = 2.0 * S->nv, N = nrhs;
  const double cb = prec == MGLMA_FP64 ? 16.0 : (S->phi16 ? 4.0 : 8.0);
  const double cf = prec == MGLMA_FP64 ? 16.0 : 8.0;
  return V * n2 * 6.0 * cb + N * (V * 12.0 * cf + V1 * n2 * cf) + (S->phi16 && prec != MGLMA_FP64 ? V1 * n2 * 4.0 : 0.0);
}

// ------------------------------------------------------------ coarse gamma5 gamma_k (level 1)
// out[((y b0 + t) n2 + i) n2 + j] = sum over the sites x of B_y on the block's
// local time slice t of phi_i(x)^dag gamma5 gamma_k phi_j(x).  In the chiral
// basis gamma5 gamma_k = [[0, -i sigma_k], [-i sigma_k, 0]] couples the two
// chiralities only, so blocks with alpha_i = alpha_j vanish; phi_i keeps the
// two spins of its chirality (q = spin * 3 + colour within them).
template <typename B>
__global__ void gamma_level1_kernel(const void* base, const float* scale, BlockGeo g, int nv, int k,
                                    double2* __restrict__ out) {
  const int64_t y = blockIdx.x / g.b[0];
  const int t = (int)(blockIdx.x % g.b[0]);
  const int n2 = 2 * nv;
  const int per_t = g.nB / g.b[0];  // site-in-block index: local time slowest
  // -i sigma_k as (re, im) of m00, m01, m10, m11
  double m[4][2];
  if (k == 1) {
    const double v[4][2] = {{0, 0}, {0, -1}, {0, -1}, {0, 0}};
    for (int a = 0; a < 4; ++a) m[a][0] = v[a][0], m[a][1] = v[a][1];
  } else if (k == 2) {
    const double v[4][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, 0}};
    for (int a = 0; a < 4; ++a) m[a][0] = v[a][0], m[a][1] = v[a][1];
  } else {
    const double v[4][2] = {{0, -1}, {0, 0}, {0, 0}, {0, 1}};
    for (int a = 0; a < 4; ++a) m[a][0] = v[a][0], m[a][1] = v[a][1];
  }
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
    const int i = e / n2, j = e % n2;
    Cx<double> acc = cx(0.0, 0.0);
    if (i / nv != j / nv) {
      for (int kk = t * per_t; kk < (t + 1) * per_t; ++kk) {
        Cx<double> pi[6], pj[6];
        BIO<B>::template load<double>(base, scale, (size_t)y * n2 + i, g.nB, kk, pi);
        BIO<B>::template load<double>(base, scale, (size_t)y * n2 + j, g.nB, kk, pj);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const Cx<double> u = pj[c], l = pj[3 + c];
          const Cx<double> w0 = cx(m[0][0], m[0][1]) * u + cx(m[1][0], m[1][1]) * l;
          const Cx<double> w1 = cx(m[2][0], m[2][1]) * u + cx(m[3][0], m[3][1]) * l;
          cfma_conj(acc, pi[c], w0);
          cfma_conj(acc, pi[3 + c], w1);
        }
      }
    }
    out[((size_t)blockIdx.x * n2 + i) * n2 + j] = make_double2(acc.re, acc.im);
  }
}

mglma_status coarse_gamma_level1(mglma_ctx ctx, const mglma_subspace_s* S, int k, double2* out, cudaStream_t s) {
  const BlockGeo& g = S->geo;
  const unsigned blocks = (unsigned)(g.V1 * g.b[0]);
  ProfScope ps(ctx, K_SETUP, s);
  if (S->phi64)
    gamma_level1_kernel<double><<<blocks, 256, 0, s>>>(S->phi64, nullptr, g, S->nv, k, out);
  else if (S->phi16)
    gamma_level1_kernel<__half><<<blocks, 256, 0, s>>>(S->phi16, S->scale16, g, S->nv, k, out);
  else
    gamma_level1_kernel<float><<<blocks, 256, 0, s>>>(S->phi32, nullptr, g, S->nv, k, out);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

template <typename B>
static mglma_status launch_r16(const void* basis, const float* scale, const BlockGeo& g, int nv, const Spinor& in,
                               int threads, unsigned grid, void* out, cudaStream_t s) {
  const int n2 = 2 * nv;
  const size_t smem = std::max(2 * r16_buf<B>(n2) + (size_t)g.nB * sizeof(int64_t),
                               (size_t)threads * 16 * sizeof(float2));
  static std::mutex mu;
  static size_t granted = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (smem > granted) {
      MG_CUDA(cudaFuncSetAttribute(restrict16_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      granted = smem;
    }
  }
  restrict16_kernel<B><<<grid, threads, smem, s>>>((const float4*)in.p, in.nrhs, basis, scale, g, nv, (float2*)out);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

template <typename B>
static mglma_status launch_p16(const void* basis, const float* scale, const BlockGeo& g, int nv, const void* coarse,
                               Spinor& out, bool accumulate, unsigned grid, cudaStream_t s) {
  const size_t smem = 2 * (size_t)T16_TKC * p16_row<B>(2 * nv);
  static std::mutex mu;
  static size_t granted = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (smem > granted) {
      MG_CUDA(cudaFuncSetAttribute(prolong16_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      granted = smem;
    }
  }
  prolong16_kernel<B><<<grid, 256, smem, s>>>((const float2*)coarse, out.nrhs, basis, scale, g, nv, (float4*)out.p,
                                              accumulate ? 1 : 0);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// the many-RHS R0 / T0 kernels: FP32 fields, at least 8 RHS, Nv % 4 == 0 and
// 2 Nv <= 64, FP32 or FP16 basis
static bool use_t16(const mglma_subspace_s* S, int nrhs) {
  return nrhs >= 8 && S->nv % 4 == 0 && 2 * S->nv <= 64 && (S->phi16 || S->phi32);
}

mglma_status restrict_fine(mglma_ctx ctx, const mglma_subspace_s* S, const Spinor& in, void* out_coarse,
                           cudaStream_t s) {
  ProfScope ps(ctx, K_RESTRICT, s, transfer_bytes(S, in.prec, in.nrhs), 8.0 * S->geo.V * 12.0 * S->nv * in.nrhs);
  if (in.prec == MGLMA_FP64) {
    if (S->phi64) return launch_restrict<double, double, 2>(S, in.p, in.nrhs, S->phi64, out_coarse, s);
    if (!S->lean) return fail(MGLMA_ERR_INVALID, "restrict: FP64 needs a subspace stored in FP64");
    if (S->phi16) return launch_restrict<double, __half, 2>(S, in.p, in.nrhs, S->phi16, out_coarse, s);
    return launch_restrict<double, float, 2>(S, in.p, in.nrhs, S->phi32, out_coarse, s);
  }
  if (use_t16(S, in.nrhs)) {
    const BlockGeo g = S->geo;
    const int n2 = 2 * S->nv, ntt = n2;
    const int threads = (T16_MAXT / ntt) * ntt;
    const unsigned grid = (unsigned)(g.V1 * ((in.nrhs + 15) / 16));
    if (S->phi16)
      return launch_r16<__half>(S->phi16, S->scale16, g, S->nv, in, threads, grid, out_coarse, s);
    return launch_r16<float>(S->phi32, nullptr, g, S->nv, in, threads, grid, out_coarse, s);
  }
  if (S->phi16) return launch_restrict<float, __half, 4>(S, in.p, in.nrhs, S->phi16, out_coarse, s);
  return launch_restrict<float, float, 4>(S, in.p, in.nrhs, S->phi32, out_coarse, s);
}

mglma_status prolong_coarse(mglma_ctx ctx, const mglma_subspace_s* S, const void* in_coarse, Spinor& out,
                            bool accumulate, cudaStream_t s) {
  ProfScope ps(ctx, K_PROLONG, s, transfer_bytes(S, out.prec, out.nrhs), 8.0 * S->geo.V * 12.0 * S->nv * out.nrhs);
  if (out.prec == MGLMA_FP64) {
    if (S->phi64) return launch_prolong<double, double, 2>(S, in_coarse, out.nrhs, S->phi64, out.p, accumulate, s);
    if (!S->lean) return fail(MGLMA_ERR_INVALID, "prolong: FP64 needs a subspace stored in FP64");
    if (S->phi16) return launch_prolong<double, __half, 2>(S, in_coarse, out.nrhs, S->phi16, out.p, accumulate, s);
    return launch_prolong<double, float, 2>(S, in_coarse, out.nrhs, S->phi32, out.p, accumulate, s);
  }
  if (use_t16(S, out.nrhs)) {
    const BlockGeo g = S->geo;
    const unsigned grid = (unsigned)(g.V1 * ((out.nrhs + 15) / 16));
    if (S->phi16)
      return launch_p16<__half>(S->phi16, S->scale16, g, S->nv, in_coarse, out, accumulate, grid, s);
    return launch_p16<float>(S->phi32, nullptr, g, S->nv, in_coarse, out, accumulate, grid, s);
  }
  if (S->phi16) return launch_prolong<float, __half, 4>(S, in_coarse, out.nrhs, S->phi16, out.p, accumulate, s);
  return launch_prolong<float, float, 4>(S, in_coarse, out.nrhs, S->phi32, out.p, accumulate, s);
}

// Builds the orthonormal basis from Nv test vectors (internal FP64 layout)
// and fills the storage precisions requested.
static mglma_status finish_basis(mglma_ctx ctx, mglma_subspace_s* S, const Spinor& vecs, cudaStream_t s) {
  const BlockGeo g = S->geo;
  const int nv = S->nv;
  const size_t nyj = (size_t)g.V1 * 2 * nv;
  double2* p64 = nullptr;
  MG_CUDA(cudaMalloc(&p64, nyj * 6 * g.nB * sizeof(double2)));
  split_kernel<<<dim3((unsigned)g.V1, 2 * nv, 1), 128, 0, s>>>((const double2*)vecs.p, nv, g, p64);
  MG_LAUNCH_CHECK();
  int* flag = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&flag, sizeof(int), s));
  MG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  const int smem = (2 * nv * nv + GS_TR * nv) * (int)sizeof(double2);
  cudaFuncSetAttribute(cholqr2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  {
    ProfScope ps(ctx, K_SETUP, s);
    cholqr2_kernel<<<dim3((unsigned)g.V1, 2, 1), GS_THREADS, smem, s>>>(p64, nv, g, 1e-6, flag);
  }
  MG_LAUNCH_CHECK();
  int hflag = 0;
  MG_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  dfree(ctx, flag, s);
  MG_CUDA(cudaStreamSynchronize(s));
  if (hflag) {
    cudaFree(p64);
    return fail(MGLMA_ERR_RANK, "subspace: a block basis vector is linearly dependent on earlier ones");
  }
  const size_t n3 = nyj * 3 * g.nB;
  MG_CUDA(cudaMalloc(&S->phi32, n3 * sizeof(float4)));
  basis_to32_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(p64, S->phi32, nyj, g.nB);
  MG_LAUNCH_CHECK();
  if (S->store == MGLMA_FP16) {
    MG_CUDA(cudaMalloc(&S->scale16, nyj * sizeof(float)));
    MG_CUDA(cudaMalloc(&S->phi16, n3 * sizeof(uint2)));
    basis_scale_kernel<<<(unsigned)nyj, 128, 0, s>>>(p64, S->scale16, g.nB);
    basis_to16_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(p64, S->scale16, S->phi16, nyj, g.nB);
    MG_LAUNCH_CHECK();
  }
  S->phi64 = p64;  // kept until the coarse operator is built (or for good with FP64 storage)
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

mglma_status cg_relax(mglma_ctx ctx, const mglma_gauge_s* G, Spinor& v, int n_cg, cudaStream_t s);

// Lean variant: test vectors in FP32; CholeskyQR2 in FP64 on chunks of
// blocks; only the store copy (FP32 or FP16 + scales) is kept.
static mglma_status finish_basis_lean(mglma_ctx ctx, mglma_subspace_s* S, const Spinor& vecs, cudaStream_t s) {
  const BlockGeo g = S->geo;
  const int nv = S->nv;
  const size_t nyj = (size_t)g.V1 * 2 * nv;
  const size_t n3 = nyj * 3 * g.nB;
  const bool half = S->store == MGLMA_FP16;
  if (half) {
    MG_CUDA(cudaMalloc(&S->scale16, nyj * sizeof(float)));
    MG_CUDA(cudaMalloc(&S->phi16, n3 * sizeof(uint2)));
  } else {
    MG_CUDA(cudaMalloc(&S->phi32, n3 * sizeof(float4)));
  }
  // chunks of blocks whose FP64 copy takes at most 1 GiB
  const size_t per_block = (size_t)2 * nv * 6 * g.nB * sizeof(double2);
  const int64_t cb = std::max<int64_t>(1, std::min<int64_t>(g.V1, ((size_t)1 << 30) / per_block));
  FreeList fl(ctx, s);
  double2* p64 = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&p64, (size_t)cb * per_block, s));
  fl.add(p64);
  int* flag = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&flag, sizeof(int), s));
  fl.add(flag);
  MG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  const int smem = (2 * nv * nv + GS_TR * nv) * (int)sizeof(double2);
  cudaFuncSetAttribute(cholqr2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  for (int64_t y0 = 0; y0 < g.V1; y0 += cb) {
    const int64_t nyc = std::min<int64_t>(cb, g.V1 - y0);
    ProfScope ps(ctx, K_SETUP, s);
    split32_kernel<<<dim3((unsigned)nyc, 2 * nv, 1), 128, 0, s>>>((const float4*)vecs.p, nv, g, y0, p64);
    cholqr2_kernel<<<dim3((unsigned)nyc, 2, 1), GS_THREADS, smem, s>>>(p64, nv, g, 1e-6, flag);
    const size_t cyj = (size_t)nyc * 2 * nv, c3 = cyj * 3 * g.nB, off = (size_t)y0 * 2 * nv;
    if (half) {
      basis_scale_kernel<<<(unsigned)cyj, 128, 0, s>>>(p64, S->scale16 + off, g.nB);
      basis_to16_kernel<<<(unsigned)((c3 + 255) / 256), 256, 0, s>>>(p64, S->scale16 + off,
                                                                     S->phi16 + off * 3 * g.nB, cyj, g.nB);
    } else {
      basis_to32_kernel<<<(unsigned)((c3 + 255) / 256), 256, 0, s>>>(p64, S->phi32 + off * 3 * g.nB, cyj, g.nB);
    }
    MG_LAUNCH_CHECK();
  }
  int hflag = 0;
  MG_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  if (hflag) return fail(MGLMA_ERR_RANK, "subspace: a block basis vector is linearly dependent on earlier ones");
  return MGLMA_OK;
}

// Lean set-up: FP32 test vectors relaxed `group` at a time in place.
static mglma_status build_lean(mglma_ctx ctx, const mglma_gauge_s* G, mglma_subspace_s* S,
                               const mglma_subspace_params* prm, uint64_t key, cudaStream_t s) {
  const int nv = S->nv, grp = prm->lean_group;
  Spinor all;
  FreeList fl(ctx, s);
  MG_CHECK(alloc_spinor(ctx, all, MGLMA_FP32, nv, G->g.V, s));
  fl.add(all.p);
  for (int c0 = 0; c0 < nv; c0 += grp) {
    Spinor v = all;
    v.nrhs = std::min(grp, nv - c0);
    v.p = static_cast<float*>(all.p) + (size_t)c0 * all.rhs_reals();
    random_starts32_kernel<<<dim3((unsigned)((G->g.V + 127) / 128), v.nrhs, 1), 128, 0, s>>>(
        (float4*)v.p, G->g.V, v.nrhs, c0, key);
    MG_LAUNCH_CHECK();
    MG_CHECK(mr_smooth(ctx, G, v, prm->n_smooth, s));
    MG_CHECK(cg_relax(ctx, G, v, prm->n_cg, s));
  }
  return finish_basis_lean(ctx, S, all, s);
}

mglma_status mr_smooth(mglma_ctx ctx, const mglma_gauge_s* G, Spinor& v, int n_smooth, cudaStream_t s) {
  const int n = v.nrhs;
  FreeList fr(ctx, s);
  Spinor r, w;
  MG_CHECK(alloc_spinor(ctx, r, v.prec, n, v.V, s));
  fr.add(r.p);
  MG_CHECK(alloc_spinor(ctx, w, v.prec, n, v.V, s));
  fr.add(w.p);
  Scalars sc;
  MG_CHECK(sc.alloc(ctx, n, 1, 1, s));
  Vec vv = as_vec(v), vr = as_vec(r), vw = as_vec(w);
  // r = -D v
  MG_CHECK(dslash(ctx, G, v, r, false, false, s));
  MG_CHECK(axpby(ctx, nullptr, C0, vr, nullptr, CM1, vr, s));
  for (int it = 0; it < n_smooth; ++it) {
    MG_CHECK(dslash(ctx, G, r, w, false, false, s));
    MG_CHECK(cdot(ctx, vw, vr, sc.z, s));  // <D r, r>
    MG_CHECK(norm2(ctx, vw, sc.d, s));     // <D r, D r>
    MG_CHECK(mr_alpha(ctx, sc.z, sc.d, sc.z, n, s));
    MG_CHECK(axpy2(ctx, sc.z, vr, vv, vw, vr, s));  // v += a r ; r -= a D r
  }
  return MGLMA_OK;
}

// n_cg CG steps on the normal equations of D x = 0 from x0 = v, all RHS of v
// at once, fixed step count (no host synchronisation).
mglma_status cg_relax(mglma_ctx ctx, const mglma_gauge_s* G, Spinor& v, int n_cg, cudaStream_t s) {
  if (n_cg <= 0) return MGLMA_OK;
  const int n = v.nrhs;
  FreeList fr(ctx, s);
  Spinor r, z, p, w;
  for (Spinor* f : {&r, &z, &p, &w}) {
    MG_CHECK(alloc_spinor(ctx, *f, v.prec, n, v.V, s));
    fr.add(f->p);
  }
  Scalars sc;
  MG_CHECK(sc.alloc(ctx, n, 3, 2, s));
  double *zz = sc.d, *zzn = sc.d + n, *ww = sc.d + 2 * n;
  double2 *alpha = sc.z, *beta = sc.z + n;
  Vec vv = as_vec(v), vr = as_vec(r), vz = as_vec(z), vp = as_vec(p), vw = as_vec(w);
  MG_CHECK(dslash(ctx, G, v, r, false, false, s));
  MG_CHECK(axpby(ctx, nullptr, C0, vr, nullptr, CM1, vr, s));  // r = -D v
  MG_CHECK(dslash(ctx, G, r, z, true, false, s));
  MG_CHECK(copy_vec(ctx, vz, vp, s));
  MG_CHECK(norm2(ctx, vz, zz, s));
  for (int it = 0; it < n_cg; ++it) {
    MG_CHECK(dslash(ctx, G, p, w, false, false, s));
    MG_CHECK(norm2(ctx, vw, ww, s));
    MG_CHECK(cg_scalars(ctx, zz, ww, alpha, sc.active, n, s));
    MG_CHECK(axpy2(ctx, alpha, vp, vv, vw, vr, s));
    MG_CHECK(dslash(ctx, G, r, z, true, false, s));
    MG_CHECK(norm2(ctx, vz, zzn, s));
    MG_CHECK(cg_beta(ctx, zzn, zz, beta, sc.active, n, s));
    MG_CHECK(axpby(ctx, nullptr, C1, vz, beta, C0, vp, s));
  }
  return MGLMA_OK;
}

}  // namespace mglma

using namespace mglma;

extern "C" {

static mglma_status subspace_common(mglma_ctx ctx, mglma_gauge G, const int block[4], int nv, mglma_prec store,
                                    mglma_subspace_s** out) {
  if (!ctx || !G || !block || !out) return fail(MGLMA_ERR_INVALID, "subspace: NULL argument");
  if (!G->ready) return fail(MGLMA_ERR_INVALID, "subspace: gauge field incomplete");
  if (nv < 1 || 2 * nv > 128) return fail(MGLMA_ERR_INVALID, "subspace: need 1 <= nv <= 64");
  if (store != MGLMA_FP64 && store != MGLMA_FP32 && store != MGLMA_FP16)
    return fail(MGLMA_ERR_INVALID, "subspace: store must be FP64, FP32 or FP16");
  int nB = 1;
  for (int m = 0; m < 4; ++m) {
    if (block[m] < 1 || G->g.L[m] % block[m]) return fail(MGLMA_ERR_INVALID, "subspace: block sides must divide L");
    nB *= block[m];
  }
  if (6 * nB < nv) return fail(MGLMA_ERR_RANK, "subspace: block too small for nv vectors per chirality");
  mglma_subspace_s* S = new mglma_subspace_s();
  S->ctx = ctx;
  S->gauge = G;
  S->nv = nv;
  S->store = store;
  S->geo = make_blockgeo(G->g.L, block);
  *out = S;
  return MGLMA_OK;
}

mglma_status mglma_subspace_build(mglma_ctx ctx, mglma_gauge G, const int block[4], int nv, int n_smooth,
                                  uint64_t seed, mglma_prec store, mglma_subspace* out) {
  if (!block) return fail(MGLMA_ERR_INVALID, "subspace: NULL block");
  mglma_subspace_params p;
  for (int m = 0; m < 4; ++m) p.block[m] = block[m];
  p.nv = nv;
  p.n_smooth = n_smooth;
  p.n_cg = 0;
  p.cg_prec = MGLMA_FP64;
  p.seed = seed;
  p.store = store;
  p.lean_group = 0;
  return mglma_subspace_create(ctx, G, &p, out);
}

mglma_status mglma_subspace_create(mglma_ctx ctx, mglma_gauge G, const mglma_subspace_params* prm,
                                   mglma_subspace* out) {
  if (!prm) return fail(MGLMA_ERR_INVALID, "subspace: NULL parameters");
  const int* block = prm->block;
  const int nv = prm->nv, n_smooth = prm->n_smooth;
  const uint64_t seed = prm->seed;
  const mglma_prec store = (mglma_prec)prm->store;
  mglma_subspace_s* S = nullptr;
  MG_CHECK(subspace_common(ctx, G, block, nv, store, &S));
  if (n_smooth < 0 || prm->n_cg < 0 || (prm->cg_prec != MGLMA_FP64 && prm->cg_prec != MGLMA_FP32)) {
    delete S;
    return fail(MGLMA_ERR_INVALID, "subspace: bad smoothing parameters");
  }
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const uint64_t key = [&] {
    // key = mix64(mix64(seed) ^ tag), tag 3 = start vectors
    auto h = [](uint64_t z) {
      z += 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    return h(h(seed) ^ 3ull);
  }();
  if (prm->lean_group != 0) {
    if (prm->lean_group < 0 || (store != MGLMA_FP32 && store != MGLMA_FP16)) {
      delete S;
      return fail(MGLMA_ERR_INVALID, "subspace: the lean set-up needs lean_group > 0 and store FP32 or FP16");
    }
    S->lean = true;
    mglma_status st = build_lean(ctx, G, S, prm, key, s);
    cudaStreamSynchronize(s);
    cudaMemPoolTrimTo(ctx->pool, 0);  // hand the set-up's work fields back to the device
    if (st != MGLMA_OK) {
      mglma_subspace_free(S);
      return st;
    }
    *out = S;
    return MGLMA_OK;
  }
  Spinor v;
  mglma_status st = alloc_spinor(ctx, v, MGLMA_FP64, nv, G->g.V, s);
  if (st == MGLMA_OK) {
    random_starts_kernel<<<dim3((unsigned)((G->g.V + 127) / 128), nv, 1), 128, 0, s>>>((double2*)v.p, G->g.V, nv,
                                                                                       key);
    if (cudaGetLastError() != cudaSuccess) st = fail(MGLMA_ERR_CUDA, "random starts launch failed");
  }
  if (st == MGLMA_OK) st = mr_smooth(ctx, G, v, n_smooth, s);
  if (st == MGLMA_OK && prm->n_cg > 0) {
    if (prm->cg_prec == MGLMA_FP64) {
      st = cg_relax(ctx, G, v, prm->n_cg, s);
    } else {
      Spinor v32;
      st = alloc_spinor(ctx, v32, MGLMA_FP32, nv, G->g.V, s);
      if (st == MGLMA_OK) st = convert_spinor(ctx, v, v32, s);
      if (st == MGLMA_OK) st = cg_relax(ctx, G, v32, prm->n_cg, s);
      if (st == MGLMA_OK) st = convert_spinor(ctx, v32, v, s);
      dfree(ctx, v32.p, s);
    }
  }
  if (st == MGLMA_OK) st = finish_basis(ctx, S, v, s);
  dfree(ctx, v.p, s);
  cudaStreamSynchronize(s);
  cudaMemPoolTrimTo(ctx->pool, 0);  // hand the set-up's work fields back to the device
  if (st != MGLMA_OK) {
    mglma_subspace_free(S);
    return st;
  }
  *out = S;
  return MGLMA_OK;
}

mglma_status mglma_subspace_load(mglma_ctx ctx, mglma_gauge G, const int block[4], int nv, const double* vecs,
                                 mglma_prec store, mglma_subspace* out) {
  if (!vecs) return fail(MGLMA_ERR_INVALID, "subspace_load: NULL vectors");
  mglma_subspace_s* S = nullptr;
  MG_CHECK(subspace_common(ctx, G, block, nv, store, &S));
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  Spinor v;
  const size_t bytes = (size_t)nv * G->g.V * 24 * sizeof(double);
  mglma_status st;
  {
    Staged in;
    st = stage_in(ctx, vecs, bytes, s, in);
    if (st == MGLMA_OK) st = alloc_spinor(ctx, v, MGLMA_FP64, nv, G->g.V, s);
    if (st == MGLMA_OK) st = pack_spinor(ctx, in.dev, v, s);
    if (st == MGLMA_OK) st = finish_basis(ctx, S, v, s);
    dfree(ctx, v.p, s);
  }
  if (st != MGLMA_OK) {
    mglma_subspace_free(S);
    return st;
  }
  *out = S;
  return MGLMA_OK;
}

void mglma_subspace_free(mglma_subspace S) {
  if (!S) return;
  if (S->ctx) cudaSetDevice(S->ctx->device);
  cudaFree(S->phi64);
  cudaFree(S->phi32);
  cudaFree(S->phi16);
  cudaFree(S->scale16);
  cudaFree(S->rt_img);
  cudaFree(S->pt_img);
  cudaFree(S->rt_err);
  delete S;
}

mglma_status mglma_subspace_info(mglma_subspace S, int* nv, int Lb[4], int64_t* coarse_volume) {
  if (!S) return fail(MGLMA_ERR_INVALID, "subspace_info: NULL handle");
  if (nv) *nv = S->nv;
  if (Lb)
    for (int m = 0; m < 4; ++m) Lb[m] = S->geo.Lb[m];
  if (coarse_volume) *coarse_volume = S->geo.V1;
  return MGLMA_OK;
}

mglma_status mglma_subspace_export(mglma_subspace S, double* phi) {
  if (!S || !phi) return fail(MGLMA_ERR_INVALID, "subspace_export: NULL argument");
  if (!S->phi64 && !S->lean)
    return fail(MGLMA_ERR_INVALID, "subspace_export: FP64 basis released (store FP64 keeps it)");
  mglma_ctx ctx = S->ctx;
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const size_t nyj = (size_t)S->geo.V1 * 2 * S->nv;
  const size_t bytes = nyj * S->geo.nB * 12 * sizeof(double2);
  Staged o;
  MG_CHECK(stage_out_alloc(ctx, phi, bytes, s, o));
  const size_t n = nyj * S->geo.nB;
  const double2* src = S->phi64;
  FreeList fl(ctx, s);
  if (!src) {  // lean: widen the stored copy
    double2* w = nullptr;
    MG_CHECK(dalloc(ctx, (void**)&w, n * 6 * sizeof(double2), s));
    fl.add(w);
    if (S->phi16)
      basis_widen_kernel<__half><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S->phi16, S->scale16, w, nyj, S->geo.nB);
    else
      basis_widen_kernel<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S->phi32, nullptr, w, nyj, S->geo.nB);
    src = w;
  }
  basis_export_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, (double2*)o.dev, S->nv, S->geo.nB, nyj);
  MG_LAUNCH_CHECK();
  MG_CHECK(stage_out_finish(phi, bytes, s, o));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

static mglma_status transfer(mglma_ctx ctx, mglma_subspace S, int nrhs, const double* in, double* out,
                             mglma_prec compute, void* stream, bool to_coarse) {
  if (!ctx || !S || !in || !out) return fail(MGLMA_ERR_INVALID, "restrict/prolong: NULL argument");
  if (compute != MGLMA_FP64 && compute != MGLMA_FP32 && compute != MGLMA_BF16)
    return fail(MGLMA_ERR_INVALID, "restrict/prolong: compute must be FP64, FP32 or BF16");
  if (compute == MGLMA_BF16 && to_coarse && !restrict_tc_supported(S))
    return fail(MGLMA_ERR_INVALID, "restrict: the BF16 tensor-core path needs Nv % 8 == 0, Nv <= 32, 64 | |B| <= 512");
  if (compute == MGLMA_BF16 && !to_coarse && !prolong_tc_supported(S))
    return fail(MGLMA_ERR_INVALID, "prolong: the BF16 tensor-core path needs Nv % 8 == 0, Nv <= 32, 128 | |B| <= 512");
  // BF16: the tensor-core R0 / T0 on FP32 fields
  const bool tc = compute == MGLMA_BF16;
  if (tc) compute = MGLMA_FP32;
  if (nrhs <= 0) return nrhs == 0 ? MGLMA_OK : fail(MGLMA_ERR_INVALID, "restrict/prolong: nrhs < 0");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, stream);
  const int64_t V = S->geo.V, V1 = S->geo.V1;
  const int n2 = 2 * S->nv;
  const size_t fb = (size_t)nrhs * V * 24 * sizeof(double), cb = (size_t)nrhs * V1 * n2 * sizeof(double2);
  Staged si, so;
  MG_CHECK(stage_in(ctx, in, to_coarse ? fb : cb, s, si));
  MG_CHECK(stage_out_alloc(ctx, out, to_coarse ? cb : fb, s, so));
  FreeList fr(ctx, s);
  Spinor f;
  MG_CHECK(alloc_spinor(ctx, f, compute, nrhs, V, s));
  fr.add(f.p);
  void* c = nullptr;
  const int rb = compute == MGLMA_FP64 ? 16 : 8;
  MG_CHECK(dalloc(ctx, &c, (size_t)nrhs * V1 * n2 * rb, s));
  fr.add(c);
  if (to_coarse) {
    MG_CHECK(pack_spinor(ctx, si.dev, f, s));
    if (tc) {
      MG_CHECK(restrict_tc(ctx, S, f, c, s));
      MG_CHECK(restrict_tc_check(S, s));
    } else {
      MG_CHECK(restrict_fine(ctx, S, f, c, s));
    }
    MG_CHECK(coarse_to_canonical(ctx, c, compute, (size_t)nrhs * V1 * n2, so.dev, s));
  } else {
    MG_CHECK(coarse_from_canonical(ctx, si.dev, (size_t)nrhs * V1 * n2, c, compute, s));
    if (tc) {
      MG_CHECK(prolong_tc(ctx, S, c, f, s));
      MG_CHECK(restrict_tc_check(S, s));
    } else {
      MG_CHECK(prolong_coarse(ctx, S, c, f, false, s));
    }
    MG_CHECK(unpack_spinor(ctx, f, so.dev, s));
  }
  MG_CHECK(stage_out_finish(out, to_coarse ? cb : fb, s, so));
  return MGLMA_OK;
}

mglma_status mglma_restrict(mglma_ctx ctx, mglma_subspace S, int nrhs, const double* in, double* out,
                            mglma_prec compute, void* cuda_stream) {
  return transfer(ctx, S, nrhs, in, out, compute, cuda_stream, true);
}

mglma_status mglma_prolong(mglma_ctx ctx, mglma_subspace S, int nrhs, const double* in, double* out,
                           mglma_prec compute, void* cuda_stream) {
  return transfer(ctx, S, nrhs, in, out, compute, cuda_stream, false);
}

}  // extern "C"
