// Halo-free periodic indexing on the canonical lexicographic site order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mglma {

struct LatIdx {
  int L[4];
  int64_t S[4];  // strides: S3 = 1, S2 = L3, S1 = L2 L3, S0 = L1 L2 L3
  int64_t V;
};

inline LatIdx make_latidx(const int L[4]) {
  LatIdx q;
  for (int m = 0; m < 4; ++m) q.L[m] = L[m];
  q.S[3] = 1;
  q.S[2] = L[3];
  q.S[1] = (int64_t)L[2] * L[3];
  q.S[0] = (int64_t)L[1] * L[2] * L[3];
  q.V = q.S[0] * L[0];
  return q;
}

__device__ __forceinline__ void site_coords(const LatIdx& q, int64_t site, int x[4]) {
  int64_t t = site;
  x[3] = (int)(t % q.L[3]);
  t /= q.L[3];
  x[2] = (int)(t % q.L[2]);
  t /= q.L[2];
  x[1] = (int)(t % q.L[1]);
  x[0] = (int)(t / q.L[1]);
}

// neighbour of `site` (coordinates x) one step in +mu / -mu, periodic
__device__ __forceinline__ int64_t nbr_fwd(const LatIdx& q, int64_t site, const int x[4], int mu) {
  return x[mu] == q.L[mu] - 1 ? site - (int64_t)(q.L[mu] - 1) * q.S[mu] : site + q.S[mu];
}
__device__ __forceinline__ int64_t nbr_bwd(const LatIdx& q, int64_t site, const int x[4], int mu) {
  return x[mu] == 0 ? site + (int64_t)(q.L[mu] - 1) * q.S[mu] : site - q.S[mu];
}

// site x + a*mu + b*nu for a, b in {-1, 0, 1}
__device__ __forceinline__ int64_t shifted(const LatIdx& q, const int x[4], int mu, int a, int nu, int b) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] = (y[mu] + a + q.L[mu]) % q.L[mu];
  y[nu] = (y[nu] + b + q.L[nu]) % q.L[nu];
  return ((int64_t)y[0] * q.L[1] + y[1]) * q.L[2] * (int64_t)q.L[3] + (int64_t)y[2] * q.L[3] + y[3];
}

}  // namespace mglma
