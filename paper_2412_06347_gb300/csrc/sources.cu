// Sources for the propagator solves (Sec. 5, stochastic estimator): Z2 and
// Z4 noise ({+-1 +- i}/sqrt 2, the paper's choice) from the counter-based
// generator, point sources, and optional time dilution (support on one time
// slice, the paper's time-diluted wall sources).
//
// Counter definition (shared with the Python input generators): stream key =
// mix64(mix64(seed) ^ 2); component (spin s, colour c) of RHS g at site x
// uses draw mix64(key + (g V + x) 12 + 3 s + c); bit 63 gives the sign of the
// real part, bit 62 the sign of the imaginary part (Z4).
#include <cmath>
#include <vector>

#include "internal.h"

namespace mglma {

__host__ __device__ inline uint64_t src_mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void noise_kernel(double2* __restrict__ out, int64_t V, int64_t slice, int nrhs, uint64_t key, int64_t first,
                             int z4, int t_slice) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // site*12 + sc
  const int r = blockIdx.y;
  if (i >= V * 12 || r >= nrhs) return;
  const int64_t site = i / 12;
  double2 v = make_double2(0.0, 0.0);
  if (t_slice < 0 || site / slice == t_slice) {
    const uint64_t n = (uint64_t)((first + r) * V) * 12 + (uint64_t)i;
    const uint64_t z = src_mix64(key + n);
    const double re = (z >> 63) ? -1.0 : 1.0;
    if (z4) {
      const double im = ((z >> 62) & 1) ? -1.0 : 1.0;
      const double s2 = sqrt(2.0);  // correctly rounded, as on the host
      v = make_double2(re / s2, im / s2);
    } else {
      v = make_double2(re, 0.0);
    }
  }
  out[(size_t)r * V * 12 + i] = v;
}

}  // namespace mglma

using namespace mglma;

extern "C" mglma_status mglma_sources(mglma_ctx ctx, const mglma_lattice* lat, int kind, int nrhs, uint64_t seed,
                                      int64_t first, const int64_t* point_sites, const int* point_sc, int t_slice,
                                      double* out, void* cuda_stream) {
  if (!ctx || !lat || !out) return fail(MGLMA_ERR_INVALID, "sources: NULL argument");
  if (nrhs < 0 || first < 0) return fail(MGLMA_ERR_INVALID, "sources: negative count");
  if (kind < MGLMA_SOURCE_Z2 || kind > MGLMA_SOURCE_POINT) return fail(MGLMA_ERR_INVALID, "sources: bad kind");
  int64_t V = 1;
  for (int m = 0; m < 4; ++m) {
    if (lat->L[m] < 1) return fail(MGLMA_ERR_INVALID, "sources: bad extent");
    V *= lat->L[m];
  }
  if (t_slice >= lat->L[0]) return fail(MGLMA_ERR_INVALID, "sources: time slice outside the lattice");
  if (nrhs == 0) return MGLMA_OK;
  if (kind == MGLMA_SOURCE_POINT) {
    if (!point_sites || !point_sc) return fail(MGLMA_ERR_INVALID, "sources: point sources need sites and columns");
    for (int r = 0; r < nrhs; ++r)
      if (point_sites[r] < 0 || point_sites[r] >= V || point_sc[r] < 0 || point_sc[r] >= 12)
        return fail(MGLMA_ERR_INVALID, "sources: point site or spin-colour out of range");
  }
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, cuda_stream);
  const size_t bytes = (size_t)nrhs * V * 24 * sizeof(double);
  Staged o;
  MG_CHECK(stage_out_alloc(ctx, out, bytes, s, o));
  const int64_t slice = V / lat->L[0];
  if (kind == MGLMA_SOURCE_POINT) {
    MG_CUDA(cudaMemsetAsync(o.dev, 0, bytes, s));
    const double one = 1.0;
    for (int r = 0; r < nrhs; ++r) {
      if (t_slice >= 0 && point_sites[r] / slice != t_slice) continue;
      double* p = o.dev + ((size_t)r * V + point_sites[r]) * 24 + 2 * point_sc[r];
      MG_CUDA(cudaMemcpyAsync(p, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    }
  } else {
    const uint64_t key = src_mix64(src_mix64(seed) ^ 2ull);
    ProfScope ps(ctx, K_PACK, s);
    dim3 g((unsigned)((V * 12 + 255) / 256), (unsigned)nrhs, 1);
    noise_kernel<<<g, 256, 0, s>>>((double2*)o.dev, V, slice, nrhs, key, first, kind == MGLMA_SOURCE_Z4 ? 1 : 0,
                                   t_slice);
    MG_LAUNCH_CHECK();
  }
  MG_CHECK(stage_out_finish(out, bytes, s, o));
  return MGLMA_OK;
}
