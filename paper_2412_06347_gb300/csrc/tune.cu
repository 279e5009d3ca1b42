// Autotuner of the RHS tile widths: the stencil's tile shape (RHS per thread
// 1, 2, 4 times RHS tiles per CTA 1, 2, 4, or the staged-tile kernel with 4, 8
// or 16 RHS per CTA) and the tensor-core coarse
// kernel's RHS per tile (8, 16, 32) are timed with
// CUDA events on the context stream for a given RHS count, and the fastest
// is kept per (kernel, RHS bucket, lattice volume) in the context; the table
// can be saved to and loaded from a text file keyed by GPU name.  The solver
// tunes the shapes of a (lattice, RHS bucket) on its first batch
// (autotune_for_batch); with MGLMA_TUNE_CACHE naming a file, a context loads
// that file when created and saves the table after each automatic tuning.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <sstream>
#include <string>
#include <tuple>

#include "internal.h"
#include "solver.h"
#include "subspace.h"

namespace mglma {

static mglma_status time_ms(mglma_ctx ctx, cudaStream_t s, int reps, const std::function<mglma_status()>& f,
                            double* ms) {
  cudaEvent_t a, b;
  MG_CUDA(cudaEventCreate(&a));
  MG_CUDA(cudaEventCreate(&b));
  mglma_status st = f();  // warm-up
  if (st == MGLMA_OK) {
    cudaEventRecord(a, s);
    for (int i = 0; i < reps && st == MGLMA_OK; ++i) st = f();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float t = 0;
    cudaEventElapsedTime(&t, a, b);
    *ms = t / reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  (void)ctx;
  return st;
}

static std::string gpu_name(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string n = p.name;
  for (auto& c : n)
    if (c == ' ') c = '_';
  return n;
}

// Tunes the tile shapes of this (lattice, RHS bucket) unless the context
// holds them already, and saves the table to the context's cache file.
mglma_status autotune_for_batch(mglma_ctx ctx, mglma_gauge_s* G, mglma_coarse_s* C, int nrhs) {
  const bool need_d = !has_tuned(ctx, TUNE_DSLASH32_NR, nrhs, G->g.V);
  const bool need_c = C && C->Aimg && !has_tuned(ctx, TUNE_COARSE_NT, nrhs, C->geo.V1);
  if (!need_d && !need_c) return MGLMA_OK;
  MG_CHECK(mglma_autotune(ctx, need_d ? G : nullptr, need_c ? C : nullptr, nrhs));
  if (!ctx->tune_cache.empty()) mglma_autotune_save(ctx, ctx->tune_cache.c_str());  // best effort
  return MGLMA_OK;
}

}  // namespace mglma

using namespace mglma;

extern "C" {

mglma_status mglma_autotune(mglma_ctx ctx, mglma_gauge G, mglma_coarse C, int nrhs) {
  if (!ctx || nrhs < 1) return fail(MGLMA_ERR_INVALID, "autotune: bad arguments");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const bool prof = ctx->profile;
  ctx->profile = false;
  const int bucket = rhs_bucket(nrhs);
  mglma_status st = MGLMA_OK;
  const auto key_d = std::make_tuple((int)TUNE_DSLASH32_NR, bucket, G ? G->g.V : (int64_t)0);
  const auto key_c = std::make_tuple((int)TUNE_COARSE_NT, bucket, C ? C->geo.V1 : (int64_t)0);
  if (G && G->ready) {
    Spinor a, b;
    FreeList fl(ctx, s);
    st = alloc_spinor(ctx, a, MGLMA_FP32, nrhs, G->g.V, s);
    if (st == MGLMA_OK) st = alloc_spinor(ctx, b, MGLMA_FP32, nrhs, G->g.V, s);
    fl.add(a.p);
    fl.add(b.p);
    if (st == MGLMA_OK) MG_CUDA(cudaMemsetAsync(a.p, 0, a.bytes(), s));
    double best = 1e30;
    int choice = 1;
    // {NR, RW} of the one-site-per-thread kernel; {0, NRT} the staged-tile kernel
    const int shapes[][2] = {{1, 1}, {2, 1}, {4, 1}, {1, 2}, {1, 4}, {2, 2}, {2, 4}, {0, 4}, {0, 8}, {0, 16}};
    for (const auto& sh : shapes) {
      if (st != MGLMA_OK) break;
      const int width = sh[0] ? sh[0] * sh[1] : sh[1];
      if (width > 1 && width > nrhs) continue;  // tiles mostly idle
      const int code = sh[0] ? dslash32_tile_code(sh[0], sh[1]) : 64 + sh[1];
      ctx->tune[key_d] = {code, 0.0};
      double ms = 0;
      st = time_ms(ctx, s, 5, [&] { return dslash(ctx, G, a, b, false, false, s); }, &ms);
      if (st == MGLMA_OK && ms < best) {
        best = ms;
        choice = code;
      }
    }
    ctx->tune[key_d] = {choice, best};
  }
  if (st == MGLMA_OK && C && C->Aimg) {
    const size_t n = (size_t)nrhs * C->geo.V1 * C->n2;
    FreeList fl(ctx, s);
    void *X = nullptr, *Y = nullptr;
    st = dalloc(ctx, &X, n * sizeof(float2), s);
    if (st == MGLMA_OK) st = dalloc(ctx, &Y, n * sizeof(float2), s);
    fl.add(X);
    fl.add(Y);
    if (st == MGLMA_OK) MG_CUDA(cudaMemsetAsync(X, 0, n * sizeof(float2), s));
    double best = 1e30;
    int choice = 8;
    for (int nt : {8, 16, 32}) {
      if (st != MGLMA_OK || (nt > 8 && nt >= 2 * nrhs)) break;  // tiles mostly padding
      ctx->tune[key_c] = {nt, 0.0};
      double ms = 0;
      st = time_ms(ctx, s, 5, [&] { return coarse_apply(ctx, C, X, Y, nrhs, MGLMA_FP32, CMODE_D, s); }, &ms);
      if (st == MGLMA_OK && ms < best) {
        best = ms;
        choice = nt;
      }
    }
    ctx->tune[key_c] = {choice, best};
    if (st == MGLMA_OK) st = coarse_tc_check(C, s);
  }
  ctx->profile = prof;
  return st;
}

mglma_status mglma_autotune_get(mglma_ctx ctx, int kernel, int nrhs, int* choice, double* ms) {
  if (!ctx) return fail(MGLMA_ERR_INVALID, "autotune_get: NULL context");
  if (choice) *choice = 0;
  if (ms) *ms = 0;
  // the entry set for every lattice (volume 0), else the one of the largest
  // tuned lattice (the map is ordered by volume within a kernel and bucket)
  const int b = rhs_bucket(nrhs);
  const std::pair<int, double>* hit = nullptr;
  for (auto& kv : ctx->tune) {
    if (std::get<0>(kv.first) != kernel || std::get<1>(kv.first) != b) continue;
    if (std::get<2>(kv.first) == 0) {
      hit = &kv.second;
      break;
    }
    hit = &kv.second;
  }
  if (hit) {
    if (choice) *choice = hit->first;
    if (ms) *ms = hit->second;
  }
  return MGLMA_OK;
}

mglma_status mglma_autotune_set(mglma_ctx ctx, int kernel, int nrhs, int choice) {
  if (!ctx || nrhs < 1) return fail(MGLMA_ERR_INVALID, "autotune_set: bad arguments");
  const bool ok = (kernel == TUNE_DSLASH32_NR && dslash32_tile_valid(choice)) ||
                  (kernel == TUNE_COARSE_NT && (choice == 8 || choice == 16 || choice == 32));
  if (!ok) return fail(MGLMA_ERR_INVALID, "autotune_set: unknown kernel or choice");
  ctx->tune[std::make_tuple(kernel, rhs_bucket(nrhs), (int64_t)0)] = {choice, 0.0};
  return MGLMA_OK;
}

mglma_status mglma_autotune_save(mglma_ctx ctx, const char* path) {
  if (!ctx || !path) return fail(MGLMA_ERR_INVALID, "autotune_save: NULL argument");
  std::ofstream f(path);
  if (!f) return fail(MGLMA_ERR_INVALID, std::string("autotune_save: cannot write ") + path);
  const std::string gpu = gpu_name(ctx->device);
  for (auto& kv : ctx->tune)
    f << gpu << ' ' << std::get<0>(kv.first) << ' ' << std::get<1>(kv.first) << ' ' << std::get<2>(kv.first) << ' '
      << kv.second.first << ' ' << kv.second.second << '\n';
  return MGLMA_OK;
}

mglma_status mglma_autotune_load(mglma_ctx ctx, const char* path) {
  if (!ctx || !path) return fail(MGLMA_ERR_INVALID, "autotune_load: NULL argument");
  std::ifstream f(path);
  if (!f) return fail(MGLMA_ERR_INVALID, std::string("autotune_load: cannot read ") + path);
  const std::string gpu = gpu_name(ctx->device);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string g;
    int k, b, c;
    long long vol;
    double ms;
    if (!(is >> g >> k >> b >> vol >> c >> ms) || g != gpu) continue;
    const bool ok = (k == TUNE_DSLASH32_NR && dslash32_tile_valid(c)) ||
                    (k == TUNE_COARSE_NT && (c == 8 || c == 16 || c == 32));
    if (ok && b >= 1 && b <= 64 && vol >= 0) ctx->tune[std::make_tuple(k, b, (int64_t)vol)] = {c, ms};
  }
  return MGLMA_OK;
}

}  // extern "C"
