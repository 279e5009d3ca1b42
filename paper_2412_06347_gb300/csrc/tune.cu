// Autotuner of the RHS tile widths: the stencil's tile shape (RHS per thread
// 1, 2, 4 times RHS tiles per CTA 1, 2, 4) and the tensor-core coarse
// kernel's RHS per tile (8, 16, 32) are timed with
// CUDA events on the context stream for a given RHS count, and the fastest
// is kept per (kernel, RHS bucket) in the context; the table can be saved to
// and loaded from a text file keyed by GPU name.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <sstream>
#include <string>

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
    const int shapes[][2] = {{1, 1}, {2, 1}, {4, 1}, {1, 2}, {1, 4}, {2, 2}, {2, 4}};
    for (const auto& sh : shapes) {
      if (st != MGLMA_OK) break;
      if (sh[0] * sh[1] > 1 && sh[0] * sh[1] > nrhs) continue;  // tiles mostly idle
      const int code = dslash32_tile_code(sh[0], sh[1]);
      ctx->tune[TUNE_DSLASH32_NR * 1024 + bucket] = {code, 0.0};
      double ms = 0;
      st = time_ms(ctx, s, 5, [&] { return dslash(ctx, G, a, b, false, false, s); }, &ms);
      if (st == MGLMA_OK && ms < best) {
        best = ms;
        choice = code;
      }
    }
    ctx->tune[TUNE_DSLASH32_NR * 1024 + bucket] = {choice, best};
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
      ctx->tune[TUNE_COARSE_NT * 1024 + bucket] = {nt, 0.0};
      double ms = 0;
      st = time_ms(ctx, s, 5, [&] { return coarse_apply(ctx, C, X, Y, nrhs, MGLMA_FP32, CMODE_D, s); }, &ms);
      if (st == MGLMA_OK && ms < best) {
        best = ms;
        choice = nt;
      }
    }
    ctx->tune[TUNE_COARSE_NT * 1024 + bucket] = {choice, best};
    if (st == MGLMA_OK) st = coarse_tc_check(C, s);
  }
  ctx->profile = prof;
  return st;
}

mglma_status mglma_autotune_get(mglma_ctx ctx, int kernel, int nrhs, int* choice, double* ms) {
  if (!ctx) return fail(MGLMA_ERR_INVALID, "autotune_get: NULL context");
  auto it = ctx->tune.find(kernel * 1024 + rhs_bucket(nrhs));
  if (it == ctx->tune.end()) {
    if (choice) *choice = 0;
    if (ms) *ms = 0;
    return MGLMA_OK;
  }
  if (choice) *choice = it->second.first;
  if (ms) *ms = it->second.second;
  return MGLMA_OK;
}

mglma_status mglma_autotune_set(mglma_ctx ctx, int kernel, int nrhs, int choice) {
  if (!ctx || nrhs < 1) return fail(MGLMA_ERR_INVALID, "autotune_set: bad arguments");
  const bool ok = (kernel == TUNE_DSLASH32_NR && dslash32_tile_valid(choice)) ||
                  (kernel == TUNE_COARSE_NT && (choice == 8 || choice == 16 || choice == 32));
  if (!ok) return fail(MGLMA_ERR_INVALID, "autotune_set: unknown kernel or choice");
  ctx->tune[kernel * 1024 + rhs_bucket(nrhs)] = {choice, 0.0};
  return MGLMA_OK;
}

mglma_status mglma_autotune_save(mglma_ctx ctx, const char* path) {
  if (!ctx || !path) return fail(MGLMA_ERR_INVALID, "autotune_save: NULL argument");
  std::ofstream f(path);
  if (!f) return fail(MGLMA_ERR_INVALID, std::string("autotune_save: cannot write ") + path);
  const std::string gpu = gpu_name(ctx->device);
  for (auto& kv : ctx->tune)
    f << gpu << ' ' << kv.first / 1024 << ' ' << kv.first % 1024 << ' ' << kv.second.first << ' ' << kv.second.second
      << '\n';
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
    double ms;
    if (!(is >> g >> k >> b >> c >> ms) || g != gpu) continue;
    const bool ok = (k == TUNE_DSLASH32_NR && dslash32_tile_valid(c)) ||
                    (k == TUNE_COARSE_NT && (c == 8 || c == 16 || c == 32));
    if (ok && b >= 1 && b <= 64) ctx->tune[k * 1024 + b] = {c, ms};
  }
  return MGLMA_OK;
}

}  // extern "C"
