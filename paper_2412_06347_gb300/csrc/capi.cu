// C ABI of libmglma: context, errors, per-kernel timing, gauge loading and the
// Dirac operator entry point.  Argument checking and host<->device staging
// live here; all arithmetic runs in the kernels of the other units.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "solver.h"

namespace mglma {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

mglma_status fail(mglma_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

static const char* kKindNames[K_NKINDS] = {"dslash64", "dslash32", "blas",  "reduce", "restrict", "prolong",
                                           "coarse",   "pack",     "setup", "scalar", "cblas",    "creduce",
                                           "contract"};

CoarseLevelScope::CoarseLevelScope(mglma_ctx c) : ctx(c), prev(c ? c->coarse_level : false) {
  if (ctx) ctx->coarse_level = true;
}
CoarseLevelScope::~CoarseLevelScope() {
  if (ctx) ctx->coarse_level = prev;
}
const char* kernel_kind_name(int k) { return (k >= 0 && k < K_NKINDS) ? kKindNames[k] : "?"; }

void resolve_profile(mglma_ctx ctx);

static cudaEvent_t take_event(mglma_ctx ctx) {
  if (!ctx->event_cache.empty()) {
    cudaEvent_t e = ctx->event_cache.back();
    ctx->event_cache.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(mglma_ctx c, int k, cudaStream_t st, double bytes_, double flops_)
    : ctx(c), kind(k), s(st), bytes(bytes_), flops(flops_) {
  if (ctx && ctx->coarse_level) {
    if (kind == K_BLAS) kind = K_CBLAS;
    if (kind == K_REDUCE) kind = K_CREDUCE;
  }
  if (ctx && ctx->profile) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone) {
      if (!ctx->capture_events) return;
      cudaEventCreate(&a);  // owned by the graph's list
      cudaEventCreate(&b);
      cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
      captured = true;
      return;
    }
    a = take_event(ctx);
    b = take_event(ctx);
    cudaEventRecord(a, s);
  }
}

ProfScope::~ProfScope() {
  if (a && captured) {
    cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
    ctx->capture_events->push_back({kind, a, b, bytes, flops});
    return;
  }
  if (a) {
    cudaEventRecord(b, s);
    ctx->pending.push_back({kind, a, b, bytes, flops});
    if (ctx->pending.size() > 4096) resolve_profile(ctx);  // bound the list
  }
}

void resolve_graph_events(mglma_ctx ctx, const std::vector<mglma_ctx_s::Pending>& ev) {
  for (auto& p : ev) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    ctx->stats[p.kind].launches += 1;
    ctx->stats[p.kind].ms += ms;
    ctx->stats[p.kind].bytes += p.bytes;
    ctx->stats[p.kind].flops += p.flops;
  }
}

void resolve_profile(mglma_ctx ctx) {
  for (auto& p : ctx->pending) {
    cudaEventSynchronize(p.b);
    float ms = 0;
    cudaEventElapsedTime(&ms, p.a, p.b);
    ctx->stats[p.kind].launches += 1;
    ctx->stats[p.kind].ms += ms;
    ctx->stats[p.kind].bytes += p.bytes;
    ctx->stats[p.kind].flops += p.flops;
    ctx->event_cache.push_back(p.a);
    ctx->event_cache.push_back(p.b);
  }
  ctx->pending.clear();
}

mglma_status dalloc(mglma_ctx ctx, void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) return MGLMA_OK;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? MGLMA_ERR_OOM : MGLMA_ERR_CUDA,
                std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                    cudaGetErrorString(e));
  }
  return MGLMA_OK;
}

void dfree(mglma_ctx, void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

size_t device_room(mglma_ctx ctx, cudaStream_t s) {
  cudaStreamSynchronize(s);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  uint64_t reserved = 0, used = 0;
  if (cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
      cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
    cudaGetLastError();
    return fr;
  }
  return fr + (reserved > used ? (size_t)(reserved - used) : 0);
}

mglma_status check_gauge_device(mglma_ctx ctx, const mglma_gauge_s* G, const char* who) {
  if (!G->ctx || G->ctx->device != ctx->device)
    return fail(MGLMA_ERR_INVALID, std::string(who) + ": gauge field was loaded on another device");
  return MGLMA_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// declared in dslash.cu
mglma_status gauge_pack_slab(mglma_ctx ctx, mglma_gauge_s* G, const double* links_dev, int64_t site0,
                             int64_t nsites, double* dev_max, cudaStream_t s);
mglma_status clover_build(mglma_ctx ctx, mglma_gauge_s* G, cudaStream_t s);
mglma_status debug_tables(mglma_ctx ctx, const mglma_gauge_s* G, const int* block, int32_t* nbr_dev,
                          int32_t* blk_dev, cudaStream_t s);

mglma_status stage_in(mglma_ctx ctx, const double* p, size_t bytes, cudaStream_t s, Staged& st) {
  st.ctx = ctx;
  st.s = s;
  if (is_device_pointer(p)) {
    st.dev = const_cast<double*>(p);
    return MGLMA_OK;
  }
  MG_CHECK(dalloc(ctx, (void**)&st.dev, bytes, s));
  st.owned = true;
  MG_CUDA(cudaMemcpyAsync(st.dev, p, bytes, cudaMemcpyHostToDevice, s));
  return MGLMA_OK;
}

mglma_status stage_out_alloc(mglma_ctx ctx, double* p, size_t bytes, cudaStream_t s, Staged& st) {
  st.ctx = ctx;
  st.s = s;
  if (is_device_pointer(p)) {
    st.dev = p;
    return MGLMA_OK;
  }
  MG_CHECK(dalloc(ctx, (void**)&st.dev, bytes, s));
  st.owned = true;
  return MGLMA_OK;
}

mglma_status stage_out_finish(double* p, size_t bytes, cudaStream_t s, Staged& st) {
  if (!st.owned) return MGLMA_OK;
  MG_CUDA(cudaMemcpyAsync(p, st.dev, bytes, cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

cudaStream_t pick_stream(mglma_ctx ctx, void* s) { return s ? (cudaStream_t)s : ctx->stream; }

}  // namespace mglma

using namespace mglma;

extern "C" {

const char* mglma_last_error(void) { return g_last_error.c_str(); }
const char* mglma_version(void) { return "mglma 0.1 (sm_103a)"; }

mglma_status mglma_create(int device, mglma_ctx* out) {
  if (!out) return fail(MGLMA_ERR_INVALID, "mglma_create: out is NULL");
  *out = nullptr;
  int n = 0;
  MG_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(MGLMA_ERR_INVALID, "mglma_create: no such device");
  MG_CUDA(cudaSetDevice(device));
  mglma_ctx c = new mglma_ctx_s();
  c->device = device;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return fail(MGLMA_ERR_CUDA, std::string("stream create: ") + cudaGetErrorString(e));
  }
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  e = cudaMemPoolCreate(&c->pool, &props);
  if (e != cudaSuccess) {
    cudaStreamDestroy(c->stream);
    delete c;
    return fail(MGLMA_ERR_CUDA, std::string("mem pool create: ") + cudaGetErrorString(e));
  }
  uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool
  cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  for (int k = 0; k < K_NKINDS; ++k) c->stats[k].name = kernel_kind_name(k);
  if (const char* cache = getenv("MGLMA_TUNE_CACHE")) {
    c->tune_cache = cache;
    FILE* f = fopen(cache, "r");
    if (f) {
      fclose(f);
      mglma_autotune_load(c, cache);  // entries of other GPUs are skipped
    }
  }
  *out = c;
  return MGLMA_OK;
}

void mglma_destroy(mglma_ctx ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  resolve_profile(ctx);
  for (auto e : ctx->event_cache) cudaEventDestroy(e);
  for (auto& kv : ctx->red) {
    cudaFreeAsync(kv.second.part, ctx->stream);
    cudaFreeAsync(kv.second.count, ctx->stream);
  }
  cudaStreamSynchronize(ctx->stream);
  cudaStreamDestroy(ctx->stream);
  cudaDeviceSynchronize();
  cudaMemPoolDestroy(ctx->pool);
  delete ctx;
}

mglma_status mglma_profile(mglma_ctx ctx, int enable, int reset) {
  if (!ctx) return fail(MGLMA_ERR_INVALID, "mglma_profile: NULL context");
  resolve_profile(ctx);
  if (reset)
    for (int k = 0; k < K_NKINDS; ++k) {
      ctx->stats[k].launches = 0;
      ctx->stats[k].ms = 0;
      ctx->stats[k].bytes = 0;
      ctx->stats[k].flops = 0;
    }
  ctx->profile = enable != 0;
  return MGLMA_OK;
}

mglma_status mglma_profile_get(mglma_ctx ctx, const char* name, long long* launches, double* ms, double* bytes,
                               double* flops) {
  if (!ctx || !name) return fail(MGLMA_ERR_INVALID, "mglma_profile_get: NULL argument");
  resolve_profile(ctx);
  for (int k = 0; k < K_NKINDS; ++k)
    if (ctx->stats[k].name == name) {
      if (launches) *launches = ctx->stats[k].launches;
      if (ms) *ms = ctx->stats[k].ms;
      if (bytes) *bytes = ctx->stats[k].bytes;
      if (flops) *flops = ctx->stats[k].flops;
      return MGLMA_OK;
    }
  return fail(MGLMA_ERR_INVALID, std::string("mglma_profile_get: unknown kernel class ") + name);
}

mglma_status mglma_gauge_load(mglma_ctx ctx, const mglma_lattice* lat, const double* links, int64_t t_begin,
                              int64_t t_count, double kappa, double csw, mglma_gauge* inout) {
  if (!ctx || !lat || !links || !inout) return fail(MGLMA_ERR_INVALID, "mglma_gauge_load: NULL argument");
  for (int m = 0; m < 4; ++m)
    if (lat->L[m] < 1 || lat->L[m] > 4096) return fail(MGLMA_ERR_INVALID, "mglma_gauge_load: bad extent");
  if (lat->t_bc != 1 && lat->t_bc != -1) return fail(MGLMA_ERR_INVALID, "mglma_gauge_load: t_bc must be +-1");
  if (!(kappa > 0)) return fail(MGLMA_ERR_INVALID, "mglma_gauge_load: kappa must be positive");
  if (t_begin < 0 || t_count < 1 || t_begin + t_count > lat->L[0])
    return fail(MGLMA_ERR_INVALID, "mglma_gauge_load: slab outside the lattice");
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  mglma_gauge_s* G = *inout;
  if (G) {
    for (int m = 0; m < 4; ++m)
      if (G->g.L[m] != lat->L[m]) return fail(MGLMA_ERR_INVALID, "mglma_gauge_load: lattice differs from handle");
    if (G->kappa != kappa || G->csw != csw)
      return fail(MGLMA_ERR_INVALID, "mglma_gauge_load: kappa/csw differ from handle");
  } else {
    G = new mglma_gauge_s();
    G->ctx = ctx;
    G->g = make_geom(lat->L, lat->t_bc);
    G->kappa = kappa;
    G->csw = csw;
    G->m0 = 1.0 / (2.0 * kappa) - 4.0;
    const size_t V = (size_t)G->g.V;
    cudaError_t e1 = cudaMalloc(&G->U64, V * 36 * sizeof(double2));
    cudaError_t e2 = cudaMalloc(&G->U32, V * 12 * sizeof(float4));
    cudaError_t e3 = cudaMalloc(&G->C64, V * 36 * sizeof(double2));
    cudaError_t e4 = cudaMalloc(&G->C32, V * 18 * sizeof(float4));
    if (e1 || e2 || e3 || e4) {
      cudaGetLastError();
      mglma_gauge_free(G);
      return fail(MGLMA_ERR_OOM, "mglma_gauge_load: device allocation failed");
    }
    G->slab_seen.assign(lat->L[0], 0);
  }
  const int64_t slice = G->g.V / G->g.L[0];
  const int64_t site0 = t_begin * slice, nsites = t_count * slice;
  const size_t bytes = (size_t)nsites * 4 * 18 * sizeof(double);
  mglma_status st;
  {
    Staged in;
    st = stage_in(ctx, links, bytes, s, in);
    double* dmax = nullptr;
    if (st == MGLMA_OK) st = dalloc(ctx, (void**)&dmax, sizeof(double), s);
    if (st == MGLMA_OK) {
      cudaMemsetAsync(dmax, 0, sizeof(double), s);
      st = gauge_pack_slab(ctx, G, in.dev, site0, nsites, dmax, s);
      double hmax = 0;
      cudaMemcpyAsync(&hmax, dmax, sizeof(double), cudaMemcpyDeviceToHost, s);
      dfree(ctx, dmax, s);
      cudaError_t e = cudaStreamSynchronize(s);
      if (st == MGLMA_OK && e != cudaSuccess) st = fail(MGLMA_ERR_CUDA, cudaGetErrorString(e));
      if (st == MGLMA_OK) {
        G->unitarity_dev = std::max(G->unitarity_dev, hmax);
        if (!(hmax <= 1e-10)) {
          char buf[160];
          snprintf(buf, sizeof buf, "mglma_gauge_load: links are not SU(3) (max deviation %.3e > 1e-10)", hmax);
          st = fail(MGLMA_ERR_INVALID, buf);
        }
      }
    }
  }
  if (st != MGLMA_OK) {
    if (!*inout) mglma_gauge_free(G);
    return st;
  }
  for (int64_t t = t_begin; t < t_begin + t_count; ++t)
    if (!G->slab_seen[t]) {
      G->slab_seen[t] = 1;
      G->slabs_loaded++;
    }
  *inout = G;
  if (G->slabs_loaded == G->g.L[0]) {
    MG_CHECK(clover_build(ctx, G, s));
    MG_CUDA(cudaStreamSynchronize(s));
    G->ready = true;
  }
  return MGLMA_OK;
}

void mglma_gauge_free(mglma_gauge G) {
  if (!G) return;
  if (G->ctx) cudaSetDevice(G->ctx->device);
  cudaFree(G->U64);
  cudaFree(G->U32);
  cudaFree(G->C64);
  cudaFree(G->C32);
  cudaFree(G->Cinv64);
  cudaFree(G->Udf);
  cudaFree(G->Cdf);
  delete G;
}

mglma_status mglma_gauge_info(mglma_gauge g, int L[4], int64_t* volume) {
  if (!g) return fail(MGLMA_ERR_INVALID, "mglma_gauge_info: NULL handle");
  if (L)
    for (int m = 0; m < 4; ++m) L[m] = g->g.L[m];
  if (volume) *volume = g->g.V;
  return MGLMA_OK;
}

mglma_status mglma_dirac_apply(mglma_ctx ctx, mglma_gauge G, mglma_op op, int nrhs, const double* in, double* out,
                               mglma_prec compute, void* cuda_stream) {
  if (!ctx || !G || !in || !out) return fail(MGLMA_ERR_INVALID, "mglma_dirac_apply: NULL argument");
  if (!G->ready) return fail(MGLMA_ERR_INVALID, "mglma_dirac_apply: gauge field incomplete");
  MG_CHECK(check_gauge_device(ctx, G, "mglma_dirac_apply"));
  if (nrhs < 0) return fail(MGLMA_ERR_INVALID, "mglma_dirac_apply: nrhs < 0");
  if (op < MGLMA_OP_D || op > MGLMA_OP_SCHUR_Q) return fail(MGLMA_ERR_INVALID, "mglma_dirac_apply: bad op");
  if (compute != MGLMA_FP64 && compute != MGLMA_FP32)
    return fail(MGLMA_ERR_INVALID, "mglma_dirac_apply: compute must be FP64 or FP32");
  const bool schur = op == MGLMA_OP_SCHUR || op == MGLMA_OP_SCHUR_Q;
  if (schur && compute != MGLMA_FP64)
    return fail(MGLMA_ERR_INVALID, "mglma_dirac_apply: the even-odd operators are FP64 only");
  if (nrhs == 0) return MGLMA_OK;
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = pick_stream(ctx, cuda_stream);
  const size_t bytes = (size_t)nrhs * G->g.V * 24 * sizeof(double);
  Staged sin, sout;
  MG_CHECK(stage_in(ctx, in, bytes, s, sin));
  MG_CHECK(stage_out_alloc(ctx, out, bytes, s, sout));
  if (schur) {
    MG_CHECK(dirac_schur64(ctx, G, nrhs, sin.dev, sout.dev, op == MGLMA_OP_SCHUR_Q, s));
    return stage_out_finish(out, bytes, s, sout);
  }
  Spinor a, b;
  a.prec = b.prec = compute;
  a.nrhs = b.nrhs = nrhs;
  a.V = b.V = G->g.V;
  mglma_status st = dalloc(ctx, &a.p, a.bytes(), s);
  if (st == MGLMA_OK) st = dalloc(ctx, &b.p, b.bytes(), s);
  if (st == MGLMA_OK) st = pack_spinor(ctx, sin.dev, a, s);
  const Spinor* res = &b;
  if (st == MGLMA_OK) {
    switch (op) {
      case MGLMA_OP_D: st = dslash(ctx, G, a, b, false, false, s); break;
      case MGLMA_OP_DDAG: st = dslash(ctx, G, a, b, true, false, s); break;
      case MGLMA_OP_Q: st = dslash(ctx, G, a, b, false, true, s); break;
      case MGLMA_OP_DDAGD:
        st = dslash(ctx, G, a, b, false, false, s);
        if (st == MGLMA_OK) st = dslash(ctx, G, b, a, true, false, s);
        res = &a;
        break;
    }
  }
  if (st == MGLMA_OK) st = unpack_spinor(ctx, *res, sout.dev, s);
  dfree(ctx, a.p, s);
  dfree(ctx, b.p, s);
  if (st == MGLMA_OK) st = stage_out_finish(out, bytes, s, sout);
  return st;
}

mglma_status mglma_debug_tables(mglma_gauge G, const int block[4], int32_t* nbr, int32_t* block_of_site) {
  if (!G || !nbr) return fail(MGLMA_ERR_INVALID, "mglma_debug_tables: NULL argument");
  if (block)
    for (int m = 0; m < 4; ++m)
      if (block[m] < 1 || G->g.L[m] % block[m])
        return fail(MGLMA_ERR_INVALID, "mglma_debug_tables: block sides must divide L");
  mglma_ctx ctx = G->ctx;
  MG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const size_t V = (size_t)G->g.V;
  int32_t *dn = nullptr, *db = nullptr;
  MG_CHECK(dalloc(ctx, (void**)&dn, V * 8 * sizeof(int32_t), s));
  if (block && block_of_site) MG_CHECK(dalloc(ctx, (void**)&db, V * sizeof(int32_t), s));
  MG_CHECK(debug_tables(ctx, G, block, dn, db, s));
  MG_CUDA(cudaMemcpyAsync(nbr, dn, V * 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (db) MG_CUDA(cudaMemcpyAsync(block_of_site, db, V * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  dfree(ctx, dn, s);
  dfree(ctx, db, s);
  MG_CUDA(cudaStreamSynchronize(s));
  return MGLMA_OK;
}

}  // extern "C"
