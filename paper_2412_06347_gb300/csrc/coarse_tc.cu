// Coarse stencil Y(y) = sum_d Dhat_d(y) X(nbr_d(y)) on the 5th-generation
// tensor cores (tcgen05, sm_103a): BF16 operands, FP32 accumulation in TMEM.
//
// The complex product is one real GEMM per coarse site without duplicating
// the operator:
//     Yhat (n2 x 2N) = Ahat (n2 x K) . Bhat (K x 2N),   K = 9 * 2 * n2
//     Ahat[i][(d, part, j)] = part ? Im Dhat_d[i][j] : Re Dhat_d[i][j]
//     Bhat[(d, 0, j)][r] =  Re X_d[j][r]    Bhat[(d, 0, j)][N + r] = Im X_d[j][r]
//     Bhat[(d, 1, j)][r] = -Im X_d[j][r]    Bhat[(d, 1, j)][N + r] = Re X_d[j][r]
// so Yhat[:, r] = Re Y[:, r] and Yhat[:, N + r] = Im Y[:, r].
//
// Data layout: the BF16 operator of each site is stored in HBM already in the
// no-swizzle K-major core-matrix order the MMA reads from shared memory
// ([k chunk of 8][row group of 8][8 rows][8 values]), so a single bulk async
// copy per site stages it; two stage buffers let the next site's operator
// stream in while the current one is multiplied.  The MMA shape is M = 128
// (rows >= n2 read neighbouring shared memory and are never stored).
//
// Every mbarrier wait is bounded: on a timeout the kernel records an error,
// stops issuing work, waits (bounded) for its own copies, frees its TMEM and
// returns; the host reports MGLMA_ERR_TIMEOUT.
#include <algorithm>
#include <string>

#include "internal.h"
#include "lattice.cuh"
#include "solver.h"
#include "subspace.h"

namespace mglma {

constexpr int TC_THREADS = 256;
constexpr uint32_t TC_TMEM_COLS = 32;
constexpr long long TC_WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// no-swizzle K-major shared-memory matrix descriptor (sm_100 family):
// start >> 4 in bits 0-13, leading (K-direction core-matrix stride) >> 4 in
// 16-29, stride (8-row-group stride) >> 4 in 32-45, descriptor version 1 at 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D F32, A BF16, B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<uint16_t*>(&h);
}

template <int NT>  // right-hand sides per tile; the MMA N is 2 NT
__global__ void __launch_bounds__(TC_THREADS, 1)
    coarse_tc_kernel(const uint8_t* __restrict__ Aimg, const float2* __restrict__ X, float2* __restrict__ Y, LatIdx q,
                     int n2, int nrhs, int mode, int* __restrict__ err) {
  constexpr int NN = 2 * NT;
  extern __shared__ __align__(1024) uint8_t sm[];
  const int K = 18 * n2, NC = K / 8, G = n2 / 8;
  const uint32_t abytes = (uint32_t)NC * G * 128;
  uint8_t* Abuf0 = sm;
  uint8_t* Bsm = sm + 2 * (size_t)abytes;
  const uint32_t bbytes = (uint32_t)NC * (NN / 8) * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bsm + bbytes);  // full[0], full[1], mma
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int64_t V1 = q.V;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + b)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  auto issue_copy = [&](int64_t ysite, int buf) {
    const uint32_t bar = smem_u32(bars + buf);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(abytes) : "memory");
    const uint8_t* src = Aimg + (size_t)ysite * abytes;
    const uint32_t dst = smem_u32(Abuf0 + (size_t)buf * abytes);
    for (uint32_t off = 0; off < abytes; off += 32768) {
      const uint32_t len = min(32768u, abytes - off);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       dst + off),
                   "l"(src + off), "r"(len), "r"(bar)
                   : "memory");
    }
  };

  const int64_t y0 = blockIdx.x;
  bool pending[2] = {false, false};
  uint32_t full_phase[2] = {0u, 0u};
  if (tid == 0 && y0 < V1) {
    issue_copy(y0, 0);
    pending[0] = true;
  }
  const uint32_t idesc = idesc_bf16(128, NN);
  const uint32_t lboA = (uint32_t)G * 128, lboB = (uint32_t)(NN / 8) * 128;
  uint32_t mma_phase = 0;
  const int ntiles = (nrhs + NT - 1) / NT;
  const int nv = n2 / 2;
  // ---- B operand: each thread owns items w = tid + q*TC_THREADS of a work
  // unit (site, RHS tile); item = (d, j octet, RHS r): 8 complex of X.
  // The next unit's items are loaded into registers while the current
  // unit's MMA runs.
  constexpr int IT = (9 * 8 * NT + TC_THREADS - 1) / TC_THREADS;  // G <= 8
  const int nitems = 9 * G * NT;
  float4 xr[IT][4];
  auto load_unit = [&](int64_t yy, int rt) {
    int xx[4];
    site_coords(q, yy, xx);
    const int r0 = rt * NT;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int w = tid + it * TC_THREADS;
      if (w >= nitems) break;
      const int r = w % NT, jo = (w / NT) % G, d = w / (NT * G);
      if (r0 + r < nrhs) {
        const int64_t z = d == 8 ? yy : (d < 4 ? nbr_fwd(q, yy, xx, d) : nbr_bwd(q, yy, xx, d - 4));
        const float4* src = reinterpret_cast<const float4*>(X + ((size_t)(r0 + r) * V1 + z) * n2 + jo * 8);
#pragma unroll
        for (int h = 0; h < 4; ++h) xr[it][h] = __ldg(src + h);
      } else {
#pragma unroll
        for (int h = 0; h < 4; ++h) xr[it][h] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  auto store_unit = [&]() {
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int w = tid + it * TC_THREADS;
      if (w >= nitems) break;
      const int r = w % NT, jo = (w / NT) % G, d = w / (NT * G);
      float re[8], im[8];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        re[2 * h] = xr[it][h].x;
        im[2 * h] = xr[it][h].y;
        re[2 * h + 1] = xr[it][h].z;
        im[2 * h + 1] = xr[it][h].w;
      }
      if (mode & 1) {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (jo * 8 + e >= nv) {
            re[e] = -re[e];
            im[e] = -im[e];
          }
      }
      uint32_t pr[4], pim[4], nim[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        pr[e] = (uint32_t)bf16_bits(re[2 * e]) | ((uint32_t)bf16_bits(re[2 * e + 1]) << 16);
        pim[e] = (uint32_t)bf16_bits(im[2 * e]) | ((uint32_t)bf16_bits(im[2 * e + 1]) << 16);
        nim[e] = (uint32_t)bf16_bits(-im[2 * e]) | ((uint32_t)bf16_bits(-im[2 * e + 1]) << 16);
      }
      // k chunk of (d, part, jo): c = (d * 2 + part) * G + jo; columns r and NT + r
      const int c0 = (d * 2) * G + jo, c1 = (d * 2 + 1) * G + jo;
      auto put = [&](int c, int col, const uint32_t* v) {
        uint4* p = reinterpret_cast<uint4*>(Bsm + ((size_t)c * (NN / 8) + col / 8) * 128 + (col % 8) * 16);
        *p = make_uint4(v[0], v[1], v[2], v[3]);
      };
      put(c0, r, pr);        // Re X  -> Re Y column
      put(c1, r, nim);       // -Im X -> Re Y column
      put(c0, NT + r, pim);  // Im X  -> Im Y column
      put(c1, NT + r, pr);   // Re X  -> Im Y column
    }
  };

  int t = 0;
  if (y0 < V1) load_unit(y0, 0);
  for (int64_t y = y0; y < V1; y += gridDim.x, ++t) {
    const int buf = t & 1;
    const int64_t yn = y + gridDim.x;
    if (tid == 0 && yn < V1) {
      issue_copy(yn, buf ^ 1);
      pending[buf ^ 1] = true;
    }
    for (int rt = 0; rt < ntiles; ++rt) {
      const int r0 = rt * NT;
      store_unit();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0 && !abort_flag) {
        bool ok = true;
        if (rt == 0) {
          ok = mbar_wait(smem_u32(bars + buf), full_phase[buf]);
          if (ok) {
            full_phase[buf] ^= 1u;
            pending[buf] = false;
          }
        }
        if (!ok) {
          abort_flag = 1;
          atomicExch(err, 1);
        } else {
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = smem_u32(Abuf0 + (size_t)buf * abytes), b0 = smem_u32(Bsm);
          for (int s = 0; s < K / 16; ++s) {
            const uint64_t ad = smem_desc(a0 + s * 2 * lboA, lboA, 128);
            const uint64_t bd = smem_desc(b0 + s * 2 * lboB, lboB, 128);
            const uint32_t acc = s > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(bars + 2)));
        }
      }
      // next unit's gather overlaps the MMA
      if (rt + 1 < ntiles)
        load_unit(y, rt + 1);
      else if (yn < V1)
        load_unit(yn, 0);
      __syncthreads();
      if (abort_flag) break;
      if (tid == 0) {
        if (!mbar_wait(smem_u32(bars + 2), mma_phase)) {
          atomicExch(err, 2);
          abort_flag = 1;
        }
        mma_phase ^= 1u;
      }
      __syncthreads();
      if (abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      // ---- epilogue: warps 0..3 own TMEM lanes 0..127; rows >= n2 are padding
      if (warp < 4 && warp * 32 < n2) {
        uint32_t v[NN];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        if constexpr (NN == 16) {
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
        } else {
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
                "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                "=r"(v[30]), "=r"(v[31])
              : "r"(taddr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int i = warp * 32 + lane;
        if (i < n2) {
          const float sg = ((mode & 2) && i >= nv) ? -1.f : 1.f;
#pragma unroll
          for (int r = 0; r < NT; ++r)
            if (r0 + r < nrhs)
              Y[((size_t)(r0 + r) * V1 + y) * n2 + i] =
                  make_float2(sg * __uint_as_float(v[r]), sg * __uint_as_float(v[NT + r]));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (abort_flag) break;
    }
    if (abort_flag) break;
  }
  // copies still in flight (only after an abort): wait for them, bounded
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      if (pending[b]) mbar_wait(smem_u32(bars + b), full_phase[b]);
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// operator image for the kernel: per site [c][g][8 rows][8 bf16] with
// k = 8c + kk = (d * 2 + part) * n2 + j and row i = 8g + ri
__global__ void a_image_kernel(const double2* __restrict__ A64, uint16_t* __restrict__ img, int64_t V1, int n2) {
  const size_t per = (size_t)18 * n2 * n2;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * V1) return;
  const int64_t y = (int64_t)(t / per);
  const size_t e = t % per;
  const int G = n2 / 8;
  const int kk = (int)(e % 8), ri = (int)((e / 8) % 8), g = (int)((e / 64) % G), c = (int)(e / (64 * (size_t)G));
  const int i = 8 * g + ri, k = 8 * c + kk;
  const int d = k / (2 * n2), part = (k / n2) % 2, j = k % n2;
  const double2 a = A64[(((size_t)y * 9 + d) * n2 + j) * n2 + i];
  img[t] = bf16_bits((float)(part ? a.y : a.x));
}

bool coarse_tc_supported(int n2) { return n2 % 8 == 0 && n2 >= 8 && n2 <= 48; }

static size_t tc_smem(int n2, int NT) {
  const size_t K = 18 * (size_t)n2, abytes = K * n2 * 2, bbytes = K * 2 * NT * 2;
  return 2 * abytes + bbytes + 3 * 8 + 16;
}

mglma_status coarse_tc_image(mglma_ctx ctx, mglma_coarse_s* C, cudaStream_t s) {
  const size_t n = (size_t)18 * C->n2 * C->n2 * C->geo.V1;
  MG_CUDA(cudaMalloc(&C->Aimg, n * sizeof(uint16_t)));
  MG_CUDA(cudaMalloc(&C->tc_err, sizeof(int)));
  MG_CUDA(cudaMemsetAsync(C->tc_err, 0, sizeof(int), s));
  ProfScope ps(ctx, K_SETUP, s);
  a_image_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C->A64, C->Aimg, C->geo.V1, C->n2);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

template <int NT>
static mglma_status launch_tc(mglma_ctx ctx, const mglma_coarse_s* C, const float2* X, float2* Y, int nrhs,
                              int mode, int* err, cudaStream_t s) {
  const size_t smem = tc_smem(C->n2, NT);
  static size_t attr = 0;  // largest dynamic shared memory granted so far
  if (smem > attr) {
    MG_CUDA(cudaFuncSetAttribute(coarse_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  const unsigned grid = (unsigned)std::min<int64_t>(C->geo.V1, (int64_t)ctx->sm_count);
  coarse_tc_kernel<NT><<<grid, TC_THREADS, smem, s>>>((const uint8_t*)C->Aimg, X, Y, make_latidx(C->geo.Lb), C->n2,
                                                      nrhs, mode, err);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status coarse_tc_check(mglma_coarse_s* C, cudaStream_t s) {
  if (!C->tc_err) return MGLMA_OK;
  int h = 0;
  MG_CUDA(cudaMemcpyAsync(&h, C->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  if (h) {
    MG_CUDA(cudaMemsetAsync(C->tc_err, 0, sizeof(int), s));
    return fail(MGLMA_ERR_TIMEOUT, "coarse tensor-core apply: a bounded wait gave up (code " + std::to_string(h) + ")");
  }
  return MGLMA_OK;
}

mglma_status coarse_apply_tc(mglma_ctx ctx, const mglma_coarse_s* C, const float2* X, float2* Y, int nrhs,
                             int mode, cudaStream_t s) {
  if (!C->Aimg || !coarse_tc_supported(C->n2)) return fail(MGLMA_ERR_INVALID, "coarse_apply_tc: no tensor image");
  int* err = C->tc_err;
  const bool fit16 = tc_smem(C->n2, 16) <= 227 * 1024;
  const int nt = tuned(ctx, TUNE_COARSE_NT, nrhs, (nrhs <= 8 || !fit16) ? 8 : 16);
  if (nt == 16 && fit16) return launch_tc<16>(ctx, C, X, Y, nrhs, mode, err, s);
  return launch_tc<8>(ctx, C, X, Y, nrhs, mode, err, s);
}

}  // namespace mglma
