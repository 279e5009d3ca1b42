// Block restriction R0 (Eq. res_mg) and prolongation T0 (Eq. pro_mg) on the
// 5th-generation tensor cores (tcgen05, sm_103a) for FP32 fields at many RHS:
// BF16 operands, FP32 accumulation in TMEM.  R0 first, T0 after it, the host
// side at the end of the file.
//
// Per block y and chirality alpha the restriction is one complex product
//     c[j][r] = sum_{k in B_y, q < 6} conj(phi_{y j}(k)_q) psi_r(k)_{6 alpha + q}
// over the Nv dofs j of that chirality, written as one real GEMM without
// duplicating the basis:
//     Chat (Nv x 2N) = Ahat (Nv x K) . Bhat (K x 2N),   K = 2 x 6 |B|
//     Ahat[j][(p, k, q)] = p ? Im phi_j(k)_q : Re phi_j(k)_q
//     Bhat[(0, k, q)][r] = Re psi_r   Bhat[(0, k, q)][N + r] =  Im psi_r
//     Bhat[(1, k, q)][r] = Im psi_r   Bhat[(1, k, q)][N + r] = -Re psi_r
// so Chat[:, r] = Re c[:, r] and Chat[:, N + r] = Im c[:, r].
//
// K is walked in segments of 64 sites of one component pair (2c, 2c + 1):
// 32 chunks of 8 K values, chunk kc = (o 2 + h) 2 + p for octet o of the
// segment's sites, component 2c + h and part p, the 8 values being the
// octet's sites.  The basis (with its FP16 scale) is imaged once per
// subspace in BF16 in exactly the shared-memory order the MMA reads
// ([segment][chunk][row group][8 rows][8 values], no swizzle, K-major), so a
// stage's A operand is one bulk copy.  The B operand is the residual itself:
// four producer warps read it in FP32 and write its BF16 embedding into the
// stage ([chunk][column group][8 columns][8 values]).  The MMA shape is
// M = 128, N = 32 (16 RHS); rows >= Nv read neighbouring shared memory and
// are never stored, as in the coarse stencil kernel.
//
// Roles (192 threads): warps 0-3 fill stages (warp 0 lane 0 also issues the
// A copy), warp 4 reads the accumulators (TMEM lanes 0-31 hold the rows),
// warp 5 lane 0 issues the MMAs.  Work units (block, RHS tile of 16) are
// taken persistently; the two chiralities of a unit use two accumulators and
// consecutive units alternate between two TMEM buffers.  Every wait is
// bounded; on a timeout the kernel records an error and returns after its
// copies in flight have landed.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"
#include "subspace.h"
#include "tcgen05.cuh"

namespace mglma {

constexpr int RT_THREADS = 192;
constexpr int RT_NT = 16;             // RHS per tile
constexpr int RT_N = 2 * RT_NT;       // MMA N
constexpr int RT_SEG = 64;            // sites per segment
constexpr int RT_CH = 32;             // chunks of 8 K values per segment
constexpr uint32_t RT_B_BYTES = RT_CH * (RT_N / 8) * 128;  // 16 KB
constexpr int RT_MAX_STAGES = 8;
constexpr int RT_MAX_NB = 512;        // sites per block the site table holds

__device__ __forceinline__ int64_t rt_block_site(const BlockGeo& g, int64_t y, int k) {
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

// the basis image, one thread per BF16 value: [y][alpha][seg][kc][g][ri][e]
// with seg = c (nB / 64) + og, kc = (o 2 + h) 2 + p, j = alpha Nv + 8 g + ri,
// site k = 64 og + 8 o + e, component q = 2c + h
template <typename B>
__global__ void rt_image_kernel(const void* __restrict__ basis, const float* __restrict__ scale, BlockGeo g, int nv,
                                uint16_t* __restrict__ img) {
  const int GA = nv / 8, nog = g.nB / RT_SEG, nseg = 3 * nog;
  const size_t per_seg = (size_t)RT_CH * GA * 64;
  const size_t per_y = 2 * (size_t)nseg * per_seg;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per_y * (size_t)g.V1) return;
  const int64_t y = (int64_t)(t / per_y);
  size_t e2 = t % per_y;
  const int alpha = (int)(e2 / ((size_t)nseg * per_seg));
  e2 %= (size_t)nseg * per_seg;
  const int seg = (int)(e2 / per_seg);
  e2 %= per_seg;
  const int e = (int)(e2 % 8), ri = (int)((e2 / 8) % 8), gg = (int)((e2 / 64) % GA), kc = (int)(e2 / (64 * (size_t)GA));
  const int p = kc % 2, h = (kc / 2) % 2, o = kc / 4;
  const int c = seg / nog, og = seg % nog;
  const int n2 = 2 * nv;
  const int j = alpha * nv + 8 * gg + ri;
  const int k = RT_SEG * og + 8 * o + e;
  const size_t yj = (size_t)y * n2 + j;
  float re, im;
  if (sizeof(B) == 2) {
    uint2 v = __ldg(reinterpret_cast<const uint2*>(basis) + (yj * 3 + c) * g.nB + k);
    const float2 f = __half22float2(*reinterpret_cast<__half2*>(h ? &v.y : &v.x));
    const float sc = __ldg(scale + yj);
    re = f.x * sc;
    im = f.y * sc;
  } else {
    const float4 v = __ldg(reinterpret_cast<const float4*>(basis) + (yj * 3 + c) * g.nB + k);
    re = h ? v.z : v.x;
    im = h ? v.w : v.y;
  }
  img[t] = bf16_bits(p ? im : re);
}

// barrier 1 over the four producer warps, returning whether any of them
// passed true (a uniform decision)
__device__ __forceinline__ bool rt_producers_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, 128, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ uint32_t rt_pack(float a, float b) {
  return (uint32_t)bf16_bits(a) | ((uint32_t)bf16_bits(b) << 16);
}

struct RtRun {
  const float4* fine;  // FP32 spinors [rhs][6][V]
  const uint8_t* img;  // basis image
  float2* out;         // [rhs][V1][2 Nv]
  int nrhs;
  int* err;
};

__global__ void __launch_bounds__(RT_THREADS, 2) restrict_tc_kernel(RtRun run, BlockGeo g, int nv, int nstages) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int GA = nv / 8, nog = g.nB / RT_SEG, nseg = 3 * nog, n2 = 2 * nv;
  const uint32_t a_bytes = (uint32_t)RT_CH * GA * 128;
  const uint32_t stage_bytes = a_bytes + RT_B_BYTES;
  const int S = nstages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (size_t)S * stage_bytes);
  uint64_t* afull = bars;                      // [S] A copy landed
  uint64_t* bfull = bars + RT_MAX_STAGES;      // [S] B written (128 arrivals)
  uint64_t* empty = bars + 2 * RT_MAX_STAGES;  // [S] MMAs done reading
  uint64_t* accf = bars + 3 * RT_MAX_STAGES;   // [2]
  uint64_t* acce = accf + 2;                   // [2]
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int64_t* site_of = reinterpret_cast<int64_t*>(bars + 3 * RT_MAX_STAGES + 8);
  __shared__ int abort_flag;
  volatile int* abrt = &abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int ntiles = (run.nrhs + RT_NT - 1) / RT_NT;
  const int64_t nunits = g.V1 * ntiles;
  constexpr uint32_t TMEM_COLS = 4 * RT_N;  // two buffers x two chiralities

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int b = 0; b < S; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(afull + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(bfull + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(empty + b)));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(accf + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(acce + b)));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  auto give_up = [&](int code) {
    abort_flag = 1;
    atomicExch(run.err, code);
  };

  if (warp < 4) {
    // ------------------------------------------------------------ producers
    uint32_t it = 0;
    bool ok = true;
    const int r = tid % RT_NT, o = tid / RT_NT;  // RHS of the tile, octet of the segment
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
      const int64_t y = u / ntiles;
      const int t = (int)(u % ntiles);
      // all producers stop together (a wait gave up); the same barrier
      // guarantees the previous unit's site table is consumed
      if (rt_producers_any(!ok || *abrt)) break;
      for (int k = tid; k < g.nB; k += 128) site_of[k] = rt_block_site(g, y, k);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const int rr = t * RT_NT + r;
      for (int alpha = 0; alpha < 2 && ok; ++alpha) {
        for (int seg = 0; seg < nseg; ++seg, ++it) {
          const int st = (int)(it % S);
          const uint32_t ph = (it / S) & 1u;
          if (!mbar_wait(smem_u32(empty + st), ph ^ 1u, abrt)) {
            if (!*abrt) give_up(1);
            ok = false;
            break;
          }
          uint8_t* sa = sm + (size_t)st * stage_bytes;
          uint4* sb = reinterpret_cast<uint4*>(sa + a_bytes);
          const int c = seg / nog, og = seg % nog;
          float4 v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int64_t site = site_of[RT_SEG * og + 8 * o + e];
            v[e] = rr < run.nrhs ? __ldg(run.fine + ((size_t)rr * 6 + 3 * alpha + c) * g.V + site)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float re[8], im[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              re[e] = h ? v[e].z : v[e].x;
              im[e] = h ? v[e].w : v[e].y;
            }
            const int kc0 = (o * 2 + h) * 2;  // part 0; part 1 at kc0 + 1
            const uint4 pre = make_uint4(rt_pack(re[0], re[1]), rt_pack(re[2], re[3]), rt_pack(re[4], re[5]),
                                         rt_pack(re[6], re[7]));
            const uint4 pim = make_uint4(rt_pack(im[0], im[1]), rt_pack(im[2], im[3]), rt_pack(im[4], im[5]),
                                         rt_pack(im[6], im[7]));
            const uint4 nre = make_uint4(rt_pack(-re[0], -re[1]), rt_pack(-re[2], -re[3]), rt_pack(-re[4], -re[5]),
                                         rt_pack(-re[6], -re[7]));
            sb[kc0 * RT_N + r] = pre;                 // part 0, Re column
            sb[kc0 * RT_N + RT_NT + r] = pim;         // part 0, Im column
            sb[(kc0 + 1) * RT_N + r] = pim;           // part 1, Re column
            sb[(kc0 + 1) * RT_N + RT_NT + r] = nre;   // part 1, Im column
          }
          // the MMA reads the stage through the async proxy
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bfull + st)) : "memory");
          if (tid == 0) {
            const uint32_t bar = smem_u32(afull + st);
            const uint8_t* src = run.img + (((size_t)y * 2 + alpha) * nseg + seg) * a_bytes;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(a_bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sa)),
                "l"(src), "r"(a_bytes), "r"(bar)
                : "memory");
          }
        }
      }
    }
    // copies still in flight (after an abort): wait for each stage's last
    // A fill, bounded and regardless of the abort flag
    if (tid == 0)
      for (uint32_t st = 0; st < (uint32_t)S && st < it; ++st) {
        const uint32_t fills = (it - st + S - 1) / S;
        mbar_wait(smem_u32(afull + st), (fills - 1) & 1u, nullptr);
      }
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, RT_N);
      const uint32_t lboA = (uint32_t)GA * 128, lboB = (uint32_t)(RT_N / 8) * 128;
      uint32_t it = 0, ua = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++ua) {
        const uint32_t b = ua & 1u, aph = (ua >> 1) & 1u;
        if (!mbar_wait(smem_u32(acce + b), aph ^ 1u, abrt)) {
          if (!*abrt) give_up(2);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int alpha = 0; alpha < 2 && ok; ++alpha) {
          const uint32_t dcol = tmem + b * 2 * RT_N + alpha * RT_N;
          for (int seg = 0; seg < nseg; ++seg, ++it) {
            const int st = (int)(it % S);
            const uint32_t ph = (it / S) & 1u;
            if (!mbar_wait(smem_u32(afull + st), ph, abrt) || !mbar_wait(smem_u32(bfull + st), ph, abrt)) {
              if (!*abrt) give_up(3);
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sm + (size_t)st * stage_bytes), b0 = a0 + a_bytes;
            for (int m = 0; m < RT_CH / 2; ++m) {
              const uint64_t ad = smem_desc(a0 + m * 2 * lboA, lboA, 128);
              const uint64_t bd = smem_desc(b0 + m * 2 * lboB, lboB, 128);
              const uint32_t acc = (seg > 0 || m > 0) ? 1u : 0u;
              asm volatile(
                  "{\n\t.reg .pred p;\n\t"
                  "setp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(empty + st)));
          }
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(accf + b)));
      }
      // every MMA issued by this thread has completed before TMEM is freed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(done)));
      mbar_wait(smem_u32(done), 0u, nullptr);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warp 4: TMEM lanes 0-31)
    uint32_t ua = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++ua) {
      const int64_t y = u / ntiles;
      const int t = (int)(u % ntiles);
      const uint32_t b = ua & 1u, aph = (ua >> 1) & 1u;
      const bool mine = mbar_wait(smem_u32(accf + b), aph, abrt);
      if (!__all_sync(0xffffffffu, mine)) {
        if (lane == 0 && !*abrt) give_up(4);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t v0[RT_N], v1[RT_N];
      tmem_ld<RT_N>(tmem + b * 2 * RT_N, v0);
      tmem_ld<RT_N>(tmem + b * 2 * RT_N + RT_N, v1);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acce + b)) : "memory");
      if (lane < nv) {
#pragma unroll
        for (int r = 0; r < RT_NT; ++r) {
          const int rr = t * RT_NT + r;
          if (rr < run.nrhs) {
            float2* o = run.out + ((size_t)rr * g.V1 + y) * n2;
            o[lane] = make_float2(__uint_as_float(v0[r]), __uint_as_float(v0[RT_NT + r]));
            o[nv + lane] = make_float2(__uint_as_float(v1[r]), __uint_as_float(v1[RT_NT + r]));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ============================================================ T0
// Per block y and chirality alpha the prolongation is
//     f_r(k)_{6 alpha + q} = sum_j phi_{y j}(k)_q c[r][j]
// with rows (q, k) of the block (M) and the Nv dofs (K); as a real GEMM
//     Fhat (M x 2N) = Phat (M x 2 Nv) . Chat (2 Nv x 2N)
//     Phat[(q, k)][(p, j)] = p ? Im phi_j(k)_q : Re phi_j(k)_q
//     Chat[(0, j)][r] =  Re c_r[j]   Chat[(0, j)][N + r] = Im c_r[j]
//     Chat[(1, j)][r] = -Im c_r[j]   Chat[(1, j)][N + r] = Re c_r[j]
// M is cut into tiles of 128 sites of one component q: tile m = (cq nhalf +
// half) 2 + h for q = 2 cq + h and sites 128 half .. 128 half + 127, so the
// two components of one FP32 float4 chunk come out in consecutive tiles.  The
// basis is imaged per tile ([chunk of 8 (p, j)][row group][8 rows][8
// values]); the coefficients of a work unit are imaged in shared memory by a
// warp of their own.
constexpr int PT_THREADS = 224;  // warps 0-3 epilogue (TMEM lanes 0-127), 4 basis copies, 5 MMA, 6 coefficients
constexpr int PT_MAX_STAGES = 8;
constexpr int PT_PAIRS = 2;      // accumulator pairs (tiles h = 0, 1 of one float4 chunk), 64 columns each

// the T0 basis image, one thread per BF16 value: [y][alpha][m][kc][g][ri][e],
// row 8 g + ri = site k - 128 half of the tile, K = 8 kc + e = p Nv + jj
template <typename B>
__global__ void pt_image_kernel(const void* __restrict__ basis, const float* __restrict__ scale, BlockGeo g, int nv,
                                uint16_t* __restrict__ img) {
  const int KC = nv / 4, nhalf = g.nB / 128, ntile = 6 * nhalf;
  const size_t per_tile = (size_t)KC * 16 * 64;
  const size_t per_y = 2 * (size_t)ntile * per_tile;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per_y * (size_t)g.V1) return;
  const int64_t y = (int64_t)(t / per_y);
  size_t e2 = t % per_y;
  const int alpha = (int)(e2 / ((size_t)ntile * per_tile));
  e2 %= (size_t)ntile * per_tile;
  const int m = (int)(e2 / per_tile);
  e2 %= per_tile;
  const int e = (int)(e2 % 8), ri = (int)((e2 / 8) % 8), gg = (int)((e2 / 64) % 16), kc = (int)(e2 / 1024);
  const int h = m % 2, half = (m / 2) % nhalf, cq = m / (2 * nhalf);
  const int K = 8 * kc + e, p = K / nv, jj = K % nv;
  const int n2 = 2 * nv;
  const int j = alpha * nv + jj;
  const int k = 128 * half + 8 * gg + ri;
  const size_t yj = (size_t)y * n2 + j;
  float re, im;
  if (sizeof(B) == 2) {
    uint2 v = __ldg(reinterpret_cast<const uint2*>(basis) + (yj * 3 + cq) * g.nB + k);
    const float2 f = __half22float2(*reinterpret_cast<__half2*>(h ? &v.y : &v.x));
    const float sc = __ldg(scale + yj);
    re = f.x * sc;
    im = f.y * sc;
  } else {
    const float4 v = __ldg(reinterpret_cast<const float4*>(basis) + (yj * 3 + cq) * g.nB + k);
    re = h ? v.z : v.x;
    im = h ? v.w : v.y;
  }
  img[t] = bf16_bits(p ? im : re);
}

struct PtRun {
  const float2* coarse;  // FP32 [rhs][V1][2 Nv]
  const uint8_t* img;    // T0 basis image
  float4* fine;          // FP32 spinors [rhs][6][V]
  int nrhs;
  int* err;
};

// Roles: warps 0-3 read the accumulators and store the fine fields (TMEM
// lanes = the 128 sites of a tile), warp 4 lane 0 streams the basis tiles
// into S stages by bulk copies, warp 5 lane 0 issues the MMAs, warp 6
// writes each unit's coefficient image into one of two buffers.  The two
// tiles h = 0, 1 of one component pair go to the two halves of an
// accumulator pair, so each site's float4 chunk is stored whole.
__global__ void __launch_bounds__(PT_THREADS, 2) prolong_tc_kernel(PtRun run, BlockGeo g, int nv, int nstages) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int KC = nv / 4, nhalf = g.nB / 128, ntile = 6 * nhalf, n2 = 2 * nv;
  const uint32_t a_bytes = (uint32_t)KC * 16 * 128;
  const uint32_t b_bytes = (uint32_t)KC * (RT_N / 8) * 128;  // one chirality
  const int S = nstages;
  uint8_t* bbuf = sm + (size_t)S * a_bytes;  // [2 units][2 chiralities]
  uint64_t* bars = reinterpret_cast<uint64_t*>(bbuf + 4 * (size_t)b_bytes);
  uint64_t* afull = bars;                      // [S]
  uint64_t* aempty = bars + PT_MAX_STAGES;     // [S]
  uint64_t* bfull = bars + 2 * PT_MAX_STAGES;  // [2] (32 arrivals)
  uint64_t* bempty = bfull + 2;                // [2]
  uint64_t* accf = bempty + 2;                 // [PT_PAIRS]
  uint64_t* acce = accf + PT_PAIRS;            // [PT_PAIRS] (4 arrivals)
  uint64_t* done = acce + PT_PAIRS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int abort_flag;
  volatile int* abrt = &abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int ntiles = (run.nrhs + RT_NT - 1) / RT_NT;
  const int64_t nunits = g.V1 * ntiles;
  constexpr uint32_t TMEM_COLS = PT_PAIRS * 2 * RT_N;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int b = 0; b < S; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(afull + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(aempty + b)));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(smem_u32(bfull + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bempty + b)));
    }
    for (int b = 0; b < PT_PAIRS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(accf + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(acce + b)));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  auto give_up = [&](int code) {
    abort_flag = 1;
    atomicExch(run.err, code);
  };
  if (warp == 6) {
    // ------------------------------------------------------------ coefficient image: group (r, alpha,
    // octet o) holds 8 coarse values, written as four 16-byte rows (p, n) of the K chunks o (p = 0)
    // and Nv / 8 + o (p = 1)
    const int NO = nv / 8;
    uint32_t ua = 0;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x, ++ua) {
      const int64_t y = u / ntiles;
      const int t = (int)(u % ntiles);
      const uint32_t ub = ua & 1u, bph = (ua >> 1) & 1u;
      const bool free_b = mbar_wait(smem_u32(bempty + ub), bph ^ 1u, abrt);
      if (!__all_sync(0xffffffffu, free_b)) {
        if (lane == 0 && !*abrt) give_up(11);
        break;
      }
      uint4* bw = reinterpret_cast<uint4*>(bbuf + (size_t)ub * 2 * b_bytes);
      for (int idx = lane; idx < RT_NT * 2 * NO; idx += 32) {
        const int r = idx / (2 * NO), ao = idx % (2 * NO), alpha = ao / NO, o = ao % NO;
        const int rr = t * RT_NT + r;
        float4 c4[4];
        if (rr < run.nrhs) {
          const float4* src =
              reinterpret_cast<const float4*>(run.coarse + ((size_t)rr * g.V1 + y) * n2 + alpha * nv + 8 * o);
#pragma unroll
          for (int q = 0; q < 4; ++q) c4[q] = __ldg(src + q);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) c4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const uint4 re = make_uint4(rt_pack(c4[0].x, c4[0].z), rt_pack(c4[1].x, c4[1].z), rt_pack(c4[2].x, c4[2].z),
                                    rt_pack(c4[3].x, c4[3].z));
        const uint4 im = make_uint4(rt_pack(c4[0].y, c4[0].w), rt_pack(c4[1].y, c4[1].w), rt_pack(c4[2].y, c4[2].w),
                                    rt_pack(c4[3].y, c4[3].w));
        const uint4 nim = make_uint4(im.x ^ 0x80008000u, im.y ^ 0x80008000u, im.z ^ 0x80008000u, im.w ^ 0x80008000u);
        uint4* ba = bw + alpha * (KC * RT_N);
        ba[o * RT_N + r] = re;
        ba[o * RT_N + RT_NT + r] = im;
        ba[(NO + o) * RT_N + r] = nim;
        ba[(NO + o) * RT_N + RT_NT + r] = re;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bfull + ub)) : "memory");
    }
  } else if (warp == 4) {
    // ------------------------------------------------------------ basis tiles, in the MMA's order
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const int64_t y = u / ntiles;
        for (int at = 0; at < 2 * ntile; ++at, ++it) {
          const int st = (int)(it % S);
          const uint32_t ph = (it / S) & 1u;
          if (!mbar_wait(smem_u32(aempty + st), ph ^ 1u, abrt)) {
            if (!*abrt) give_up(12);
            ok = false;
            break;
          }
          const uint32_t bar = smem_u32(afull + st);
          const uint8_t* src = run.img + ((size_t)y * 2 * ntile + at) * a_bytes;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(a_bytes) : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(sm + (size_t)st * a_bytes)),
              "l"(src), "r"(a_bytes), "r"(bar)
              : "memory");
        }
      }
      for (uint32_t st = 0; st < (uint32_t)S && st < it; ++st) {
        const uint32_t fills = (it - st + S - 1) / S;
        mbar_wait(smem_u32(afull + st), (fills - 1) & 1u, nullptr);
      }
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA: tiles h = 0, 1 of a pair into the
    // two halves of accumulator pair sp
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, RT_N);
      const uint32_t lboA = 16u * 128u, lboB = (uint32_t)(RT_N / 8) * 128;
      uint32_t it = 0, tp = 0, ua = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++ua) {
        const uint32_t ub = ua & 1u, bph = (ua >> 1) & 1u;
        if (!mbar_wait(smem_u32(bfull + ub), bph, abrt)) {
          if (!*abrt) give_up(13);
          break;
        }
        for (int alpha = 0; alpha < 2 && ok; ++alpha)
          for (int mp = 0; mp < ntile / 2 && ok; ++mp, ++tp) {
            const uint32_t sp = tp % PT_PAIRS, aph = (tp / PT_PAIRS) & 1u;
            if (!mbar_wait(smem_u32(acce + sp), aph ^ 1u, abrt)) {
              if (!*abrt) give_up(14);
              ok = false;
              break;
            }
            for (int h = 0; h < 2; ++h, ++it) {
              const int st = (int)(it % S);
              const uint32_t ph = (it / S) & 1u;
              if (!mbar_wait(smem_u32(afull + st), ph, abrt)) {
                if (!*abrt) give_up(16);
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
              const uint32_t a0 = smem_u32(sm + (size_t)st * a_bytes);
              const uint32_t b0 = smem_u32(bbuf + ((size_t)ub * 2 + alpha) * b_bytes);
              const uint32_t d = tmem + (sp * 2 + h) * RT_N;
              for (int i = 0; i < KC / 2; ++i) {
                const uint64_t ad = smem_desc(a0 + i * 2 * lboA, lboA, 128);
                const uint64_t bd = smem_desc(b0 + i * 2 * lboB, lboB, 128);
                const uint32_t acc = i > 0 ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
              }
              asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_u32(aempty + st)));
            }
            if (!ok) break;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(accf + sp)));
          }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bempty + ub)));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(done)));
      mbar_wait(smem_u32(done), 0u, nullptr);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 0-3: TMEM lanes = sites)
    uint32_t tp = 0;
    bool ok = true;
    const int kk = warp * 32 + lane;
    for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      const int64_t y = u / ntiles;
      const int t = (int)(u % ntiles);
      int64_t site_h[4];
      for (int hf = 0; hf < nhalf; ++hf) site_h[hf] = rt_block_site(g, y, 128 * hf + kk);
      for (int alpha = 0; alpha < 2 && ok; ++alpha)
        for (int mp = 0; mp < ntile / 2; ++mp, ++tp) {
          const uint32_t sp = tp % PT_PAIRS, aph = (tp / PT_PAIRS) & 1u;
          const bool mine = mbar_wait(smem_u32(accf + sp), aph, abrt);
          if (!__all_sync(0xffffffffu, mine)) {
            if (lane == 0 && !*abrt) give_up(15);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          uint32_t v[2 * RT_N];
          tmem_ld<2 * RT_N>(tmem + ((uint32_t)(warp * 32) << 16) + sp * 2 * RT_N, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acce + sp)) : "memory");
          const int hf = mp % nhalf, cq = mp / nhalf;
          float4* f = run.fine + ((size_t)t * RT_NT * 6 + 3 * (size_t)alpha + cq) * g.V + site_h[hf];
#pragma unroll
          for (int r = 0; r < RT_NT; ++r)
            if (t * RT_NT + r < run.nrhs)
              f[(size_t)r * 6 * g.V] = make_float4(__uint_as_float(v[r]), __uint_as_float(v[RT_NT + r]),
                                                   __uint_as_float(v[RT_N + r]), __uint_as_float(v[RT_N + RT_NT + r]));
        }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ============================================================ host side
bool restrict_tc_supported(const mglma_subspace_s* S) {
  return S->nv % 8 == 0 && S->nv <= 32 && S->geo.nB % RT_SEG == 0 && S->geo.nB <= RT_MAX_NB &&
         (S->phi16 || S->phi32);
}

static mglma_status rt_image_ready(mglma_ctx ctx, mglma_subspace_s* S, cudaStream_t s) {
  if (S->rt_img) return MGLMA_OK;
  const BlockGeo& g = S->geo;
  const size_t n = (size_t)g.V1 * 2 * 3 * (g.nB / RT_SEG) * RT_CH * (S->nv / 8) * 64;  // BF16 values
  MG_CUDA(cudaMalloc(&S->rt_img, n * sizeof(uint16_t)));
  MG_CUDA(cudaMalloc(&S->rt_err, sizeof(int)));
  MG_CUDA(cudaMemsetAsync(S->rt_err, 0, sizeof(int), s));
  ProfScope ps(ctx, K_SETUP, s);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (S->phi16)
    rt_image_kernel<__half><<<blocks, 256, 0, s>>>(S->phi16, S->scale16, g, S->nv, S->rt_img);
  else
    rt_image_kernel<float><<<blocks, 256, 0, s>>>(S->phi32, nullptr, g, S->nv, S->rt_img);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status restrict_tc(mglma_ctx ctx, mglma_subspace_s* S, const Spinor& in, void* out, cudaStream_t s) {
  if (!restrict_tc_supported(S)) return fail(MGLMA_ERR_INVALID, "restrict_tc: Nv % 8, block size or basis not supported");
  if (in.prec != MGLMA_FP32 || in.V != S->geo.V) return fail(MGLMA_ERR_INVALID, "restrict_tc: FP32 fine fields needed");
  if (in.nrhs == 0) return MGLMA_OK;
  MG_CHECK(rt_image_ready(ctx, S, s));
  const BlockGeo& g = S->geo;
  const uint32_t stage = (uint32_t)RT_CH * (S->nv / 8) * 128 + RT_B_BYTES;
  // two CTAs per SM: half of 227 KB each, less the barriers, the site table
  // and 1 KB of static shared memory
  const size_t fixed = (size_t)(3 * RT_MAX_STAGES + 8) * 8 + (size_t)RT_MAX_NB * 8;
  const int S_ = (int)std::min<size_t>(RT_MAX_STAGES, (113 * 1024 - 1024 - fixed) / stage);
  const size_t smem = (size_t)S_ * stage + fixed;
  {
    static std::mutex mu;
    static size_t granted = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (smem > granted) {
      MG_CUDA(cudaFuncSetAttribute(restrict_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      granted = smem;
    }
  }
  const int64_t units = g.V1 * ((in.nrhs + RT_NT - 1) / RT_NT);
  const unsigned grid = (unsigned)std::min<int64_t>(units, 2 * (int64_t)ctx->sm_count);
  RtRun run;
  run.fine = (const float4*)in.p;
  run.img = (const uint8_t*)S->rt_img;
  run.out = (float2*)out;
  run.nrhs = in.nrhs;
  run.err = S->rt_err;
  {
    // algorithmic bytes: the basis image once per RHS tile, the fields once
    const double V = (double)g.V, V1 = (double)g.V1, n2 = 2.0 * S->nv, N = in.nrhs;
    ProfScope ps(ctx, K_RESTRICT, s, V * n2 * 6.0 * 4.0 * std::ceil(N / RT_NT) + N * (V * 96.0 + V1 * n2 * 8.0),
                 8.0 * V * 12.0 * S->nv * N);
    restrict_tc_kernel<<<grid, RT_THREADS, smem, s>>>(run, g, S->nv, S_);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

bool prolong_tc_supported(const mglma_subspace_s* S) {
  return S->nv % 8 == 0 && S->nv <= 32 && S->geo.nB % 128 == 0 && S->geo.nB <= 512 && (S->phi16 || S->phi32);
}

static mglma_status pt_image_ready(mglma_ctx ctx, mglma_subspace_s* S, cudaStream_t s) {
  if (S->pt_img) return MGLMA_OK;
  const BlockGeo& g = S->geo;
  const size_t n = (size_t)g.V1 * 2 * 6 * (g.nB / 128) * (S->nv / 4) * 16 * 64;  // BF16 values
  MG_CUDA(cudaMalloc(&S->pt_img, n * sizeof(uint16_t)));
  if (!S->rt_err) {
    MG_CUDA(cudaMalloc(&S->rt_err, sizeof(int)));
    MG_CUDA(cudaMemsetAsync(S->rt_err, 0, sizeof(int), s));
  }
  ProfScope ps(ctx, K_SETUP, s);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (S->phi16)
    pt_image_kernel<__half><<<blocks, 256, 0, s>>>(S->phi16, S->scale16, g, S->nv, S->pt_img);
  else
    pt_image_kernel<float><<<blocks, 256, 0, s>>>(S->phi32, nullptr, g, S->nv, S->pt_img);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status prolong_tc(mglma_ctx ctx, mglma_subspace_s* S, const void* in_coarse, Spinor& out, cudaStream_t s) {
  if (!prolong_tc_supported(S)) return fail(MGLMA_ERR_INVALID, "prolong_tc: Nv % 8, block size or basis not supported");
  if (out.prec != MGLMA_FP32 || out.V != S->geo.V) return fail(MGLMA_ERR_INVALID, "prolong_tc: FP32 fine fields needed");
  if (out.nrhs == 0) return MGLMA_OK;
  MG_CHECK(pt_image_ready(ctx, S, s));
  const BlockGeo& g = S->geo;
  const int KC = S->nv / 4;
  const size_t a_bytes = (size_t)KC * 16 * 128, b_bytes = (size_t)KC * (RT_N / 8) * 128;
  // two CTAs per SM as for R0
  const size_t fixed = 4 * b_bytes + (size_t)(2 * PT_MAX_STAGES + 4 + 2 * PT_PAIRS + 2) * 8;
  const int S_ = (int)std::min<size_t>(PT_MAX_STAGES, (113 * 1024 - 1024 - fixed) / a_bytes);
  const size_t smem = (size_t)S_ * a_bytes + fixed;
  {
    static std::mutex mu;
    static size_t granted = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (smem > granted) {
      MG_CUDA(cudaFuncSetAttribute(prolong_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      granted = smem;
    }
  }
  const int64_t units = g.V1 * ((out.nrhs + RT_NT - 1) / RT_NT);
  const unsigned grid = (unsigned)std::min<int64_t>(units, 2 * (int64_t)ctx->sm_count);
  PtRun run;
  run.coarse = (const float2*)in_coarse;
  run.img = (const uint8_t*)S->pt_img;
  run.fine = (float4*)out.p;
  run.nrhs = out.nrhs;
  run.err = S->rt_err;
  {
    const double V = (double)g.V, V1 = (double)g.V1, n2 = 2.0 * S->nv, N = out.nrhs;
    ProfScope ps(ctx, K_PROLONG, s, V * n2 * 6.0 * 4.0 * std::ceil(N / RT_NT) + N * (V * 96.0 + V1 * n2 * 8.0),
                 8.0 * V * 12.0 * S->nv * N);
    prolong_tc_kernel<<<grid, PT_THREADS, smem, s>>>(run, g, S->nv, S_);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status restrict_tc_check(const mglma_subspace_s* S, cudaStream_t s) {
  if (!S->rt_err) return MGLMA_OK;
  int h = 0;
  MG_CUDA(cudaMemcpyAsync(&h, S->rt_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MG_CUDA(cudaStreamSynchronize(s));
  if (h) {
    MG_CUDA(cudaMemsetAsync(S->rt_err, 0, sizeof(int), s));
    return fail(MGLMA_ERR_TIMEOUT, "tensor-core restriction / prolongation: a bounded wait gave up (code " + std::to_string(h) + ")");
  }
  return MGLMA_OK;
}

}  // namespace mglma
