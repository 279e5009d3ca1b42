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
// ([k chunk of 8][row group of 8][8 rows][8 values]); the nine slots are nine
// contiguous blocks.  A first kernel writes X once per call as the matching
// B blocks (one per site and RHS tile, shared by the nine sites that use it).
// The stencil kernel then only moves bytes with bulk async copies: a ring of
// shared-memory stages, one stencil slot (A_d and B_d) per stage, filled by
// one thread, drained by one MMA-issuing thread, with the accumulator of
// consecutive work units alternating between two TMEM buffers so that the
// epilogue of one unit overlaps the MMAs of the next.  Two CTAs share an SM,
// so one CTA's copies proceed while the other waits for its MMAs to finish
// reading a stage.  The MMA shape is
// M = 128 (rows >= n2 read neighbouring shared memory and are never stored).
//
// Every mbarrier wait is bounded: on a timeout the kernel records an error,
// the other roles stop at their next wait, the copy thread waits (bounded)
// for its copies in flight, the MMA thread for its MMAs, TMEM is freed and
// the kernel returns; the host reports MGLMA_ERR_TIMEOUT.
#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"
#include "lattice.cuh"
#include "tcgen05.cuh"
#include "solver.h"
#include "subspace.h"

namespace mglma {

constexpr int TC_THREADS = 128;  // warps 0-1 epilogue, warp 2 copies, warp 3 MMA
constexpr int TC_EPI_WARPS = 2;    // TMEM lanes 0..63 (rows i < n2 <= 48)
constexpr int TC_MAX_STAGES = 16;
constexpr uint32_t TC_PAD = 2048;  // M = 128 rows read past the n2 real rows
// B-operand image of X for RHS tiles of NT: per (tile t, site z) the rows
// k = (part, j) of one slot, 2 G chunks of 8, times N = 2 NT columns, in the
// no-swizzle K-major order [chunk c][column group][8 columns][8 k] (16-byte
// row (c, n) at index c N + n):
//   part 0: column r <- Re X_j,r, column NT + r <- Im X_j,r
//   part 1: column r <- -Im X_j,r, column NT + r <- Re X_j,r
// RHS beyond nrhs are zero; mode bit 0 applies gamma5hat (j >= nv negated).
// the four 16-byte rows of dof group jo (8 dofs) for column ri of a tile,
// dst = the image of one (tile, site)
__device__ __forceinline__ void x_image_store(uint4* dst, int jo, int G, int NT, int ri, const float* re,
                                              const float* im) {
  uint32_t w[3][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    w[0][e] = (uint32_t)bf16_bits(re[2 * e]) | ((uint32_t)bf16_bits(re[2 * e + 1]) << 16);
    w[1][e] = (uint32_t)bf16_bits(im[2 * e]) | ((uint32_t)bf16_bits(im[2 * e + 1]) << 16);
    w[2][e] = (uint32_t)bf16_bits(-im[2 * e]) | ((uint32_t)bf16_bits(-im[2 * e + 1]) << 16);
  }
  const int N = 2 * NT;
  dst[(size_t)jo * N + ri] = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
  dst[(size_t)jo * N + NT + ri] = make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
  dst[(size_t)(G + jo) * N + ri] = make_uint4(w[2][0], w[2][1], w[2][2], w[2][3]);
  dst[(size_t)(G + jo) * N + NT + ri] = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
}

__global__ void x_image_kernel(const float2* __restrict__ X, uint4* __restrict__ XB, int64_t V1, int n2, int nrhs,
                               int NT, int mode) {
  // one thread per (tile t, site z, group jo of 8 dofs, RHS r of the tile):
  // reads the group's 64 bytes of X once and writes its four 16-byte rows
  const int G = n2 / 8, N = 2 * NT, nv = n2 / 2;
  const size_t rows = (size_t)2 * G * N;  // 16-byte rows per (tile, site)
  const size_t ntiles = (size_t)(nrhs + NT - 1) / NT;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= ntiles * V1 * G * NT) return;
  const int ri = (int)(u % NT);
  const int jo = (int)((u / NT) % G);
  const int64_t z = (int64_t)((u / ((size_t)NT * G)) % V1);
  const int t = (int)(u / ((size_t)NT * G * V1));
  const int rr = t * NT + ri;
  float re[8] = {}, im[8] = {};
  if (rr < nrhs) {
    const float4* src = reinterpret_cast<const float4*>(X + ((size_t)rr * V1 + z) * n2 + jo * 8);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const float4 q = __ldg(src + h);
      re[2 * h] = q.x;
      im[2 * h] = q.y;
      re[2 * h + 1] = q.z;
      im[2 * h + 1] = q.w;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float sg = ((mode & 1) && jo * 8 + e >= nv) ? -1.f : 1.f;
      re[e] *= sg;
      im[e] *= sg;
    }
  }
  x_image_store(XB + ((size_t)t * V1 + z) * rows, jo, G, NT, ri, re, im);
}

// The coarse MINRES update (w_new = cf0 v + cf1 w1 + cf2 w2, x += cf3 w_new,
// z *= cf4 for RHS with cf5 != 0; cf_j[r] = cf[j stride + r]) on FP32
// half-lattice fields, which also writes the B-operand image (tiles of NT,
// no gamma5hat) of the scaled z -- the next iteration's Lanczos vector -- so
// its operator application needs no image pass.  One thread per (site, group
// of 8 dofs) of RHS blockIdx.y.
__global__ void minres_update_image_kernel(const float4* __restrict__ v, const float4* __restrict__ w1,
                                           const float4* __restrict__ w2, float4* __restrict__ wn,
                                           float4* __restrict__ x, float4* __restrict__ z,
                                           const double* __restrict__ cf, int stride, int64_t Vh, int n2, int NT,
                                           uint4* __restrict__ XB) {
  const int r = blockIdx.y;
  if (cf[5 * (size_t)stride + r] == 0.0) return;
  const float c0 = (float)cf[r], c1 = (float)cf[stride + r], c2 = (float)cf[2 * (size_t)stride + r],
              c3 = (float)cf[3 * (size_t)stride + r], c4 = (float)cf[4 * (size_t)stride + r];
  const int G = n2 / 8;
  const size_t ng = (size_t)Vh * G, off = (size_t)r * Vh * (n2 / 2);
  const size_t rows = (size_t)2 * G * 2 * NT;
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (size_t)gridDim.x * blockDim.x) {
    float re[8], im[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const size_t i = off + 4 * g + q;
      const float4 a = v[i], b = w1[i], c = w2[i];
      const float4 w = make_float4(c0 * a.x + c1 * b.x + c2 * c.x, c0 * a.y + c1 * b.y + c2 * c.y,
                                   c0 * a.z + c1 * b.z + c2 * c.z, c0 * a.w + c1 * b.w + c2 * c.w);
      wn[i] = w;
      const float4 xo = x[i];
      x[i] = make_float4(xo.x + c3 * w.x, xo.y + c3 * w.y, xo.z + c3 * w.z, xo.w + c3 * w.w);
      const float4 zo = z[i];
      const float4 zn = make_float4(c4 * zo.x, c4 * zo.y, c4 * zo.z, c4 * zo.w);
      z[i] = zn;
      re[2 * q] = zn.x;
      im[2 * q] = zn.y;
      re[2 * q + 1] = zn.z;
      im[2 * q + 1] = zn.w;
    }
    x_image_store(XB + ((size_t)(r / NT) * Vh + (int64_t)(g / G)) * rows, (int)(g % G), G, NT, r % NT, re, im);
  }
}

// Warp-specialised persistent kernel: CTA b takes sites y = b, b + grid, ...
// and every RHS tile of each; a work unit (site, tile) runs through nine
// pipeline stages, one per stencil slot d, each holding the slot's operator
// block A_d (n2 x 2 n2 BF16) and the B image of X at nbr_d(y).
//   warp 2 (one lane): waits for a free stage, bulk-copies A_d and B_d into it
//   warp 3 (one lane): waits for a full stage, issues the slot's MMAs into the
//     unit's accumulator (two TMEM buffers, alternating by unit), commits the
//     stage back to warp 2 and, after slot 8, the accumulator to the epilogue
//   warps 0-1: read the accumulator (rows = TMEM lanes), release it, store Y
// One launch of the stencil: which sites, which slots, which operands.
//   par < 0: every site y, fields indexed by y;  par = 0 / 1: the sites of
//     that parity (x0 + x1 + x2 + x3 mod 2), fields of half the sites indexed
//     by y >> 1 (every extent even, so y and y + 1 differ in parity) -- the
//     hop slots then read a field of the other parity, the self slot one of
//     the same parity (even-odd preconditioning)
//   slots d_lo .. d_hi of the nine (0..8 all, 0..7 the hops, 8 the self block)
//   A: operator image (nine slots per site); Aself: a one-slot-per-site image
//     that replaces slot 8 (NULL: slot 8 of A)
//   XB / XBself: B images for the hop slots / the self slot
//   Y = sign * (the sum), gamma5hat on rows by mode bit 1 as before
struct TcRun {
  const uint8_t* A;
  const uint8_t* Aself;
  // optional dot in the epilogue (one RHS tile only): dout[r] = <dotX_r, Y_r>
  // = sum conj(dotX) Y over this launch's units, per-CTA partials in dpart
  // ([CTA][nrhs]) summed in a fixed order by the last CTA (ticket dcount)
  const float2* dotX;
  double2* dpart;
  unsigned* dcount;
  double2* dout;
  int a_unit;  // 1: A holds eight hop slots per unit u ([u][8]), else nine per site ([y][9])
  const uint8_t* XB;
  const uint8_t* XBself;
  float2* Y;
  int d_lo, d_hi;
  int par;
  float sign;
};

// site of parity `par` with half-lattice index u (needs an even extent L3)
__device__ __forceinline__ int64_t parity_site(const LatIdx& q, int64_t u, int par) {
  const int64_t y0 = 2 * u;
  int xc[4];
  site_coords(q, y0, xc);
  return y0 + ((par ^ (xc[0] + xc[1] + xc[2] + xc[3])) & 1);
}

template <int NT>
__global__ void __launch_bounds__(TC_THREADS, 2)
    coarse_tc_kernel(TcRun run, LatIdx q, int n2, int nrhs, int mode, int nstages, int* __restrict__ err) {
  constexpr int N = 2 * NT;
  constexpr uint32_t TMEM_COLS = 2 * N < 32 ? 32 : 2 * N;
  extern __shared__ __align__(1024) uint8_t sm[];
  const int G = n2 / 8;
  const uint32_t a_slot = (uint32_t)256 * G * G;  // 2 G chunks x G row groups x 128 B
  const uint32_t b_slot = (uint32_t)32 * G * N;   // 2 G chunks x N/8 column groups x 128 B
  const uint32_t stage_bytes = a_slot + b_slot;
  const int S = nstages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (size_t)S * stage_bytes + TC_PAD);
  uint64_t* full = bars;                  // [S] copies landed
  uint64_t* empty = bars + TC_MAX_STAGES;  // [S] MMAs done reading
  uint64_t* accf = bars + 2 * TC_MAX_STAGES;
  uint64_t* acce = accf + 2;
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int abort_flag;
  volatile int* abrt = &abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int64_t nunits = run.par < 0 ? q.V : q.V / 2;  // sites this launch computes (and field length)
  const int ntiles = (nrhs + NT - 1) / NT;
  const int nslots = run.d_hi - run.d_lo + 1;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int b = 0; b < S; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(empty + b)));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(accf + b)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(acce + b)), "r"(TC_EPI_WARPS));
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
    atomicExch(err, code);
  };

  float dre[NT], dim[NT];  // epilogue: this thread's share of the optional dot
#pragma unroll
  for (int r = 0; r < NT; ++r) dre[r] = dim[r] = 0.f;

  if (warp == 2) {
    // ------------------------------------------------------------ copies
    uint32_t it = 0;
    if (lane == 0) {
      bool ok = true;
      for (int64_t u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const int64_t y = run.par < 0 ? u : parity_site(q, u, run.par);
        int xx[4];
        site_coords(q, y, xx);
        // row of the B image slot d reads: the neighbour (full or half-lattice
        // index), or this unit for the self slot (constant-index cases only,
        // so nothing lands in local memory)
        auto row_of = [&](int d) -> int64_t {
          int64_t z;
          switch (d) {
            case 0: z = nbr_fwd(q, y, xx, 0); break;
            case 1: z = nbr_fwd(q, y, xx, 1); break;
            case 2: z = nbr_fwd(q, y, xx, 2); break;
            case 3: z = nbr_fwd(q, y, xx, 3); break;
            case 4: z = nbr_bwd(q, y, xx, 0); break;
            case 5: z = nbr_bwd(q, y, xx, 1); break;
            case 6: z = nbr_bwd(q, y, xx, 2); break;
            case 7: z = nbr_bwd(q, y, xx, 3); break;
            default: return u;
          }
          return run.par >= 0 ? (z >> 1) : z;
        };
        for (int t = 0; t < ntiles && ok; ++t) {
          for (int d = run.d_lo; d <= run.d_hi; ++d, ++it) {
            const int st = (int)(it % S);
            const uint32_t ph = (it / S) & 1u;
            if (!mbar_wait(smem_u32(empty + st), ph ^ 1u, abrt)) {
              if (!*abrt) give_up(1);
              ok = false;
              break;
            }
            const uint32_t bar = smem_u32(full + st);
            const uint32_t dst = smem_u32(sm + (size_t)st * stage_bytes);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(stage_bytes)
                         : "memory");
            const uint8_t* srcA = (d == 8 && run.Aself) ? run.Aself + (size_t)y * a_slot
                                  : run.a_unit          ? run.A + ((size_t)u * 8 + d) * a_slot
                                                        : run.A + ((size_t)y * 9 + d) * a_slot;
            const uint8_t* srcB = (d == 8 ? run.XBself : run.XB) + ((size_t)t * nunits + row_of(d)) * b_slot;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                "l"(srcA), "r"(a_slot), "r"(bar)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    dst + a_slot),
                "l"(srcB), "r"(b_slot), "r"(bar)
                : "memory");
          }
        }
      }
      // copies still in flight (after an abort): wait for each stage's last
      // fill, bounded and regardless of the abort flag
      for (uint32_t st = 0; st < (uint32_t)S && st < it; ++st) {
        const uint32_t fills = (it - st + S - 1) / S;
        mbar_wait(smem_u32(full + st), (fills - 1) & 1u, nullptr);
      }
    }
  } else if (warp == 3) {
    // ------------------------------------------------------------ MMA
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, N);
      const uint32_t lboA = (uint32_t)G * 128, lboB = (uint32_t)(N / 8) * 128;
      uint32_t it = 0, u = 0;
      bool ok = true;
      for (int64_t y = blockIdx.x; y < nunits && ok; y += gridDim.x) {
        for (int t = 0; t < ntiles && ok; ++t, ++u) {
          const uint32_t b = u & 1u, aph = (u >> 1) & 1u;
          if (!mbar_wait(smem_u32(acce + b), aph ^ 1u, abrt)) {
            if (!*abrt) give_up(2);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t dcol = tmem + b * N;
          for (int d = 0; d < nslots; ++d, ++it) {
            const int st = (int)(it % S);
            const uint32_t ph = (it / S) & 1u;
            if (!mbar_wait(smem_u32(full + st), ph, abrt)) {
              if (!*abrt) give_up(3);
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sm + (size_t)st * stage_bytes), b0 = a0 + a_slot;
            for (int kk = 0; kk < G; ++kk) {
              const uint64_t ad = smem_desc(a0 + kk * 2 * lboA, lboA, 128);
              const uint64_t bd = smem_desc(b0 + kk * 2 * lboB, lboB, 128);
              const uint32_t acc = (d > 0 || kk > 0) ? 1u : 0u;
              asm volatile(
                  "{\n\t.reg .pred p;\n\t"
                  "setp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(empty + st)));
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(accf + b)));
        }
      }
      // every MMA issued by this thread has completed before TMEM is freed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(done)));
      mbar_wait(smem_u32(done), 0u, nullptr);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    uint32_t u = 0;
    const int i = warp * 32 + lane;
    const float sg = ((mode & 2) && i >= n2 / 2) ? -run.sign : run.sign;
    bool ok = true;
    for (int64_t y = blockIdx.x; y < nunits && ok; y += gridDim.x) {
      for (int t = 0; t < ntiles; ++t, ++u) {
        const uint32_t b = u & 1u, aph = (u >> 1) & 1u;
        // the dot's operand is fetched before the wait, so its latency
        // overlaps the MMAs of this unit
        float2 xq[NT];
        if (run.dotX) {
#pragma unroll
          for (int r = 0; r < NT; ++r)
            xq[r] = (i < n2 && t * NT + r < nrhs)
                        ? __ldg(run.dotX + ((size_t)(t * NT + r) * nunits + y) * n2 + i)
                        : make_float2(0.f, 0.f);
        }
        // every lane waits; the warp proceeds only if all saw the phase
        const bool mine = mbar_wait(smem_u32(accf + b), aph, abrt);
        if (!__all_sync(0xffffffffu, mine)) {
          if (lane == 0 && !*abrt) give_up(4);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        uint32_t v[N];
        tmem_ld<N>(tmem + ((uint32_t)(warp * 32) << 16) + b * N, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acce + b)) : "memory");
        if (i < n2) {
          const int r0 = t * NT;
#pragma unroll
          for (int r = 0; r < NT; ++r)
            if (r0 + r < nrhs) {
              const size_t e = ((size_t)(r0 + r) * nunits + y) * n2 + i;
              const float yr = sg * __uint_as_float(v[r]), yi = sg * __uint_as_float(v[NT + r]);
              run.Y[e] = make_float2(yr, yi);
              if (run.dotX) {
                dre[r] += xq[r].x * yr + xq[r].y * yi;
                dim[r] += xq[r].x * yi - xq[r].y * yr;
              }
            }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  if (run.dotX) {
    // the pipeline is drained: the stage buffers hold the reduction
#pragma unroll
    for (int r = 0; r < NT; ++r)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dre[r] += __shfl_down_sync(0xffffffffu, dre[r], o);
        dim[r] += __shfl_down_sync(0xffffffffu, dim[r], o);
      }
    float* red = reinterpret_cast<float*>(sm);  // [warp][2 NT]
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        red[warp * 2 * NT + r] = dre[r];
        red[warp * 2 * NT + NT + r] = dim[r];
      }
    __syncthreads();
    if (tid < nrhs && tid < NT) {
      double a = 0, c = 0;
      for (int w2 = 0; w2 < TC_THREADS / 32; ++w2) {
        a += (double)red[w2 * 2 * NT + tid];
        c += (double)red[w2 * 2 * NT + NT + tid];
      }
      run.dpart[(size_t)blockIdx.x * nrhs + tid] = make_double2(a, c);
    }
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (tid == 0) last = atomicAdd(run.dcount, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
      // all threads: RHS r = tid / GL summed by GL consecutive lanes, each over
      // a fixed stride of the CTA partials, then a fixed shuffle tree
      __threadfence();
      constexpr int GL = TC_THREADS / NT;
      const int r = tid / GL, l = tid % GL;
      double a = 0, c = 0;
      if (r < nrhs) {
#pragma unroll 4
        for (unsigned b2 = l; b2 < gridDim.x; b2 += GL) {
          const double2 q = __ldcg(run.dpart + (size_t)b2 * nrhs + r);
          a += q.x;
          c += q.y;
        }
      }
#pragma unroll
      for (int o = GL / 2; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o, GL);
        c += __shfl_down_sync(0xffffffffu, c, o, GL);
      }
      if (l == 0 && r < nrhs) run.dout[r] = make_double2(a, c);
      if (tid == 0) *run.dcount = 0;
    }
  }
}

// operator image for the kernel: per site [c][g][8 rows][8 bf16] with
// k = 8c + kk = (d * 2 + part) * n2 + j and row i = 8g + ri, from nslots
// blocks per site of A64 ([site][slot][col j][row i])
__global__ void a_image_kernel(const double2* __restrict__ A64, uint16_t* __restrict__ img, int64_t V1, int n2,
                               int nslots) {
  const size_t per = (size_t)2 * nslots * n2 * n2;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * V1) return;
  const int64_t y = (int64_t)(t / per);
  const size_t e = t % per;
  const int G = n2 / 8;
  const int kk = (int)(e % 8), ri = (int)((e / 8) % 8), g = (int)((e / 64) % G), c = (int)(e / (64 * (size_t)G));
  const int i = 8 * g + ri, k = 8 * c + kk;
  const int d = k / (2 * n2), part = (k / n2) % 2, j = k % n2;
  const double2 a = A64[(((size_t)y * nslots + d) * n2 + j) * n2 + i];
  img[t] = bf16_bits((float)(part ? a.y : a.x));
}

bool coarse_tc_supported(int n2) { return n2 % 8 == 0 && n2 >= 8 && n2 <= 48; }

static uint32_t tc_stage_bytes(int n2, int NT) {
  const uint32_t G = n2 / 8;
  return 256 * G * G + 32 * G * 2 * NT;
}
static int tc_stages(int n2, int NT) {
  // two CTAs per SM (half of 227 KB each), less the pad, the barriers and
  // 1 KB of static shared memory
  const size_t avail = 113 * 1024 - 1024 - TC_PAD - (2 * TC_MAX_STAGES + 5) * 8 - 16;
  return (int)std::min<size_t>(TC_MAX_STAGES, avail / tc_stage_bytes(n2, NT));
}
static size_t tc_smem(int n2, int NT) {
  return (size_t)tc_stages(n2, NT) * tc_stage_bytes(n2, NT) + TC_PAD + (2 * TC_MAX_STAGES + 5) * 8 + 16;
}

size_t coarse_tc_scratch_bytes(const mglma_coarse_s* C, int nrhs) {
  // B images of X for RHS rounded up to the widest tile (32)
  return (size_t)((nrhs + 31) / 32 * 32) * C->geo.V1 * C->n2 * 8;
}

mglma_status coarse_tc_image(mglma_ctx ctx, mglma_coarse_s* C, cudaStream_t s) {
  const size_t n = (size_t)18 * C->n2 * C->n2 * C->geo.V1;
  MG_CUDA(cudaMalloc(&C->Aimg, n * sizeof(uint16_t)));
  MG_CUDA(cudaMalloc(&C->tc_err, sizeof(int)));
  MG_CUDA(cudaMemsetAsync(C->tc_err, 0, sizeof(int), s));
  // epilogue-dot partials: at most two CTAs per SM, one RHS tile of <= 32
  MG_CUDA(cudaMalloc(&C->tc_dpart, sizeof(double2) * 2 * (size_t)ctx->sm_count * 32));
  MG_CUDA(cudaMalloc(&C->tc_dcount, sizeof(unsigned)));
  MG_CUDA(cudaMemsetAsync(C->tc_dcount, 0, sizeof(unsigned), s));
  ProfScope ps(ctx, K_SETUP, s);
  a_image_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C->A64, C->Aimg, C->geo.V1, C->n2, 9);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// The dynamic shared memory granted to coarse_tc_kernel<NT>: one record per
// instantiation shared by every launcher, raised only (a second record could
// lower the grant below what the first believes it holds).
template <int NT>
static mglma_status tc_grant_smem(size_t smem) {
  static std::mutex mu;
  static size_t granted = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (smem <= granted) return MGLMA_OK;
  MG_CUDA(cudaFuncSetAttribute(coarse_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  granted = smem;
  return MGLMA_OK;
}

template <int NT>
static mglma_status launch_tc(mglma_ctx ctx, const mglma_coarse_s* C, const float2* X, float2* Y, int nrhs, int mode,
                              void* xb, int* err, cudaStream_t s) {
  const int n2 = C->n2;
  const int64_t V1 = C->geo.V1;
  {
    const size_t groups = (size_t)((nrhs + NT - 1) / NT) * V1 * (n2 / 8) * NT;
    x_image_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, s>>>(X, (uint4*)xb, V1, n2, nrhs, NT, mode);
    MG_LAUNCH_CHECK();
  }
  const size_t smem = tc_smem(n2, NT);
  MG_CHECK(tc_grant_smem<NT>(smem));
  // two resident CTAs per SM: while one waits for its MMAs to release a
  // stage, the other's copies and MMAs proceed
  const unsigned grid = (unsigned)std::min<int64_t>(V1, 2 * (int64_t)ctx->sm_count);
  TcRun run;
  run.A = (const uint8_t*)C->Aimg;
  run.Aself = nullptr;
  run.a_unit = 0;
  run.dotX = nullptr;
  run.dpart = nullptr;
  run.dcount = nullptr;
  run.dout = nullptr;
  run.XB = run.XBself = (const uint8_t*)xb;
  run.Y = Y;
  run.d_lo = 0;
  run.d_hi = 8;
  run.par = -1;
  run.sign = 1.f;
  coarse_tc_kernel<NT><<<grid, TC_THREADS, smem, s>>>(run, make_latidx(C->geo.Lb), n2, nrhs, mode,
                                                      tc_stages(n2, NT), err);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status coarse_tc_image_blocks(mglma_ctx ctx, const double2* A64, int64_t V1, int n2, int nslots,
                                    uint16_t** img, cudaStream_t s) {
  const size_t n = (size_t)2 * nslots * n2 * n2 * V1;
  MG_CUDA(cudaMalloc(img, n * sizeof(uint16_t)));
  ProfScope ps(ctx, K_SETUP, s);
  a_image_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A64, *img, V1, n2, nslots);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// B image bytes of one half-lattice field (RHS rounded up to the widest tile)
size_t coarse_tc_half_image_bytes(const mglma_coarse_s* C, int nrhs) {
  return (size_t)((nrhs + 31) / 32 * 32) * (C->geo.V1 / 2) * C->n2 * 8;
}

template <int NT>
static mglma_status launch_tc_eo(mglma_ctx ctx, const mglma_coarse_s* C, const float2* Xhop, const float2* Xself,
                                 float2* Y, int nrhs, int mode, int par, int d_lo, int d_hi, const uint16_t* Aself,
                                 float sign, void* scratch, cudaStream_t s, const void* self_image,
                                 const uint16_t* Ahop, const float2* dotX, double2* dot_out, bool hop_imaged) {
  const int n2 = C->n2;
  const int64_t Vh = C->geo.V1 / 2;
  const size_t half = coarse_tc_half_image_bytes(C, nrhs);
  uint8_t* xb_hop = (uint8_t*)scratch;
  uint8_t* xb_self = self_image ? (uint8_t*)self_image : xb_hop + half;
  const size_t groups = (size_t)((nrhs + NT - 1) / NT) * Vh * (n2 / 8) * NT;
  // images of the inputs the slots read (gamma5hat on the inputs by mode bit 0)
  if (d_lo < 8 && !hop_imaged)
    x_image_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, s>>>(Xhop, (uint4*)xb_hop, Vh, n2, nrhs, NT, mode);
  if (d_hi == 8 && !self_image)
    x_image_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, s>>>(Xself, (uint4*)xb_self, Vh, n2, nrhs, NT, mode);
  MG_LAUNCH_CHECK();
  const size_t smem = tc_smem(n2, NT);
  MG_CHECK(tc_grant_smem<NT>(smem));
  const unsigned grid = (unsigned)std::min<int64_t>(Vh, 2 * (int64_t)ctx->sm_count);
  TcRun run;
  run.A = Ahop ? (const uint8_t*)Ahop : (const uint8_t*)C->Aimg;
  run.Aself = (const uint8_t*)Aself;
  run.a_unit = Ahop ? 1 : 0;
  run.dotX = dot_out && nrhs <= NT ? dotX : nullptr;
  run.dpart = C->tc_dpart;
  run.dcount = C->tc_dcount;
  run.dout = dot_out;
  run.XB = xb_hop;
  run.XBself = xb_self;
  run.Y = Y;
  run.d_lo = d_lo;
  run.d_hi = d_hi;
  run.par = par;
  run.sign = sign;
  coarse_tc_kernel<NT><<<grid, TC_THREADS, smem, s>>>(run, make_latidx(C->geo.Lb), n2, nrhs, mode & 2,
                                                      tc_stages(n2, NT), C->tc_err);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status coarse_tc_eo_launch(mglma_ctx ctx, const mglma_coarse_s* C, const float2* Xhop, const float2* Xself,
                                 float2* Y, int nrhs, int mode, int par, int d_lo, int d_hi, const uint16_t* Aself,
                                 float sign, void* scratch, cudaStream_t s, const void* self_image,
                                 const uint16_t* Ahop, const float2* dotX, double2* dot_out, bool hop_imaged) {
  if (!C->Aimg || !coarse_tc_supported(C->n2)) return fail(MGLMA_ERR_INVALID, "coarse_tc_eo: no tensor image");
  if (hop_imaged && (mode & 1)) return fail(MGLMA_ERR_INVALID, "coarse_tc_eo: a given hop image carries no gamma5hat");
  if (dot_out && (!dotX || !C->tc_dpart || nrhs > tuned(ctx, TUNE_COARSE_NT, nrhs, C->geo.V1, coarse_tc_default_nt(nrhs))))
    return fail(MGLMA_ERR_INVALID, "coarse_tc_eo: the epilogue dot needs one RHS tile");
  if (par < 0 || par > 1 || d_lo < 0 || d_hi > 8 || d_lo > d_hi)
    return fail(MGLMA_ERR_INVALID, "coarse_tc_eo: bad launch");
  if (Ahop && d_hi > 7) return fail(MGLMA_ERR_INVALID, "coarse_tc_eo: the eight-slot image has no self slot");
  const int nt = tuned(ctx, TUNE_COARSE_NT, nrhs, C->geo.V1, coarse_tc_default_nt(nrhs));
  if (nt == 32)
    return launch_tc_eo<32>(ctx, C, Xhop, Xself, Y, nrhs, mode, par, d_lo, d_hi, Aself, sign, scratch, s, self_image,
                            Ahop, dotX, dot_out, hop_imaged);
  if (nt == 16)
    return launch_tc_eo<16>(ctx, C, Xhop, Xself, Y, nrhs, mode, par, d_lo, d_hi, Aself, sign, scratch, s, self_image,
                            Ahop, dotX, dot_out, hop_imaged);
  return launch_tc_eo<8>(ctx, C, Xhop, Xself, Y, nrhs, mode, par, d_lo, d_hi, Aself, sign, scratch, s, self_image,
                         Ahop, dotX, dot_out, hop_imaged);
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

int coarse_tc_default_nt(int nrhs) { return nrhs <= 8 ? 8 : (nrhs <= 24 ? 16 : 32); }

int coarse_tc_nt(mglma_ctx ctx, const mglma_coarse_s* C, int nrhs) {
  return tuned(ctx, TUNE_COARSE_NT, nrhs, C->geo.V1, coarse_tc_default_nt(nrhs));
}

mglma_status coarse_x_image_half(mglma_ctx ctx, const mglma_coarse_s* C, const void* X, int nrhs, void* image,
                                 cudaStream_t s) {
  if (nrhs == 0) return MGLMA_OK;
  const int n2 = C->n2, NT = coarse_tc_nt(ctx, C, nrhs);
  const int64_t Vh = C->geo.V1 / 2;
  const size_t groups = (size_t)((nrhs + NT - 1) / NT) * Vh * (n2 / 8) * NT;
  ProfScope ps(ctx, K_COARSE, s);
  x_image_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, s>>>((const float2*)X, (uint4*)image, Vh, n2, nrhs, NT,
                                                                 0);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status minres_update_image(mglma_ctx ctx, const mglma_coarse_s* C, const double* cf, int stride, const Vec& v,
                                 const Vec& w1, const Vec& w2, Vec& wn, Vec& x, Vec& z, void* image, cudaStream_t s) {
  const int n2 = C->n2;
  const int64_t Vh = C->geo.V1 / 2;
  if (x.prec != MGLMA_FP32 || n2 % 8 || x.n != (size_t)Vh * n2 * 2 || v.n != x.n || w1.n != x.n || w2.n != x.n ||
      wn.n != x.n || z.n != x.n)
    return fail(MGLMA_ERR_INVALID, "minres_update_image: FP32 half-lattice fields needed");
  if (x.nrhs == 0) return MGLMA_OK;
  const int NT = coarse_tc_nt(ctx, C, x.nrhs);
  ProfScope ps(ctx, K_BLAS, s, 8.0 * x.bytes() + (double)x.nrhs * Vh * n2 * 8.0);
  const size_t ng = (size_t)Vh * (n2 / 8);
  const unsigned gx = (unsigned)std::min<size_t>((ng + 255) / 256, std::max(4, 8 * ctx->sm_count / x.nrhs + 1));
  dim3 g(gx, x.nrhs, 1);
  minres_update_image_kernel<<<g, 256, 0, s>>>((const float4*)v.p, (const float4*)w1.p, (const float4*)w2.p,
                                               (float4*)wn.p, (float4*)x.p, (float4*)z.p, cf, stride, Vh, n2, NT,
                                               (uint4*)image);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status coarse_apply_tc(mglma_ctx ctx, const mglma_coarse_s* C, const float2* X, float2* Y, int nrhs, int mode,
                             void* scratch, size_t scratch_bytes, cudaStream_t s) {
  if (!C->Aimg || !coarse_tc_supported(C->n2)) return fail(MGLMA_ERR_INVALID, "coarse_apply_tc: no tensor image");
  int* err = C->tc_err;
  const int nt = tuned(ctx, TUNE_COARSE_NT, nrhs, C->geo.V1, coarse_tc_default_nt(nrhs));
  const size_t need = coarse_tc_scratch_bytes(C, nrhs);
  void* xb = scratch;
  void* own = nullptr;
  if (!xb || scratch_bytes < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone)
      return fail(MGLMA_ERR_INVALID, "coarse_apply_tc: scratch too small inside a graph capture");
    MG_CHECK(dalloc(ctx, &own, need, s));
    xb = own;
  }
  mglma_status st;
  if (nt == 32)
    st = launch_tc<32>(ctx, C, X, Y, nrhs, mode, xb, err, s);
  else if (nt == 16)
    st = launch_tc<16>(ctx, C, X, Y, nrhs, mode, xb, err, s);
  else
    st = launch_tc<8>(ctx, C, X, Y, nrhs, mode, xb, err, s);
  if (own) dfree(ctx, own, s);
  return st;
}

}  // namespace mglma
