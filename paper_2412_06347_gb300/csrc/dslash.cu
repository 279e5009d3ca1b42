// Wilson-clover operator on GB300: layout conversion, gauge packing with an
// SU(3) check, clover construction, and the multi-RHS stencil.
//
// The operator (O(a)-improved Wilson fermions of Tab. ensembles; Q = gamma5 D
// of Sec. 2):
//   D psi(x) = A(x) psi(x) - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
//                                      + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)]
// in the chiral basis gamma_mu = [[0, e_mu], [e_mu^dag, 0]] with e_0 = -1,
// e_k = -i sigma_k.  (1 + s gamma_mu) psi for s = +-1 has upper half
// h = u + s e_mu l and lower half s e_mu^dag h (u, l: spins {0,1}, {2,3}), so
// each hop moves one two-spin half spinor through the link (spin projection).
//
// Stencil kernel design: one thread per site and NR right-hand sides held in
// registers, so each link and clover entry is read once for NR spinors; the
// spinor layout [rhs][chunk][site] makes every 16-byte load of a warp
// coalesced; neighbours are found arithmetically (no halo, no tables); links
// are stored reconstruct-12 in FP32 with the third row rebuilt in registers.
#include <mutex>
#include <type_traits>
#include <string>

#include "internal.h"
#include "cplx.cuh"
#include "lattice.cuh"
#include "stencil.cuh"

namespace mglma {

// out = op(in) for NR right-hand sides per thread.  DAG selects D^dag
// (projectors 1 +- gamma swap); g5out multiplies the result by gamma5.
// A CTA of 128 threads covers 128 / RW consecutive sites for RW RHS tiles of
// NR: thread t takes site t mod (128 / RW) of the CTA's block and RHS tile
// t / (128 / RW), so with RW > 1 the warps of one CTA read the same links and
// clover entries and all but the first find them in L1.
// resident CTAs per SM the register allocation must allow (128 threads each)
template <typename R, int NR, int RW>
constexpr int dslash_min_ctas() {
  return sizeof(R) == 8 ? 3 : (NR == 1 ? (RW == 1 ? 6 : 5) : (NR == 2 ? 4 : 3));
}

// RED (FP32, one RHS per thread, one RHS tile per CTA only) also reduces, per
// CTA, |t|^2 and <t, in> = sum conj(t) in over the CTA's 128 sites of t = op(in)
// into part[(rhs * nblk + block) * 3 + {0, 1, 2}] (|t|^2, Re, Im): FP32 over
// each warp's 32 sites, FP64 from there on, summed over the blocks in a fixed
// order by dot_finish_kernel.
//
// MRF (with RED) makes the kernel one fused minimal-residual smoothing step:
// with in = t_k and u = op(t_k), per site and RHS
//   out = t_{k+1} = t_k - alpha u,  s <- s_{k+1} = s_k - alpha t_k,
//   z <- z + alpha s_k,
// alpha = mr.alpha[rhs], and the block partials of |t_{k+1}|^2 and
// <t_{k+1}, s_{k+1}> in place of those of |t|^2 and <t, in>.  Since
// t_{k+1} = op(s_{k+1}) in exact arithmetic, the next step needs no separate
// vector update and its memory traffic runs under the stencil's.
struct MrArgs {
  void* s = nullptr;  // storage of in / out (FP32 or BF16)
  float4* z = nullptr;
  const double2* alpha = nullptr;
};

// GD makes the plain FP32 stencil (one RHS per thread, one RHS tile per CTA)
// the GCR direction image W_k = D Z_k with its dots in the epilogue: for
// k = 0, |W|^2 and <W, r>; for k = 1..3, <W_j, W> for j < k (W_j at W0 + j
// wslot float4) -- per RHS and 128-site block into part[(rhs nblk + blk) 6 +
// v], summed by gd_finish_kernel
struct GdArgs {
  const float4* W0 = nullptr;
  size_t wslot = 0;
  int k = 0;
  const float4* r = nullptr;
  double* part = nullptr;
};

template <typename R, int NR, bool DAG, int RW, bool RED = false, bool MRF = false, typename SI = R,
          typename SO = R, bool GD = false>
__global__ void __launch_bounds__(128, dslash_min_ctas<R, NR, RW>()) dslash_kernel(const void* __restrict__ in, void* __restrict__ out,
                                                     const void* __restrict__ U, const void* __restrict__ C,
                                                     DslashArgs a, double* __restrict__ part = nullptr,
                                                     MrArgs mr = MrArgs(), GdArgs gd = GdArgs()) {
  static_assert(!GD || (!RED && NR == 1 && RW == 1 && sizeof(R) == 4), "GCR dots: plain FP32 tile 1,1 only");
  static_assert(!RED || (NR == 1 && RW == 1 && sizeof(R) == 4), "fused reduction: FP32 tile 1,1 only");
  static_assert(!MRF || RED, "the fused MR step reduces its dots");
  constexpr int SW = 128 / RW;  // sites per CTA
  const int64_t V = a.q.V;
  // RHS tile groups run fastest in launch order, so the CTAs that share a
  // block of sites are resident together and its links and clover come from L2
  const int ntile = (a.nrhs + NR - 1) / NR;
  int64_t site;
  int r0;
  bool valid = true;  // with RED every thread reaches the block reduction
  if constexpr (RW == 1) {
    site = (int64_t)(blockIdx.x / ntile) * blockDim.x + threadIdx.x;
    if (site >= V) {
      if constexpr (!RED && !GD) return;
      valid = false;
      site = V - 1;
    }
    r0 = (blockIdx.x % ntile) * NR;
  } else {
    const int ngrp = (ntile + RW - 1) / RW;
    const int tile = (int)(blockIdx.x % ngrp) * RW + (int)threadIdx.x / SW;
    site = (int64_t)(blockIdx.x / ngrp) * SW + threadIdx.x % SW;
    if (site >= V || tile >= ntile) return;
    r0 = tile * NR;
  }
  int x[4];
  site_coords(a.q, site, x);
  const R sF = DAG ? R(1) : R(-1);  // forward hop carries (1 + sF gamma)
  const R sB = -sF;

  Cx<R> acc[NR][12];
  // clover term
  {
    Cx<R> psi[12];
    R c[36];
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
      Clover<R>::load(C, V, chi, site, c);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r0 + r < a.nrhs) {
          SIO<SI>::load(in, V, r0 + r, site, psi);
          clover_apply6<R>(c, psi + 6 * chi, acc[r] + 6 * chi);
        }
      }
    }
  }
  // hopping terms
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    M3<R> Um;
    Cx<R> psi[12];
    {
      const int64_t nf = nbr_fwd(a.q, site, x, mu);
      const R f = R(-0.5) * ((mu == 0 && x[0] == a.q.L[0] - 1) ? R(a.bc) : R(1));
      Link<R>::load(U, V, mu, site, Um);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r0 + r < a.nrhs) {
          SIO<SI>::load(in, V, r0 + r, nf, psi);
          hop_add<R, true>(mu, sF, f, Um, psi, acc[r]);
        }
    }
    {
      const int64_t nb = nbr_bwd(a.q, site, x, mu);
      const R f = R(-0.5) * ((mu == 0 && x[0] == 0) ? R(a.bc) : R(1));
      Link<R>::load(U, V, mu, nb, Um);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r0 + r < a.nrhs) {
          SIO<SI>::load(in, V, r0 + r, nb, psi);
          hop_add<R, false>(mu, sB, f, Um, psi, acc[r]);
        }
    }
  }
  float nn = 0.f, dr = 0.f, di = 0.f;  // RED: this thread's |t|^2 and <t, s>
  constexpr bool BF = std::is_same<SO, SpinBf16>::value;
  if constexpr (MRF && BF) {
    // t, s in BF16 ([rhs][3][V] uint4 of four complex), z in FP32; the dots
    // are taken on the values as stored
    if (valid) {
      const double2 al = mr.alpha[r0];
      const Cx<float> alpha = cx((float)al.x, (float)al.y);
      const size_t offb = (size_t)r0 * 3 * V + site, offz = (size_t)r0 * 6 * V + site;
      const uint4* tp = reinterpret_cast<const uint4*>(in) + offb;
      uint4* op = reinterpret_cast<uint4*>(out) + offb;
      uint4* sp = reinterpret_cast<uint4*>(mr.s) + offb;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const uint4 tv = __ldg(tp + j * V), sv = sp[j * V];
        const float4 z0 = mr.z[offz + 2 * j * V], z1 = mr.z[offz + (2 * j + 1) * V];
        const uint32_t tw[4] = {tv.x, tv.y, tv.z, tv.w}, sw[4] = {sv.x, sv.y, sv.z, sv.w};
        const Cx<float> zk[4] = {cx(z0.x, z0.y), cx(z0.z, z0.w), cx(z1.x, z1.y), cx(z1.z, z1.w)};
        uint32_t tno[4], sno[4];
        Cx<float> zn[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const Cx<float> t = bf16_unpack(tw[h]), sk = bf16_unpack(sw[h]);
          tno[h] = bf16_pack(t - alpha * acc[0][4 * j + h]);
          sno[h] = bf16_pack(sk - alpha * t);
          zn[h] = zk[h] + alpha * sk;
          const Cx<float> tr = bf16_unpack(tno[h]), sr = bf16_unpack(sno[h]);
          nn += tr.re * tr.re + tr.im * tr.im;
          dr += tr.re * sr.re + tr.im * sr.im;
          di += tr.re * sr.im - tr.im * sr.re;
        }
        op[j * V] = make_uint4(tno[0], tno[1], tno[2], tno[3]);
        sp[j * V] = make_uint4(sno[0], sno[1], sno[2], sno[3]);
        mr.z[offz + 2 * j * V] = make_float4(zn[0].re, zn[0].im, zn[1].re, zn[1].im);
        mr.z[offz + (2 * j + 1) * V] = make_float4(zn[2].re, zn[2].im, zn[3].re, zn[3].im);
      }
    }
  } else if constexpr (MRF) {
    if (valid) {
      const double2 al = mr.alpha[r0];
      const Cx<float> alpha = cx((float)al.x, (float)al.y);
      const size_t off = (size_t)r0 * 6 * V + site;
      const float4* tp = reinterpret_cast<const float4*>(in) + off;
      float4* op = reinterpret_cast<float4*>(out) + off;
      float4* msp = reinterpret_cast<float4*>(mr.s);
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const float4 tv = __ldg(tp + j * V), sv = msp[off + j * V], zv = mr.z[off + j * V];
        const Cx<float> t[2] = {cx(tv.x, tv.y), cx(tv.z, tv.w)}, sk[2] = {cx(sv.x, sv.y), cx(sv.z, sv.w)},
                        zk[2] = {cx(zv.x, zv.y), cx(zv.z, zv.w)};
        Cx<float> tn[2], sn[2], zn[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tn[h] = t[h] - alpha * acc[0][2 * j + h];
          sn[h] = sk[h] - alpha * t[h];
          zn[h] = zk[h] + alpha * sk[h];
          nn += tn[h].re * tn[h].re + tn[h].im * tn[h].im;
          dr += tn[h].re * sn[h].re + tn[h].im * sn[h].im;
          di += tn[h].re * sn[h].im - tn[h].im * sn[h].re;
        }
        op[j * V] = make_float4(tn[0].re, tn[0].im, tn[1].re, tn[1].im);
        msp[off + j * V] = make_float4(sn[0].re, sn[0].im, sn[1].re, sn[1].im);
        mr.z[off + j * V] = make_float4(zn[0].re, zn[0].im, zn[1].re, zn[1].im);
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r0 + r < a.nrhs && valid) {
        if constexpr (std::is_same<SO, ResidF64>::value) {
          const double sc = a.scale[r0 + r];
          double2* p = reinterpret_cast<double2*>(out) + (size_t)(r0 + r) * 12 * V + site;
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            double2 v = p[k * V];
            v.x -= sc * dfl::to_double(acc[r][k].re);
            v.y -= sc * dfl::to_double(acc[r][k].im);
            p[k * V] = v;
          }
        } else {
          if (a.g5out) {
#pragma unroll
            for (int k = 6; k < 12; ++k) acc[r][k] = -acc[r][k];
          }
          if (a.bsub) {
            Cx<R> bv[12];
            IO<R>::load(a.bsub, V, r0 + r, site, bv);
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[r][k] = bv[k] - acc[r][k];
          }
          if constexpr (BF) {
            // the dots below see the values as stored
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[r][k] = bf16_unpack(bf16_pack(acc[r][k]));
          }
          SIO<SO>::store(out, V, r0 + r, site, acc[r]);
        }
      }
    if constexpr (RED) {
      if (valid) {
        Cx<R> sv[12];
        SIO<SI>::load(in, V, r0, site, sv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const Cx<R> t = acc[0][k];
          nn += t.re * t.re + t.im * t.im;
          dr += t.re * sv[k].re + t.im * sv[k].im;
          di += t.re * sv[k].im - t.im * sv[k].re;
        }
      }
    }
  }
  if constexpr (RED) {
    // FP32 within a warp (32 sites), FP64 from the warp partials on: the
    // FP64 pipe of GB300 is too narrow for a per-thread FP64 tree
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nn += __shfl_down_sync(0xffffffffu, nn, o);
      dr += __shfl_down_sync(0xffffffffu, dr, o);
      di += __shfl_down_sync(0xffffffffu, di, o);
    }
    __shared__ float wsum[4][3];
    const int w = threadIdx.x / 32;
    if (threadIdx.x % 32 == 0) {
      wsum[w][0] = nn;
      wsum[w][1] = dr;
      wsum[w][2] = di;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      const int64_t nblk = (V + 127) / 128;
      const int c = threadIdx.x;
      part[((size_t)r0 * nblk + blockIdx.x / ntile) * 3 + c] =
          (((double)wsum[0][c] + (double)wsum[1][c]) + (double)wsum[2][c]) + (double)wsum[3][c];
    }
  }
  if constexpr (GD) {
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
      const size_t off = (size_t)r0 * 6 * V + site;
      if (gd.k == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const float4 q = __ldg(gd.r + off + c * V);
          const Cx<float> w0 = acc[0][2 * c], w1 = acc[0][2 * c + 1];
          v[0] += w0.re * w0.re + w0.im * w0.im + w1.re * w1.re + w1.im * w1.im;
          v[1] += w0.re * q.x + w0.im * q.y + w1.re * q.z + w1.im * q.w;
          v[2] += w0.re * q.y - w0.im * q.x + w1.re * q.w - w1.im * q.z;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (j >= gd.k) break;
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const float4 q = __ldg(gd.W0 + j * gd.wslot + off + c * V);
            const Cx<float> w0 = acc[0][2 * c], w1 = acc[0][2 * c + 1];
            v[2 * j] += q.x * w0.re + q.y * w0.im + q.z * w1.re + q.w * w1.im;
            v[2 * j + 1] += q.x * w0.im - q.y * w0.re + q.z * w1.im - q.w * w1.re;
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int e = 0; e < 6; ++e) v[e] += __shfl_down_sync(0xffffffffu, v[e], o);
    __shared__ float gsum[4][6];
    const int w = threadIdx.x / 32;
    if (threadIdx.x % 32 == 0)
#pragma unroll
      for (int e = 0; e < 6; ++e) gsum[w][e] = v[e];
    __syncthreads();
    if (threadIdx.x < 6) {
      const int64_t nblk = (V + 127) / 128;
      const int e = threadIdx.x;
      gd.part[((size_t)r0 * nblk + blockIdx.x / ntile) * 6 + e] =
          (((double)gsum[0][e] + (double)gsum[1][e]) + (double)gsum[2][e]) + (double)gsum[3][e];
    }
  }
}

// ------------------------------------------------------------ staged-tile FP32 stencil (many RHS)
// A CTA covers DT = 32 consecutive sites and NRT right-hand sides: warp w
// computes RHS r0 + w on the 32 sites (lane = site), so every spinor load of a
// warp is one coalesced 512-byte row.  Everything that depends on the site
// but not on the RHS is staged once per CTA in shared memory: the eight
// links a site's hops use -- U_mu(x) for the forward hops and U_mu(x-mu)^dag
// for the backward hops, third row rebuilt, already multiplied by the hop
// factor -1/2 (times t_bc where the hop crosses the time boundary) -- and the
// two clover blocks.  The per-RHS work is then projection, one 3x3 product
// per half spinor and reconstruction.  Scaling a link by +-1/2 is exact and
// commutes with every rounding, and the terms are summed in the same order
// as dslash_kernel, so both kernels give the same bits.
constexpr int kDT = 32;  // sites per CTA of the staged kernel

struct StagedTile {
  float2 U[8][9][kDT];  // hop slot (0..3 forward, 4..7 backward), entry (row*3 + col), site
  float4 C[2][9][kDT];  // clover chirality block, packed float4, site
};

// hop slot MU (forward: U_MU(x)) or 4 + MU (backward: U_MU(x - MU)^dag) of site
// `site` (coordinates x) into the tile, times -1/2 (and t_bc across the time
// boundary)
template <int MU, bool FWD>
__device__ __forceinline__ void stage_link(StagedTile& st, int ls, const float4* __restrict__ U, const DslashArgs& a,
                                           int64_t site, const int x[4]) {
  const int64_t ls_site = FWD ? site : nbr_bwd(a.q, site, x, MU);
  const bool crossing = MU == 0 && (FWD ? x[0] == a.q.L[0] - 1 : x[0] == 0);
  const float f = -0.5f * (crossing ? (float)a.bc : 1.f);
  M3<float> m;
  Link<float>::load(U, a.q.V, MU, ls_site, m);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const Cx<float> e = FWD ? m.e[i][j] : conj(m.e[j][i]);
      st.U[FWD ? MU : 4 + MU][i * 3 + j][ls] = make_float2(f * e.re, f * e.im);
    }
}

// acc += (1 + s gamma_mu) W psi(nb) with the staged, pre-scaled link W of hop
// slot MU (forward) or 4 + MU (backward)
template <int MU, bool FWD>
__device__ __forceinline__ void staged_hop(const StagedTile& st, int ls, const float4* __restrict__ in, int64_t V,
                                           int r, int64_t nb, float sg, Cx<float> acc[12]) {
  constexpr int slot = FWD ? MU : 4 + MU;
  Cx<float> psi[12];
  IO<float>::load(in, V, r, nb, psi);
  M3<float> Um;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const float2 v = st.U[slot][e][ls];
    Um.e[e / 3][e % 3] = cx(v.x, v.y);
  }
  Cx<float> h0[3], h1[3], g0[3], g1[3];
  project<float>(MU, sg, psi, h0, h1);
  mat_vec<float>(Um, h0, g0);
  mat_vec<float>(Um, h1, g1);
  reconstruct_add<float>(MU, sg, g0, g1, acc);
}

// RED: per warp (one RHS, 32 sites) |t|^2 and <t, in> in FP32, written as FP64
// partials part[((rhs * ntiles) + tile) * 3 + {0, 1, 2}] (ntiles = ceil(V / 32))
// resident warps per SM the register allocation must allow: 24 (80
// registers a thread), 20 with the reduction epilogue (which holds the
// result and the input spinor at once)
template <int NRT, bool RED>
constexpr int staged_min_ctas() {
  return (RED ? 20 : 24) / NRT > 0 ? (RED ? 20 : 24) / NRT : 1;
}

template <int NRT, bool DAG, bool RED = false>
__global__ void __launch_bounds__(NRT * 32, staged_min_ctas<NRT, RED>()) dslash_staged_kernel(const float4* __restrict__ in, float4* __restrict__ out,
                                                                 const float4* __restrict__ U, const float4* __restrict__ C,
                                                                 DslashArgs a, double* __restrict__ part = nullptr) {
  __shared__ StagedTile st;
  const int64_t V = a.q.V;
  const int ngrp = (a.nrhs + NRT - 1) / NRT;
  const int64_t tile = blockIdx.x / ngrp;
  const int r0 = (int)(blockIdx.x % ngrp) * NRT;
  const int64_t base = tile * kDT;
  // ---- stage links (one (slot, site) per job) and clover blocks
  for (int job = threadIdx.x; job < 8 * kDT; job += blockDim.x) {
    const int l = job / kDT, ls = job % kDT;  // l is uniform across a warp
    const int64_t site = base + ls;
    if (site >= V) continue;
    int x[4];
    site_coords(a.q, site, x);
    switch (l) {
      case 0: stage_link<0, true>(st, ls, U, a, site, x); break;
      case 1: stage_link<1, true>(st, ls, U, a, site, x); break;
      case 2: stage_link<2, true>(st, ls, U, a, site, x); break;
      case 3: stage_link<3, true>(st, ls, U, a, site, x); break;
      case 4: stage_link<0, false>(st, ls, U, a, site, x); break;
      case 5: stage_link<1, false>(st, ls, U, a, site, x); break;
      case 6: stage_link<2, false>(st, ls, U, a, site, x); break;
      default: stage_link<3, false>(st, ls, U, a, site, x); break;
    }
  }
  for (int job = threadIdx.x; job < 18 * kDT; job += blockDim.x) {
    const int k = job / kDT, ls = job % kDT;
    const int64_t site = base + ls;
    if (site < V) st.C[k / 9][k % 9][ls] = __ldg(C + (size_t)k * V + site);
  }
  __syncthreads();
  const int w = threadIdx.x / 32, ls = threadIdx.x % 32;
  const int r = r0 + w;
  const int64_t site = base + ls;
  const bool valid = site < V;
  if (r >= a.nrhs) return;  // no barrier follows
  float nn = 0.f, dr = 0.f, di = 0.f;
  if (valid) {
    int x[4];
    site_coords(a.q, site, x);
    const float sF = DAG ? 1.f : -1.f;  // forward hop carries (1 + sF gamma)
    const float sB = -sF;
    Cx<float> acc[12];
    {
      Cx<float> psi[12];
      IO<float>::load(in, V, r, site, psi);
#pragma unroll
      for (int chi = 0; chi < 2; ++chi) {
        float c[36];
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          const float4 v = st.C[chi][j][ls];
          c[4 * j] = v.x;
          c[4 * j + 1] = v.y;
          c[4 * j + 2] = v.z;
          c[4 * j + 3] = v.w;
        }
        clover_apply6<float>(c, psi + 6 * chi, acc + 6 * chi);
      }
    }
    // hop order of dslash_kernel: mu = 0..3, forward then backward
    staged_hop<0, true>(st, ls, in, V, r, nbr_fwd(a.q, site, x, 0), sF, acc);
    staged_hop<0, false>(st, ls, in, V, r, nbr_bwd(a.q, site, x, 0), sB, acc);
    staged_hop<1, true>(st, ls, in, V, r, nbr_fwd(a.q, site, x, 1), sF, acc);
    staged_hop<1, false>(st, ls, in, V, r, nbr_bwd(a.q, site, x, 1), sB, acc);
    staged_hop<2, true>(st, ls, in, V, r, nbr_fwd(a.q, site, x, 2), sF, acc);
    staged_hop<2, false>(st, ls, in, V, r, nbr_bwd(a.q, site, x, 2), sB, acc);
    staged_hop<3, true>(st, ls, in, V, r, nbr_fwd(a.q, site, x, 3), sF, acc);
    staged_hop<3, false>(st, ls, in, V, r, nbr_bwd(a.q, site, x, 3), sB, acc);
    if (a.g5out) {
#pragma unroll
      for (int k = 6; k < 12; ++k) acc[k] = -acc[k];
    }
    IO<float>::store(out, V, r, site, acc);
    if constexpr (RED) {
      Cx<float> sv[12];
      IO<float>::load(in, V, r, site, sv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const Cx<float> t = acc[k];
        nn += t.re * t.re + t.im * t.im;
        dr += t.re * sv[k].re + t.im * sv[k].im;
        di += t.re * sv[k].im - t.im * sv[k].re;
      }
    }
  }
  if constexpr (RED) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nn += __shfl_down_sync(0xffffffffu, nn, o);
      dr += __shfl_down_sync(0xffffffffu, dr, o);
      di += __shfl_down_sync(0xffffffffu, di, o);
    }
    if (ls == 0) {
      const int64_t ntiles = (V + kDT - 1) / kDT;
      double* p = part + ((size_t)r * ntiles + tile) * 3;
      p[0] = (double)nn;
      p[1] = (double)dr;
      p[2] = (double)di;
    }
  }
}

// nrm[r] = sum_b part[r][b][0], dot[r] = sum_b (part[r][b][1], part[r][b][2]):
// one CTA per RHS, fixed order (strided partial sums, then a fixed tree)
__global__ void __launch_bounds__(256) dot_finish_kernel(const double* __restrict__ part, int64_t nblk,
                                                         double* __restrict__ nrm, double2* __restrict__ dot) {
  const int r = blockIdx.x;
  double a = 0, b = 0, c = 0;
  for (int64_t i = threadIdx.x; i < nblk; i += 256) {
    const double* p = part + ((size_t)r * nblk + i) * 3;
    a += p[0];
    b += p[1];
    c += p[2];
  }
  __shared__ double sh[3][256];
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + h];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + h];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    nrm[r] = sh[0][0];
    dot[r] = make_double2(sh[1][0], sh[2][0]);
  }
}

// the GD partials of RHS r (one CTA each) in a fixed order: k = 0 -> nw[r] =
// |W|^2, num[r] = <W, r>; k > 0 -> dots[j n + r] = <W_j, W> for j < k
__global__ void __launch_bounds__(256) gd_finish_kernel(const double* __restrict__ part, int64_t nblk, int k, int n,
                                                        double* __restrict__ nw, double2* __restrict__ num,
                                                        double2* __restrict__ dots) {
  const int r = blockIdx.x;
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < nblk; i += 256) {
    const double* p = part + ((size_t)r * nblk + i) * 6;
#pragma unroll
    for (int e = 0; e < 6; ++e) a[e] += p[e];
  }
  __shared__ double sh[6][256];
#pragma unroll
  for (int e = 0; e < 6; ++e) sh[e][threadIdx.x] = a[e];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int e = 0; e < 6; ++e) sh[e][threadIdx.x] += sh[e][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (k == 0) {
      nw[r] = sh[0][0];
      num[r] = make_double2(sh[1][0], sh[2][0]);
    } else {
      for (int j = 0; j < k; ++j) dots[(size_t)j * n + r] = make_double2(sh[2 * j][0], sh[2 * j + 1][0]);
    }
  }
}

// ------------------------------------------------------------ hop-slot pieces (FP64, setup)
struct SlotArgs {
  LatIdx q;
  double bc;
  int b[4];
  int slot;
};

__device__ __forceinline__ bool crosses(const int x[4], const int b[4], int d) {
  const int mu = d & 3;
  const int r = x[mu] % b[mu];
  return d < 4 ? (r == b[mu] - 1) : (r == 0);
}

__global__ void __launch_bounds__(128) dslash_slot_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                                          const double2* __restrict__ U, const double2* __restrict__ C,
                                                          SlotArgs a) {
  const int64_t V = a.q.V;
  const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (site >= V) return;
  int x[4];
  site_coords(a.q, site, x);
  Cx<double> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cx(0.0, 0.0);
  Cx<double> psi[12];
  if (a.slot == 8) {
    double c[36];
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
      Clover<double>::load(C, V, chi, site, c);
      IO<double>::load(in, V, rhs, site, psi);
      clover_apply6<double>(c, psi + 6 * chi, acc + 6 * chi);
    }
  }
  for (int d = 0; d < 8; ++d) {
    const bool cr = crosses(x, a.b, d);
    if (a.slot == 8 ? cr : (d != a.slot || !cr)) continue;
    const int mu = d & 3;
    M3<double> Um;
    if (d < 4) {
      const int64_t nf = nbr_fwd(a.q, site, x, mu);
      const double f = -0.5 * ((mu == 0 && x[0] == a.q.L[0] - 1) ? a.bc : 1.0);
      Link<double>::load(U, V, mu, site, Um);
      IO<double>::load(in, V, rhs, nf, psi);
      hop_add<double, true>(mu, -1.0, f, Um, psi, acc);
    } else {
      const int64_t nb = nbr_bwd(a.q, site, x, mu);
      const double f = -0.5 * ((mu == 0 && x[0] == 0) ? a.bc : 1.0);
      Link<double>::load(U, V, mu, nb, Um);
      IO<double>::load(in, V, rhs, nb, psi);
      hop_add<double, false>(mu, 1.0, f, Um, psi, acc);
    }
  }
  IO<double>::store(out, V, rhs, site, acc);
}

// ------------------------------------------------------------ layout conversion
template <typename R>
__global__ void pack_kernel(const double* __restrict__ canon, void* __restrict__ dst, int64_t V, int nrhs) {
  const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (site >= V || r >= nrhs) return;
  const double2* p = reinterpret_cast<const double2*>(canon) + ((size_t)r * V + site) * 12;
  Cx<R> s[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 v = p[k];
    s[k] = cx((R)v.x, (R)v.y);
  }
  IO<R>::store(dst, V, r, site, s);
}

template <typename R>
__global__ void unpack_kernel(const void* __restrict__ src, double* __restrict__ canon, int64_t V, int nrhs) {
  const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (site >= V || r >= nrhs) return;
  Cx<R> s[12];
  IO<R>::load(src, V, r, site, s);
  double2* p = reinterpret_cast<double2*>(canon) + ((size_t)r * V + site) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) p[k] = make_double2((double)s[k].re, (double)s[k].im);
}

// dst = scale_r * src (+ dst if accumulate); scale NULL means 1
template <typename RI, typename RO>
__global__ void convert_kernel(const void* __restrict__ src, void* __restrict__ dst, int64_t V, int nrhs,
                               const double* __restrict__ scale, int accumulate) {
  const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (site >= V || r >= nrhs) return;
  Cx<RI> s[12];
  IO<RI>::load(src, V, r, site, s);
  const double f = scale ? scale[r] : 1.0;
  Cx<RO> t[12];
  if (accumulate) IO<RO>::load(dst, V, r, site, t);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const RO re = (RO)(f * (double)s[k].re), im = (RO)(f * (double)s[k].im);
    t[k] = accumulate ? cx(t[k].re + re, t[k].im + im) : cx(re, im);
  }
  IO<RO>::store(dst, V, r, site, t);
}

// ------------------------------------------------------------ gauge packing
__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void gauge_pack_kernel(const double* __restrict__ links, int64_t site0, int64_t nsites, int64_t V,
                                  double2* __restrict__ U64, float4* __restrict__ U32, double* dev_max) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsites * 4) return;
  const int64_t site = site0 + i / 4;
  const int mu = (int)(i % 4);
  const double2* p = reinterpret_cast<const double2*>(links) + i * 9;
  M3<double> m;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 v = p[k];
    m.e[k / 3][k % 3] = cx(v.x, v.y);
    U64[((size_t)mu * 9 + k) * V + site] = v;
  }
  float4* q = U32 + (size_t)mu * 3 * V + site;
  q[0] = make_float4((float)m.e[0][0].re, (float)m.e[0][0].im, (float)m.e[0][1].re, (float)m.e[0][1].im);
  q[V] = make_float4((float)m.e[0][2].re, (float)m.e[0][2].im, (float)m.e[1][0].re, (float)m.e[1][0].im);
  q[2 * V] = make_float4((float)m.e[1][1].re, (float)m.e[1][1].im, (float)m.e[1][2].re, (float)m.e[1][2].im);
  // SU(3) check: |U U^dag - 1| and |row2 - conj(row0 x row1)|
  M3<double> uu = mul(m, dagger(m));
  double dev = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double re = uu.e[a][b].re - (a == b ? 1.0 : 0.0);
      dev = fmax(dev, fabs(re));
      dev = fmax(dev, fabs(uu.e[a][b].im));
    }
  Cx<double> r2[3];
  r2[0] = conj(m.e[0][1] * m.e[1][2] - m.e[0][2] * m.e[1][1]);
  r2[1] = conj(m.e[0][2] * m.e[1][0] - m.e[0][0] * m.e[1][2]);
  r2[2] = conj(m.e[0][0] * m.e[1][1] - m.e[0][1] * m.e[1][0]);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    dev = fmax(dev, fabs(r2[b].re - m.e[2][b].re));
    dev = fmax(dev, fabs(r2[b].im - m.e[2][b].im));
  }
  if (!(dev == dev)) dev = 1e300;  // NaN
  atomic_max_pos(dev_max, dev);
}

// ------------------------------------------------------------ clover construction
__device__ __forceinline__ M3<double> link64(const double2* U, int64_t V, int mu, int64_t site) {
  M3<double> m;
  Link<double>::load(U, V, mu, site, m);
  return m;
}

// Fhat_{mu nu}(x) = (Q - Q^dag) / 8, Q the four mu-nu leaves at x
__device__ M3<double> field_strength(const double2* U, const LatIdx& q, const int x[4], int64_t site, int mu,
                                     int nu) {
  const int64_t V = q.V;
  M3<double> Um = link64(U, V, mu, site), Un = link64(U, V, nu, site);
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  M3<double> Q = mul(mul(Um, link64(U, V, nu, shifted(q, x, mu, 1, nu, 0))),
                     mul(dagger(link64(U, V, mu, shifted(q, x, mu, 0, nu, 1))), dagger(Un)));
  // leaf 2: U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  const int64_t xm = shifted(q, x, mu, -1, nu, 0);
  M3<double> l2 = mul(mul(Un, dagger(link64(U, V, mu, shifted(q, x, mu, -1, nu, 1)))),
                      mul(dagger(link64(U, V, nu, xm)), link64(U, V, mu, xm)));
  Q = add(Q, l2);
  // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  const int64_t xmn = shifted(q, x, mu, -1, nu, -1);
  const int64_t xn = shifted(q, x, mu, 0, nu, -1);
  M3<double> l3 = mul(mul(dagger(link64(U, V, mu, xm)), dagger(link64(U, V, nu, xmn))),
                      mul(link64(U, V, mu, xmn), link64(U, V, nu, xn)));
  Q = add(Q, l3);
  // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
  M3<double> l4 = mul(mul(dagger(link64(U, V, nu, xn)), link64(U, V, mu, xn)),
                      mul(link64(U, V, nu, shifted(q, x, mu, 1, nu, -1)), dagger(Um)));
  Q = add(Q, l4);
  M3<double> F;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) F.e[a][b] = 0.125 * (Q.e[a][b] - conj(Q.e[b][a]));
  return F;
}

// Chirality blocks of A(x) = (4 + m0) + c_sw (i/4) sum sigma_{mu nu} Fhat_{mu nu}.
// With sigma_{0k} = diag(sigma_k, -sigma_k) and sigma_{jk} = -eps_{jkl}
// diag(sigma_l, sigma_l) the upper block is sum_l sigma_l (x) G_l with
// G_l = (i c_sw/2)(F_{0l} - B_l) and the lower one uses G'_l = -(i c_sw/2)(F_{0l} + B_l),
// where B_1 = F_23, B_2 = F_31, B_3 = F_12.
__global__ void clover_kernel(const double2* __restrict__ U, LatIdx q, double diag, double csw,
                              double2* __restrict__ C64, float4* __restrict__ C32) {
  const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (site >= q.V) return;
  int x[4];
  site_coords(q, site, x);
  M3<double> F01 = field_strength(U, q, x, site, 0, 1);
  M3<double> F02 = field_strength(U, q, x, site, 0, 2);
  M3<double> F03 = field_strength(U, q, x, site, 0, 3);
  M3<double> F12 = field_strength(U, q, x, site, 1, 2);
  M3<double> F13 = field_strength(U, q, x, site, 1, 3);
  M3<double> F23 = field_strength(U, q, x, site, 2, 3);
  const Cx<double> ih = cx(0.0, 0.5 * csw);  // i c_sw / 2
  for (int chi = 0; chi < 2; ++chi) {
    const double sg = chi == 0 ? 1.0 : -1.0;
    M3<double> G[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // upper: F_0l - B_l ; lower: -(F_0l + B_l)
        Cx<double> g1 = chi == 0 ? F01.e[a][b] - F23.e[a][b] : -(F01.e[a][b] + F23.e[a][b]);
        Cx<double> g2 = chi == 0 ? F02.e[a][b] + F13.e[a][b] : -(F02.e[a][b] - F13.e[a][b]);
        Cx<double> g3 = chi == 0 ? F03.e[a][b] - F12.e[a][b] : -(F03.e[a][b] + F12.e[a][b]);
        G[0].e[a][b] = ih * g1;
        G[1].e[a][b] = ih * g2;
        G[2].e[a][b] = ih * g3;
      }
    (void)sg;
    // 6x6 block on (s, a): [[G3, G1 - i G2], [G1 + i G2, -G3]] + diag
    Cx<double> Bk[6][6];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        Bk[a][b] = G[2].e[a][b];
        Bk[a][3 + b] = G[0].e[a][b] - mul_i(G[1].e[a][b]);
        Bk[3 + a][b] = G[0].e[a][b] + mul_i(G[1].e[a][b]);
        Bk[3 + a][3 + b] = -G[2].e[a][b];
      }
    double pk[36];
#pragma unroll
    for (int i = 0; i < 6; ++i) pk[i] = Bk[i][i].re + diag;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i + 1; j < 6; ++j) {
        const int k = 6 + 2 * offdiag_slot(i, j);
        pk[k] = Bk[i][j].re;
        pk[k + 1] = Bk[i][j].im;
      }
#pragma unroll
    for (int j = 0; j < 18; ++j) C64[((size_t)chi * 18 + j) * q.V + site] = make_double2(pk[2 * j], pk[2 * j + 1]);
#pragma unroll
    for (int j = 0; j < 9; ++j)
      C32[((size_t)chi * 9 + j) * q.V + site] =
          make_float4((float)pk[4 * j], (float)pk[4 * j + 1], (float)pk[4 * j + 2], (float)pk[4 * j + 3]);
  }
}

__global__ void tables_kernel(LatIdx q, int b0, int b1, int b2, int b3, int32_t* nbr, int32_t* blk) {
  const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (site >= q.V) return;
  int x[4];
  site_coords(q, site, x);
  for (int mu = 0; mu < 4; ++mu) {
    nbr[site * 8 + mu] = (int32_t)nbr_fwd(q, site, x, mu);
    nbr[site * 8 + 4 + mu] = (int32_t)nbr_bwd(q, site, x, mu);
  }
  if (blk) {
    const int b[4] = {b0, b1, b2, b3};
    int Lb[4];
    for (int m = 0; m < 4; ++m) Lb[m] = q.L[m] / b[m];
    const int y0 = x[0] / b[0], y1 = x[1] / b[1], y2 = x[2] / b[2], y3 = x[3] / b[3];
    blk[site] = ((y0 * Lb[1] + y1) * Lb[2] + y2) * Lb[3] + y3;
  }
}

// ============================================================ host side
static inline dim3 site_grid(int64_t V, int threads, int ny = 1) {
  return dim3((unsigned)((V + threads - 1) / threads), (unsigned)ny, 1);
}

mglma_status pack_spinor(mglma_ctx ctx, const double* canon, Spinor& dst, cudaStream_t s) {
  ProfScope ps(ctx, K_PACK, s);
  if (dst.prec == MGLMA_FP64)
    pack_kernel<double><<<site_grid(dst.V, 256, dst.nrhs), 256, 0, s>>>(canon, dst.p, dst.V, dst.nrhs);
  else
    pack_kernel<float><<<site_grid(dst.V, 256, dst.nrhs), 256, 0, s>>>(canon, dst.p, dst.V, dst.nrhs);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status unpack_spinor(mglma_ctx ctx, const Spinor& src, double* canon, cudaStream_t s) {
  ProfScope ps(ctx, K_PACK, s);
  if (src.prec == MGLMA_FP64)
    unpack_kernel<double><<<site_grid(src.V, 256, src.nrhs), 256, 0, s>>>(src.p, canon, src.V, src.nrhs);
  else
    unpack_kernel<float><<<site_grid(src.V, 256, src.nrhs), 256, 0, s>>>(src.p, canon, src.V, src.nrhs);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status convert_spinor(mglma_ctx ctx, const Spinor& src, Spinor& dst, cudaStream_t s, const double* scale,
                            bool accumulate) {
  if (src.V != dst.V || src.nrhs != dst.nrhs) return fail(MGLMA_ERR_INVALID, "convert_spinor: shape mismatch");
  ProfScope ps(ctx, K_PACK, s);
  dim3 g = site_grid(src.V, 256, src.nrhs);
  const int acc = accumulate ? 1 : 0;
  if (src.prec == MGLMA_FP64 && dst.prec == MGLMA_FP32)
    convert_kernel<double, float><<<g, 256, 0, s>>>(src.p, dst.p, src.V, src.nrhs, scale, acc);
  else if (src.prec == MGLMA_FP32 && dst.prec == MGLMA_FP64)
    convert_kernel<float, double><<<g, 256, 0, s>>>(src.p, dst.p, src.V, src.nrhs, scale, acc);
  else if (src.prec == MGLMA_FP64)
    convert_kernel<double, double><<<g, 256, 0, s>>>(src.p, dst.p, src.V, src.nrhs, scale, acc);
  else
    convert_kernel<float, float><<<g, 256, 0, s>>>(src.p, dst.p, src.V, src.nrhs, scale, acc);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// algorithmic traffic of one stencil launch: links + clover once, spinor in
// and out once per RHS (FP32: 4 x 48 B reconstruct-12 links + 288 B clover;
// FP64: 4 x 144 B links + 576 B clover); 1896 flops per site per RHS
static double dslash_bytes(int64_t V, int nrhs, bool fp64) {
  return (double)V * (fp64 ? 1152.0 + 384.0 * nrhs : 480.0 + 192.0 * nrhs);
}
static double dslash_flops(int64_t V, int nrhs) { return 1896.0 * (double)V * nrhs; }

template <typename R, int NR, int RW, typename SO = R>
static void launch_dslash(const Spinor& in, Spinor& out, const void* U, const void* C, const DslashArgs& a,
                          bool dagger, cudaStream_t s) {
  constexpr int SW = 128 / RW;
  const int ntile = (in.nrhs + NR - 1) / NR;
  const size_t ctas = (size_t)((in.V + SW - 1) / SW) * ((ntile + RW - 1) / RW);
  if (dagger)
    dslash_kernel<R, NR, true, RW, false, false, R, SO><<<(unsigned)ctas, 128, 0, s>>>(in.p, out.p, U, C, a);
  else
    dslash_kernel<R, NR, false, RW, false, false, R, SO><<<(unsigned)ctas, 128, 0, s>>>(in.p, out.p, U, C, a);
}

// FP32 tile shape (RHS per thread NR, RHS tiles per CTA RW) encoded as
// NR + 16 (RW - 1), or 64 + NRT for the staged-tile kernel; the autotuner
// (tune.cu) may replace the default below for an RHS count on a context.
// Measured on GB300 (64x32^3, 1-16 RHS): one RHS per thread and one RHS tile
// per CTA was fastest at every count (16 RHS: 2.93 ms, staged tiles of 4, 8,
// 16 RHS 3.45, 3.36, 3.49 ms -- the staged kernel issues as many
// instructions per site and RHS, its shared-memory loads replacing the
// rebuilt third link row; staging the operands pre-broadcast for paired FP32
// FMAs cut the instructions by a fifth but doubled the shared-memory bytes
// per site and RHS, and at 3.63 ms was slower still: this stencil is bound
// by the L1 / shared-memory bandwidth and latency of its operand loads).
int dslash32_default_tile(int) { return dslash32_tile_code(1, 1); }

template <int NRT, bool RED>
static void launch_staged(const Spinor& in, Spinor& out, const void* U, const void* C, const DslashArgs& a,
                          bool dagger, cudaStream_t s, double* part = nullptr) {
  const int64_t ntiles = (in.V + kDT - 1) / kDT;
  const unsigned ctas = (unsigned)(ntiles * ((in.nrhs + NRT - 1) / NRT));
  const float4* x = (const float4*)in.p;
  float4* y = (float4*)out.p;
  if (dagger)
    dslash_staged_kernel<NRT, true, RED><<<ctas, NRT * 32, 0, s>>>(x, y, (const float4*)U, (const float4*)C, a, part);
  else
    dslash_staged_kernel<NRT, false, RED><<<ctas, NRT * 32, 0, s>>>(x, y, (const float4*)U, (const float4*)C, a, part);
}

static void launch_dslash32(int code, const Spinor& in, Spinor& out, const void* U, const void* C,
                            const DslashArgs& a, bool dagger, cudaStream_t s) {
  if (dslash32_tile_staged(code)) {
    const int nrt = dslash32_tile_nrt(code);
    if (nrt == 4)
      launch_staged<4, false>(in, out, U, C, a, dagger, s);
    else if (nrt == 8)
      launch_staged<8, false>(in, out, U, C, a, dagger, s);
    else
      launch_staged<16, false>(in, out, U, C, a, dagger, s);
    return;
  }
  int nr = dslash32_tile_nr(code), rw = dslash32_tile_rw(code);
  if (in.nrhs < nr) nr = in.nrhs >= 2 ? 2 : 1;
  if (nr == 4)
    launch_dslash<float, 4, 1>(in, out, U, C, a, dagger, s);
  else if (nr == 2 && rw == 4)
    launch_dslash<float, 2, 4>(in, out, U, C, a, dagger, s);
  else if (nr == 2 && rw == 2)
    launch_dslash<float, 2, 2>(in, out, U, C, a, dagger, s);
  else if (nr == 2)
    launch_dslash<float, 2, 1>(in, out, U, C, a, dagger, s);
  else if (rw == 4)
    launch_dslash<float, 1, 4>(in, out, U, C, a, dagger, s);
  else if (rw == 2)
    launch_dslash<float, 1, 2>(in, out, U, C, a, dagger, s);
  else
    launch_dslash<float, 1, 1>(in, out, U, C, a, dagger, s);
}

mglma_status dslash(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& in, Spinor& out, bool dagger,
                    bool gamma5_out, cudaStream_t s) {
  if (in.prec != out.prec || in.V != G->g.V || out.V != G->g.V || in.nrhs != out.nrhs)
    return fail(MGLMA_ERR_INVALID, "dslash: field shape/precision mismatch");
  if (in.p == out.p) return fail(MGLMA_ERR_INVALID, "dslash: in and out must differ");
  DslashArgs a;
  a.q = make_latidx(G->g.L);
  a.bc = (double)G->g.t_bc;
  a.nrhs = in.nrhs;
  a.g5out = gamma5_out ? 1 : 0;
  const double flops = dslash_flops(in.V, in.nrhs);
  if (in.prec == MGLMA_FP64) {
    ProfScope ps(ctx, K_DSLASH64, s, dslash_bytes(in.V, in.nrhs, true), flops);
    launch_dslash<double, 1, 1>(in, out, G->U64, G->C64, a, dagger, s);
  } else {
    ProfScope ps(ctx, K_DSLASH32, s, dslash_bytes(in.V, in.nrhs, false), flops);
    launch_dslash32(tuned(ctx, TUNE_DSLASH32_NR, in.nrhs, G->g.V, dslash32_default_tile(in.nrhs)), in, out, G->U32, G->C32,
                    a, dagger, s);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// FP64 values split into double-float pairs, elementwise (two per float4)
__global__ void split_df_kernel(const double2* __restrict__ in, float4* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = in[i];
  const DF a(v.x), b(v.y);
  out[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
}

static mglma_status gauge_df_ready(mglma_gauge_s* G, cudaStream_t s) {
  if (G->Udf && G->Cdf) return MGLMA_OK;
  const size_t V = (size_t)G->g.V, nu = 36 * V, nc = 36 * V;
  if (!G->Udf) {
    MG_CUDA(cudaMalloc(&G->Udf, nu * sizeof(float4)));
    split_df_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, s>>>(G->U64, G->Udf, nu);
    MG_LAUNCH_CHECK();
  }
  if (!G->Cdf) {
    MG_CUDA(cudaMalloc(&G->Cdf, nc * sizeof(float4)));
    split_df_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(G->C64, G->Cdf, nc);
    MG_LAUNCH_CHECK();
  }
  return MGLMA_OK;
}

mglma_status dslash_resid_df(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& e, Spinor& r, const double* scale,
                             cudaStream_t s) {
  if (e.prec != MGLMA_FP32 || r.prec != MGLMA_FP64 || e.V != G->g.V || r.V != G->g.V || e.nrhs != r.nrhs || !scale)
    return fail(MGLMA_ERR_INVALID, "dslash_resid_df: FP32 e, FP64 r of the gauge field's volume and a scale needed");
  if (e.nrhs == 0) return MGLMA_OK;
  MG_CHECK(gauge_df_ready(const_cast<mglma_gauge_s*>(G), s));
  DslashArgs a;
  a.q = make_latidx(G->g.L);
  a.bc = (double)G->g.t_bc;
  a.nrhs = e.nrhs;
  a.g5out = 0;
  a.scale = scale;
  // links and clover as FP64-sized double-float words, e in FP32, r read and written in FP64
  ProfScope ps(ctx, K_DSLASH64, s, (double)e.V * (1152.0 + 480.0 * e.nrhs), dslash_flops(e.V, e.nrhs));
  const size_t ctas = (size_t)((e.V + 127) / 128) * e.nrhs;
  dslash_kernel<DF, 1, false, 1, false, false, SpinF32Df, ResidF64>
      <<<(unsigned)ctas, 128, 0, s>>>(e.p, r.p, G->Udf, G->Cdf, a);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status dslash_resid(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& in, const Spinor& b, Spinor& out,
                          cudaStream_t s) {
  if (in.prec != MGLMA_FP32 || (out.prec != MGLMA_FP32 && out.prec != MGLMA_BF16) || b.prec != MGLMA_FP32 ||
      in.V != G->g.V || out.V != G->g.V || b.V != G->g.V || in.nrhs != out.nrhs || b.nrhs != out.nrhs)
    return fail(MGLMA_ERR_INVALID, "dslash_resid: FP32 in and b (FP32 or BF16 out) of the gauge field's volume needed");
  if (in.p == out.p || b.p == out.p) return fail(MGLMA_ERR_INVALID, "dslash_resid: out must differ from in and b");
  if (in.nrhs == 0) return MGLMA_OK;
  DslashArgs a;
  a.q = make_latidx(G->g.L);
  a.bc = (double)G->g.t_bc;
  a.nrhs = in.nrhs;
  a.g5out = 0;
  a.bsub = b.p;
  const bool bf = out.prec == MGLMA_BF16;
  ProfScope ps(ctx, K_DSLASH32, s,
               dslash_bytes(in.V, in.nrhs, false) + (bf ? 96.0 - 48.0 : 96.0) * (double)in.V * in.nrhs,
               dslash_flops(in.V, in.nrhs) + 24.0 * (double)in.V * in.nrhs);
  if (bf) {
    launch_dslash<float, 1, 1, SpinBf16>(in, out, G->U32, G->C32, a, false, s);
  } else {
    // the staged-tile kernel has no room for the epilogue's extra operand
    int code = tuned(ctx, TUNE_DSLASH32_NR, in.nrhs, G->g.V, dslash32_default_tile(in.nrhs));
    if (dslash32_tile_staged(code)) code = dslash32_tile_code(1, 1);
    launch_dslash32(code, in, out, G->U32, G->C32, a, false, s);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// room for the finer of the two partial-sum grids (32-site tiles)
size_t dslash_dot_part_doubles(int64_t V, int nrhs) { return (size_t)3 * nrhs * (size_t)((V + kDT - 1) / kDT); }

mglma_status dslash_dot(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& in, Spinor& out, double* part,
                        double* nrm, double2* dot, cudaStream_t s) {
  const bool bf = in.prec == MGLMA_BF16;
  if ((in.prec != MGLMA_FP32 && !bf) || out.prec != in.prec || in.V != G->g.V || out.V != G->g.V ||
      in.nrhs != out.nrhs)
    return fail(MGLMA_ERR_INVALID, "dslash_dot: FP32 or BF16 fields of the gauge field's volume needed");
  if (in.p == out.p) return fail(MGLMA_ERR_INVALID, "dslash_dot: in and out must differ");
  if (in.nrhs == 0) return MGLMA_OK;
  DslashArgs a;
  a.q = make_latidx(G->g.L);
  a.bc = (double)G->g.t_bc;
  a.nrhs = in.nrhs;
  a.g5out = 0;
  // the kernel of the tuned tile shape: the staged-tile kernel (per-warp
  // partials of 32-site tiles, RHS tiles of 4, whose epilogue fits 96
  // registers) or one site per thread (partials of 128-site blocks)
  const bool staged =
      !bf && dslash32_tile_staged(tuned(ctx, TUNE_DSLASH32_NR, in.nrhs, G->g.V, dslash32_default_tile(in.nrhs)));
  const int64_t nblk = staged ? (in.V + kDT - 1) / kDT : (in.V + 127) / 128;
  {
    ProfScope ps(ctx, K_DSLASH32, s, dslash_bytes(in.V, in.nrhs, false) - (bf ? 96.0 * (double)in.V * in.nrhs : 0.0),
                 dslash_flops(in.V, in.nrhs));
    if (staged)
      launch_staged<4, true>(in, out, G->U32, G->C32, a, false, s, part);
    else if (bf)
      dslash_kernel<float, 1, false, 1, true, false, SpinBf16, SpinBf16>
          <<<(unsigned)(nblk * in.nrhs), 128, 0, s>>>(in.p, out.p, G->U32, G->C32, a, part);
    else
      dslash_kernel<float, 1, false, 1, true><<<(unsigned)(nblk * in.nrhs), 128, 0, s>>>(in.p, out.p, G->U32,
                                                                                         G->C32, a, part);
  }
  MG_LAUNCH_CHECK();
  {
    ProfScope ps(ctx, K_REDUCE, s, (double)dslash_dot_part_doubles(in.V, in.nrhs) * 8.0);
    dot_finish_kernel<<<in.nrhs, 256, 0, s>>>(part, nblk, nrm, dot);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

size_t dslash_gcr_part_doubles(int64_t V, int nrhs) { return (size_t)6 * nrhs * (size_t)((V + 127) / 128); }

mglma_status dslash_gcr(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& in, Spinor& out, int k,
                        const void* W0, size_t wslot_reals, const void* r, double* part, double* nw, double2* num,
                        double2* dots, cudaStream_t s) {
  if (in.prec != MGLMA_FP32 || out.prec != MGLMA_FP32 || in.V != G->g.V || out.V != G->g.V || in.nrhs != out.nrhs)
    return fail(MGLMA_ERR_INVALID, "dslash_gcr: FP32 fields of the gauge field's volume needed");
  if (k < 0 || k > 3) return fail(MGLMA_ERR_INVALID, "dslash_gcr: 0 to 3 earlier directions");
  if (in.p == out.p) return fail(MGLMA_ERR_INVALID, "dslash_gcr: in and out must differ");
  if (in.nrhs == 0) return MGLMA_OK;
  DslashArgs a;
  a.q = make_latidx(G->g.L);
  a.bc = (double)G->g.t_bc;
  a.nrhs = in.nrhs;
  a.g5out = 0;
  GdArgs gd;
  gd.W0 = (const float4*)W0;
  gd.wslot = wslot_reals / 4;
  gd.k = k;
  gd.r = (const float4*)r;
  gd.part = part;
  const int64_t nblk = (in.V + 127) / 128;
  {
    // the stencil's bytes plus r (k = 0) or the k earlier images read once
    ProfScope ps(ctx, K_DSLASH32, s, dslash_bytes(in.V, in.nrhs, false) + 96.0 * (k ? k : 1) * (double)in.V * in.nrhs,
                 dslash_flops(in.V, in.nrhs) + 48.0 * (k ? k : 1) * (double)in.V * in.nrhs);
    dslash_kernel<float, 1, false, 1, false, false, float, float, true>
        <<<(unsigned)(nblk * in.nrhs), 128, 0, s>>>(in.p, out.p, G->U32, G->C32, a, nullptr, MrArgs(), gd);
  }
  MG_LAUNCH_CHECK();
  {
    ProfScope ps(ctx, K_REDUCE, s, (double)dslash_gcr_part_doubles(in.V, in.nrhs) * 8.0);
    gd_finish_kernel<<<in.nrhs, 256, 0, s>>>(part, nblk, k, in.nrhs, nw, num, dots);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

bool dslash_mr_fused(mglma_ctx ctx, const mglma_gauge_s* G, int nrhs) {
  return !dslash32_tile_staged(tuned(ctx, TUNE_DSLASH32_NR, nrhs, G->g.V, dslash32_default_tile(nrhs)));
}

mglma_status dslash_mr_step(mglma_ctx ctx, const mglma_gauge_s* G, const Spinor& t, Spinor& tn, Spinor& sk,
                            Spinor& z, const double2* alpha, double* part, double* nrm, double2* dot,
                            cudaStream_t s) {
  const Spinor* f[4] = {&t, &tn, &sk, &z};
  const bool bf = t.prec == MGLMA_BF16;
  for (const Spinor* v : f)
    if (v->V != G->g.V || v->nrhs != t.nrhs ||
        v->prec != (v == &z ? MGLMA_FP32 : (bf ? MGLMA_BF16 : MGLMA_FP32)))
      return fail(MGLMA_ERR_INVALID, "dslash_mr_step: t, tn, sk FP32 or BF16 and z FP32, of the gauge field's volume");
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (f[i]->p == f[j]->p) return fail(MGLMA_ERR_INVALID, "dslash_mr_step: the four fields must differ");
  if (t.nrhs == 0) return MGLMA_OK;
  DslashArgs a;
  a.q = make_latidx(G->g.L);
  a.bc = (double)G->g.t_bc;
  a.nrhs = t.nrhs;
  a.g5out = 0;
  MrArgs mr;
  mr.s = sk.p;
  mr.z = (float4*)z.p;
  mr.alpha = alpha;
  const int64_t nblk = (t.V + 127) / 128;
  {
    // the stencil's bytes (t in, tn out) plus s read and written and z read
    // and written once
    const double sb = bf ? 48.0 : 96.0;
    ProfScope ps(ctx, K_DSLASH32, s, 480.0 * (double)t.V + (4.0 * sb + 2.0 * 96.0) * (double)t.V * t.nrhs,
                 dslash_flops(t.V, t.nrhs) + 432.0 * (double)t.V * t.nrhs);
    if (bf)
      dslash_kernel<float, 1, false, 1, true, true, SpinBf16, SpinBf16>
          <<<(unsigned)(nblk * t.nrhs), 128, 0, s>>>(t.p, tn.p, G->U32, G->C32, a, part, mr);
    else
      dslash_kernel<float, 1, false, 1, true, true><<<(unsigned)(nblk * t.nrhs), 128, 0, s>>>(t.p, tn.p, G->U32,
                                                                                              G->C32, a, part, mr);
  }
  MG_LAUNCH_CHECK();
  {
    ProfScope ps(ctx, K_REDUCE, s, (double)dslash_dot_part_doubles(t.V, t.nrhs) * 8.0);
    dot_finish_kernel<<<t.nrhs, 256, 0, s>>>(part, nblk, nrm, dot);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// z += alpha s for FP32 z and BF16 s (the last MR step); one thread per site
// and group of four components
__global__ void mr_zupdate_kernel(float4* __restrict__ z, const uint4* __restrict__ sb,
                                  const double2* __restrict__ alpha, int64_t V) {
  const int r = blockIdx.y;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)3 * V) return;
  const int j = (int)(e / V);
  const int64_t site = (int64_t)(e % V);
  const double2 al = alpha[r];
  const Cx<float> a = cx((float)al.x, (float)al.y);
  const uint4 sv = sb[((size_t)r * 3 + j) * V + site];
  float4* z0 = z + ((size_t)r * 6 + 2 * j) * V + site;
  float4* z1 = z0 + V;
  const float4 u0 = *z0, u1 = *z1;
  const Cx<float> s0 = bf16_unpack(sv.x), s1 = bf16_unpack(sv.y), s2 = bf16_unpack(sv.z), s3 = bf16_unpack(sv.w);
  const Cx<float> w0 = cx(u0.x, u0.y) + a * s0, w1 = cx(u0.z, u0.w) + a * s1;
  const Cx<float> w2 = cx(u1.x, u1.y) + a * s2, w3 = cx(u1.z, u1.w) + a * s3;
  *z0 = make_float4(w0.re, w0.im, w1.re, w1.im);
  *z1 = make_float4(w2.re, w2.im, w3.re, w3.im);
}

mglma_status mr_zupdate(mglma_ctx ctx, const double2* alpha, const Spinor& sk, Spinor& z, cudaStream_t s) {
  if (sk.prec != MGLMA_BF16 || z.prec != MGLMA_FP32 || sk.V != z.V || sk.nrhs != z.nrhs)
    return fail(MGLMA_ERR_INVALID, "mr_zupdate: BF16 s and FP32 z of one shape needed");
  if (z.nrhs == 0) return MGLMA_OK;
  ProfScope ps(ctx, K_BLAS, s, (48.0 + 2.0 * 96.0) * (double)z.V * z.nrhs);
  const dim3 g((unsigned)((3 * z.V + 255) / 256), (unsigned)z.nrhs, 1);
  mr_zupdate_kernel<<<g, 256, 0, s>>>((float4*)z.p, (const uint4*)sk.p, alpha, z.V);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status dslash_slot64_batch(mglma_ctx ctx, const mglma_gauge_s* G, const int block[4], const Spinor& in,
                                 Spinor& out, int slot, cudaStream_t s) {
  if (in.prec != MGLMA_FP64 || out.prec != MGLMA_FP64 || in.nrhs != out.nrhs)
    return fail(MGLMA_ERR_INVALID, "dslash_slot64: needs FP64 fields of equal size");
  SlotArgs a;
  a.q = make_latidx(G->g.L);
  a.bc = (double)G->g.t_bc;
  for (int m = 0; m < 4; ++m) a.b[m] = block[m];
  a.slot = slot;
  ProfScope ps(ctx, K_SETUP, s);
  dslash_slot_kernel<<<site_grid(G->g.V, 128, in.nrhs), 128, 0, s>>>((const double2*)in.p, (double2*)out.p, G->U64,
                                                                      G->C64, a);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status gauge_pack_slab(mglma_ctx ctx, mglma_gauge_s* G, const double* links_dev, int64_t site0,
                             int64_t nsites, double* dev_max, cudaStream_t s) {
  ProfScope ps(ctx, K_SETUP, s);
  const int64_t n = nsites * 4;
  gauge_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(links_dev, site0, nsites, G->g.V, G->U64, G->U32,
                                                                 dev_max);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status clover_build(mglma_ctx ctx, mglma_gauge_s* G, cudaStream_t s) {
  ProfScope ps(ctx, K_SETUP, s);
  LatIdx q = make_latidx(G->g.L);
  clover_kernel<<<site_grid(G->g.V, 64), 64, 0, s>>>(G->U64, q, 4.0 + G->m0, G->csw, G->C64, G->C32);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

mglma_status debug_tables(mglma_ctx ctx, const mglma_gauge_s* G, const int* block, int32_t* nbr_dev,
                          int32_t* blk_dev, cudaStream_t s) {
  LatIdx q = make_latidx(G->g.L);
  int b[4] = {1, 1, 1, 1};
  if (block)
    for (int m = 0; m < 4; ++m) b[m] = block[m];
  tables_kernel<<<site_grid(G->g.V, 256), 256, 0, s>>>(q, b[0], b[1], b[2], b[3], nbr_dev, blk_dev);
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}

// ============================================================ allocation-free Dirac apply
// Some callers cannot allocate device memory at the moment they need the
// operator: code running while a CUDA graph is being captured, code called
// from inside an allocator hook, or processes whose HBM is already fully
// reserved by another caching allocator.  mglma_dirac_apply_noalloc serves
// them: its two internal-layout work fields live in this file-scope device
// array instead of in pool allocations.  Every GPU that loads the library
// holds the array until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};  // device address of the array, per device

// Once per device, with that device current: the address of the array as the
// device sees it (the array's name in host code is only a host-side stand-in).
static mglma_status noalloc_scratch(int device, void** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (device < 0 || device >= 64) return fail(MGLMA_ERR_INVALID, "dirac_apply_noalloc: device index out of range");
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(MGLMA_ERR_CUDA, std::string("dirac_apply_noalloc: cudaGetSymbolAddress failed: ") +
                                      cudaGetErrorString(e));
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return MGLMA_OK;
}

}  // namespace mglma

extern "C" mglma_status mglma_dirac_apply_noalloc(mglma_ctx ctx, mglma_gauge G, mglma_op op, int nrhs,
                                                  const double* in, double* out, mglma_prec compute,
                                                  void* cuda_stream) {
  using namespace mglma;
  if (!ctx || !G || !in || !out) return fail(MGLMA_ERR_INVALID, "dirac_apply_noalloc: NULL argument");
  if (!G->ready) return fail(MGLMA_ERR_INVALID, "dirac_apply_noalloc: gauge field incomplete");
  MG_CHECK(check_gauge_device(ctx, G, "dirac_apply_noalloc"));
  if (nrhs < 0) return fail(MGLMA_ERR_INVALID, "dirac_apply_noalloc: nrhs < 0");
  if (op < MGLMA_OP_D || op > MGLMA_OP_DDAGD) return fail(MGLMA_ERR_INVALID, "dirac_apply_noalloc: bad op");
  if (compute != MGLMA_FP64 && compute != MGLMA_FP32)
    return fail(MGLMA_ERR_INVALID, "dirac_apply_noalloc: compute must be FP64 or FP32");
  if (nrhs == 0) return MGLMA_OK;
  const size_t field = (size_t)nrhs * G->g.V * 24 * (compute == MGLMA_FP64 ? 8 : 4);
  if (2 * field > kNoAllocScratchBytes)
    return fail(MGLMA_ERR_INVALID, "dirac_apply_noalloc: nrhs x V too large: two internal fields of " +
                                       std::to_string(field) + " bytes exceed the " +
                                       std::to_string(kNoAllocScratchBytes) + "-byte scratch array");
  MG_CUDA(cudaSetDevice(ctx->device));
  if (!is_device_pointer(in) || !is_device_pointer(out))
    return fail(MGLMA_ERR_INVALID, "dirac_apply_noalloc: in and out must be device memory");
  void* scratch = nullptr;
  MG_CHECK(noalloc_scratch(ctx->device, &scratch));
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
  // Both work fields are fully overwritten (pack writes a, the stencil writes
  // b), so nothing in the array needs clearing between calls.
  Spinor a, b;
  a.prec = b.prec = compute;
  a.nrhs = b.nrhs = nrhs;
  a.V = b.V = G->g.V;
  a.p = scratch;
  b.p = static_cast<unsigned char*>(scratch) + ((field + 255) / 256) * 256;
  DslashArgs da;
  da.q = make_latidx(G->g.L);
  da.bc = (double)G->g.t_bc;
  da.nrhs = nrhs;
  da.g5out = op == MGLMA_OP_Q ? 1 : 0;
  const dim3 pg = site_grid(G->g.V, 256, nrhs);
  const bool dp = compute == MGLMA_FP64;
  const int kd = dp ? K_DSLASH64 : K_DSLASH32;
  {
    ProfScope ps(ctx, K_PACK, s);
    if (dp)
      pack_kernel<double><<<pg, 256, 0, s>>>(in, a.p, a.V, nrhs);
    else
      pack_kernel<float><<<pg, 256, 0, s>>>(in, a.p, a.V, nrhs);
  }
  const bool dag1 = op == MGLMA_OP_DDAG;
  {
    ProfScope ps(ctx, kd, s, dslash_bytes(G->g.V, nrhs, dp), dslash_flops(G->g.V, nrhs));
    if (dp)
      launch_dslash<double, 1, 1>(a, b, G->U64, G->C64, da, dag1, s);
    else
      launch_dslash<float, 1, 1>(a, b, G->U32, G->C32, da, dag1, s);
  }
  const Spinor* res = &b;
  if (op == MGLMA_OP_DDAGD) {  // second pass D^dag back into a
    ProfScope ps(ctx, kd, s, dslash_bytes(G->g.V, nrhs, dp), dslash_flops(G->g.V, nrhs));
    if (dp)
      launch_dslash<double, 1, 1>(b, a, G->U64, G->C64, da, true, s);
    else
      launch_dslash<float, 1, 1>(b, a, G->U32, G->C32, da, true, s);
    res = &a;
  }
  {
    ProfScope ps(ctx, K_PACK, s);
    if (dp)
      unpack_kernel<double><<<pg, 256, 0, s>>>(res->p, out, res->V, nrhs);
    else
      unpack_kernel<float><<<pg, 256, 0, s>>>(res->p, out, res->V, nrhs);
  }
  MG_LAUNCH_CHECK();
  return MGLMA_OK;
}
