// Leapfrog stencil step for 3D grids, TMA-pipelined persistent version.
//
// Same arithmetic as stencil_plain.cuh (Eq. 7 with the damped coefficients,
// Eq. 9 Laplacian in constant-annihilating form; with VD the Eq. 10 term
// - grad(ln rho) . grad(p), ln rho's gradient read from three precomputed
// fields), but the data movement is built for B300:
//   - persistent grid (SMs x resident CTAs); CTA b owns the contiguous range
//     [total*b/G, total*(b+1)/G) of (xy-tile, z-plane) work items, so every
//     CTA gets the same number of planes to within one;
//   - the work of one plane arrives as a "bundle" of tensor copies
//     (cp.async.bulk.tensor.3d) into one slot of an NB-deep shared-memory
//     ring, completing on the slot's mbarrier: the centre plane p[n](c) with
//     an R-row / XH-column halo, p[n-1](c), kappa(c), the interior of the
//     front plane p[n](c+R) that feeds the register z-queue, and with VD the
//     three ln(rho) gradient components at plane c.  A tile column starts
//     with W = ceil(2R / WP) warm-up bundles, each one box of WP interior
//     planes of p[n] that only fill the z-queue (fewer trips through the
//     ring than one plane per bundle);
//   - each thread keeps its columns' 2R+1 planes of p[n] in a register queue
//     (shifted once per plane); the in-plane neighbours come from the centre
//     box, each y row of a thread's window read once per plane;
//   - no thread ever waits for a slot to drain: every warp bumps the slot's
//     shared-memory counter when it is done with it, and the warp that
//     brings the count to the number of warps issues the bundle NB ahead
//     into that slot;
//   - each lane computes two adjacent columns with 64-bit shared loads and
//     packed FP32x2 arithmetic; with equal spacings the six neighbours at
//     each offset are summed before the one multiply (else three per-axis
//     chains);
//     rows with no damping skip the damping lookup;
//   - the kernel writes node values only (ragged tiles masked); Dirichlet
//     face nodes and the ghost images of the face conditions are written by
//     face_conditions_kernel right after it.
// Every mbarrier wait is bounded (wall clock); on timeout a warp raises the
// device error flag and the CTA's abort flag (no more bundles are issued),
// waits (bounded) for the copies issued into the slots it has not consumed
// and exits; the CTA's other warps follow when their own waits run out.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "layout.h"
#include "stencil_plain.cuh"
#include "tma.cuh"

namespace sw {

// One grid of a batch of 3D grids advanced by one launch (MULTI): its
// tensor maps for the step's level parity, its stencil arguments and the
// first work item of its tiles in the batch's list.  Kept in global memory
// (the tensor maps are written there from the host before any launch).
struct __align__(128) TmaGridDesc {
  CUtensorMap c, f, w, o, k;  // centre box with halo, front plane, warm-up box, p[n-1], kappa
  StencilArgs a;
  int unit0;    // first work item
  int tiles_x;  // tiles along x
  int nz;       // planes per tile column
};

struct TmaWork {
  int tiles_x;  // tiles along x
  int nz;       // planes per tile column
  int total;    // tiles * nz work items (fits 32 bits: checked on the host)
  int starve;   // failure-path test: issue no copies, so every wait runs into its bound
  const TmaGridDesc* grids = nullptr;  // MULTI: the batch's grids, unit0 ascending
  int n_grids = 0;
};

// Where work item u lies: its grid (MULTI), tile and plane.
struct TmaLoc {
  int gi, t, zb, nzg, tiles_x;
};

template <bool MULTI>
__device__ __forceinline__ TmaLoc tma_locate(const TmaGridDesc* grids, int n_grids, int nz, int tiles_x, int u) {
  TmaLoc l;
  if constexpr (MULTI) {
    int gi = 0;
    for (int i = 1; i < n_grids && grids[i].unit0 <= u; ++i) gi = i;
    const int ul = u - grids[gi].unit0;
    l.gi = gi;
    l.nzg = grids[gi].nz;
    l.tiles_x = grids[gi].tiles_x;
    l.t = ul / l.nzg;
    l.zb = ul - l.t * l.nzg;
  } else {
    l.gi = 0;
    l.nzg = nz;
    l.tiles_x = tiles_x;
    l.t = u / nz;
    l.zb = u % nz;
  }
  return l;
}

// Interior planes of p[n] in one warm-up box (its tensor map's box depth).
constexpr int kTmaWarmPlanes = 4;

// Segment of a CTA's work range: the part of one tile column inside it.
// Its bundles j = 0 .. len+W-1: for j < W the warm-up box of front planes
// zb - R + j*WP .. zb - R + j*WP + WP - 1 (those below zb + R enter the
// queue), for j >= W compute plane zb + j - W with front plane zb + j - W + R.
__device__ __forceinline__ int segment_len(int u, int u1, int nz) { return min(u1 - u, nz - u % nz); }

template <int R, int TY, int PPT, int NB, bool VD>
struct TmaConfig {
  static constexpr int TX = 64;               // 32 lanes x 2 adjacent columns
  static constexpr int XH = (R + 3) / 4 * 4;  // x halo rounded to 16 bytes (TMA x alignment)
  static constexpr int PW = TX + 2 * XH;
  static constexpr int PH = TY + 2 * R;
  static constexpr int NCW = TY / PPT;  // warps, PPT rows each
  static constexpr int NT = 32 * NCW;
  static constexpr int QL = 2 * R + 1;   // register z-queue length
  static constexpr int H = (R + 1) / 2;  // float2 loads each side for the x neighbours
  static constexpr int YW = PPT + 2 * R;  // rows of a thread's y window
  static constexpr uint32_t C_BYTES = uint32_t(PH * PW) * 4u;  // centre box with halo
  static constexpr uint32_t I_BYTES = uint32_t(TY * TX) * 4u;  // one interior box
  // Box strides are padded to 128 bytes: a tensor copy's shared-memory
  // destination must be 128-byte aligned.
  static constexpr int C_FLOATS = int((C_BYTES + 127u) / 128u * 128u) / 4;
  static constexpr int I_FLOATS = int((I_BYTES + 127u) / 128u * 128u) / 4;
  static constexpr int NI = VD ? 6 : 3;  // interior boxes: front, p[n-1], kappa (+ d/dz, d/dy, d/dx ln rho)
  static constexpr int SLOT_FLOATS = C_FLOATS + NI * I_FLOATS;
  static constexpr int WP = kTmaWarmPlanes;      // planes per warm-up bundle
  static constexpr int W = (2 * R + WP - 1) / WP;  // warm-up bundles per segment
  static_assert(WP * I_FLOATS <= SLOT_FLOATS, "a warm-up box fills one slot at most");
  static constexpr size_t SMEM = size_t(NB) * SLOT_FLOATS * 4 + size_t(NB) * 8 + size_t(NB) * 4 + 16;
  static_assert((C_FLOATS * 4) % 128 == 0 && (I_FLOATS * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");
  // tiles past the last row read zero-filled rows (tensor copies clip at the
  // field's extent) and store nothing there
  static_assert(kTileXMax % TX == 0 && TY <= kTileYMax && TY % PPT == 0, "tile shape");
  static_assert(PW <= 256 && PH <= 256 && XH % 2 == 0, "TMA box extent / float2 alignment");
};

// Ring bookkeeping kept in shared memory after the slots.
struct RingShared {
  int abort;   // set by a CTA member whose wait gave up
  int issued;  // bundles issued so far (max over issuers)
};

// Warp w owns tile rows w*PPT..w*PPT+PPT-1; lane l owns columns 2l and 2l+1,
// handled as a float2 with packed FP32x2 arithmetic.
// ISO: all three spacings are equal, so one coefficient per j serves every
// axis (fewer registers; same arithmetic).
// IMG (constant density only): the imaging pass of the misfit gradient on
// the same pipeline.  The bundle's p[n-1] box carries psi and its kappa box
// the accumulator gk, and the store writes gk + psi (L p) to a.pout (= gk):
// with p the forward state, this accumulates kappa dJ/dkappa.
template <int R, int TY, int PPT, int NB, int MINB, bool ISO, bool VD, bool IMG = false, bool MULTI = false>
__global__ void __launch_bounds__(TmaConfig<R, TY, PPT, NB, VD>::NT, MINB)
    stencil_tma_kernel(const __grid_constant__ CUtensorMap map_c, const __grid_constant__ CUtensorMap map_f,
                       const __grid_constant__ CUtensorMap map_w, const __grid_constant__ CUtensorMap map_o, const __grid_constant__ CUtensorMap map_k,
                       const __grid_constant__ CUtensorMap map_gz, const __grid_constant__ CUtensorMap map_gy,
                       const __grid_constant__ CUtensorMap map_gx, const __grid_constant__ StencilArgs a,
                       const TmaWork wk,
                       int* err_flag, unsigned long long limit_ns) {
  static_assert(!(IMG && VD), "the imaging pass is constant density");
  static_assert(!(MULTI && (IMG || VD)), "batches of 3D grids are constant density");
  using C = TmaConfig<R, TY, PPT, NB, VD>;
  constexpr int TX = C::TX, QL = C::QL, H = C::H, PW = C::PW, NCW = C::NCW, W = C::W, WP = C::WP;
  extern __shared__ __align__(128) unsigned char smem[];
  float* slots = reinterpret_cast<float*>(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(slots + NB * C::SLOT_FLOATS);
  int* cnt = reinterpret_cast<int*>(bars + NB);
  RingShared* ring = reinterpret_cast<RingShared*>(cnt + NB);
  volatile int* abort_flag = &ring->abort;

  // launched after the previous step's kernels: wait for them before any
  // global access (the next kernel may start as soon as every CTA is here)
  griddep_launch_dependents();
  griddep_wait();
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int u0 = int((long long)wk.total * blockIdx.x / gridDim.x);
  const int u1 = int((long long)wk.total * (blockIdx.x + 1) / gridDim.x);
  if (u0 >= u1) return;
  if (smem_addr(smem) & 127u) {  // tensor copies need 128-byte aligned destinations
    if (threadIdx.x == 0) atomicOr(err_flag, 2);
    return;
  }
  const uint32_t full0 = smem_addr(bars);
  auto locate = [&](int u) { return tma_locate<MULTI>(wk.grids, wk.n_grids, wk.nz, wk.tiles_x, u); };
  // planes of the segment that starts at u (the rest of its tile column within the range)
  auto seg_len = [&](int u) {
    const TmaLoc l = locate(u);
    return min(u1 - u, l.nzg - l.zb);
  };

  // Bundle `jn` counted from the start of the segment (u, len) into `slot`
  // (one lane); false when it lies past the end of the range.  `mark` > 0
  // is recorded as the number of bundles issued before the copies start.
  auto issue = [&](int slot, int u, int len, int jn, int mark) -> bool {
    while (jn >= len + W) {
      jn -= len + W;
      u += len;
      if (u >= u1) return false;
      len = seg_len(u);
    }
    if (mark > 0) atomicMax(&ring->issued, mark);
    const TmaLoc l = locate(u);
    const int x0 = (l.t % l.tiles_x) * TX, y0 = (l.t / l.tiles_x) * TY;
    const CUtensorMap *mc = &map_c, *mf = &map_f, *mw = &map_w, *mo = &map_o, *mk = &map_k;
    if constexpr (MULTI) {
      const TmaGridDesc* D = wk.grids + l.gi;
      mc = &D->c;
      mf = &D->f;
      mw = &D->w;
      mo = &D->o;
      mk = &D->k;
    }
    float* sb = slots + slot * C::SLOT_FLOATS;
    const uint32_t bar = full0 + 8u * slot;
    if (jn < W) {  // WP front planes from padded z zb + jn * WP, at the slot's start
      mbar_arrive_expect_tx(bar, uint32_t(WP) * C::I_BYTES);
      tma_load_3d(smem_addr(sb), mw, x0 + kXOff, y0 + R, l.zb + jn * WP, bar);
    } else {
      const int zf = l.zb + jn - W + 2 * R;  // padded z of the front plane
      mbar_arrive_expect_tx(bar, C::C_BYTES + uint32_t(C::NI) * C::I_BYTES);
      tma_load_3d(smem_addr(sb), mc, x0 + kXOff - C::XH, y0, zf - R, bar);
      tma_load_3d(smem_addr(sb + C::C_FLOATS), mf, x0 + kXOff, y0 + R, zf, bar);
      // p[n-1] and kappa are read once: they leave L2 first, so that p[n]
      // planes stay there for the halo rows neighbouring tiles read later
      const uint64_t once = make_policy_evict_first();
      tma_load_3d_hint(smem_addr(sb + C::C_FLOATS + C::I_FLOATS), mo, x0 + kXOff, y0 + R, zf - R, bar, once);
      tma_load_3d_hint(smem_addr(sb + C::C_FLOATS + 2 * C::I_FLOATS), mk, x0 + kXOff, y0 + R, zf - R, bar, once);
      if constexpr (VD) {
        tma_load_3d_hint(smem_addr(sb + C::C_FLOATS + 3 * C::I_FLOATS), &map_gz, x0 + kXOff, y0 + R, zf - R, bar, once);
        tma_load_3d_hint(smem_addr(sb + C::C_FLOATS + 4 * C::I_FLOATS), &map_gy, x0 + kXOff, y0 + R, zf - R, bar, once);
        tma_load_3d_hint(smem_addr(sb + C::C_FLOATS + 5 * C::I_FLOATS), &map_gx, x0 + kXOff, y0 + R, zf - R, bar, once);
      }
    }
    return true;
  };

  if (threadIdx.x == 0) {
    ring->abort = 0;
    for (int i = 0; i < NB; ++i) {
      mbar_init(full0 + 8u * i, 1);
      cnt[i] = 0;
    }
    fence_barrier_init();
    if constexpr (!MULTI) {
      prefetch_tensormap(&map_c);
      prefetch_tensormap(&map_f);
      prefetch_tensormap(&map_w);
      prefetch_tensormap(&map_o);
      prefetch_tensormap(&map_k);
    }
    if constexpr (VD) {
      prefetch_tensormap(&map_gz);
      prefetch_tensormap(&map_gy);
      prefetch_tensormap(&map_gx);
    }
    const int len0 = seg_len(u0);
    int n = 0;
    while (!wk.starve && n < NB && issue(n, u0, len0, n, 0)) ++n;
    ring->issued = n;
  }
  __syncthreads();

  // on a failed wait or an abort: raise the flags and wait (bounded) for
  // the copies issued for bundles this warp has not consumed yet
  auto give_up = [&](int k) {
    *abort_flag = 1;
    atomicOr(err_flag, 1);
    if (lane == 0) {
      const int iss = atomicAdd(&ring->issued, 0);
      for (int b = k; b < iss; ++b) mbar_wait_bounded(full0 + 8u * (b % NB), uint32_t((b / NB) & 1), limit_ns);
    }
  };

  float2 cz2[R + 1], cy2[R + 1], cx2[R + 1];  // coefficient pairs (ISO: one set)
  float2 gz2[VD ? R + 1 : 1], gy2[VD ? R + 1 : 1], gx2[VD ? R + 1 : 1];  // first-derivative weights
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    cx2[j] = make_float2(a.cx[j], a.cx[j]);
    cy2[j] = ISO ? cx2[j] : make_float2(a.cy[j], a.cy[j]);
    cz2[j] = ISO ? cx2[j] : make_float2(a.cz[j], a.cz[j]);
    if constexpr (VD) {
      gx2[j] = make_float2(a.gx[j], a.gx[j]);
      gy2[j] = ISO ? gx2[j] : make_float2(a.gy[j], a.gy[j]);
      gz2[j] = ISO ? gx2[j] : make_float2(a.gz[j], a.gz[j]);
    }
  }
  const int r0 = warp * PPT;  // first tile row of this warp
  float2 qz[PPT][QL];  // z-queue, shifted once per plane

  int k = 0;  // bundles consumed by this warp
  int s = 0;  // slot of bundle k
  uint32_t ph = 0;
  for (int u = u0; u < u1;) {
    const TmaLoc loc = locate(u);
    const int len = min(u1 - u, loc.nzg - loc.zb);
    const int t = loc.t;
    const int zb = loc.zb;
    const int x0 = (t % loc.tiles_x) * TX, y0 = (t / loc.tiles_x) * TY;
    // the segment's grid: the kernel's own, or (MULTI) one of the batch's
    const StencilArgs& A = MULTI ? wk.grids[loc.gi].a : a;
    if constexpr (MULTI) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        cx2[j] = make_float2(A.cx[j], A.cx[j]);
        cy2[j] = ISO ? cx2[j] : make_float2(A.cy[j], A.cy[j]);
        cz2[j] = ISO ? cx2[j] : make_float2(A.cz[j], A.cz[j]);
      }
    }
    const int x = x0 + 2 * lane;
    // per-segment invariants (warp-uniform unless noted)
    const bool va_ok = x < A.nx, vb_ok = x + 1 < A.nx;  // per lane
    // some lane lies past the last column or some row past the last row
    const bool ragged = __any_sync(0xffffffffu, !vb_ok) || y0 + r0 + PPT > A.ny;
    // nodes past the last column or row (ragged tiles; never stored) take
    // distance 0, so every damping-table index stays inside the table
    const int dxa = va_ok ? layer_distance(x, A.nx, A.nbl[4], A.nbl[5]) : 0;
    const int dxb = vb_ok ? layer_distance(x + 1, A.nx, A.nbl[4], A.nbl[5]) : 0;
    int d2xy_a[PPT], d2xy_b[PPT];
    bool xy_free = true;  // no node of the warp's rows is in the absorbing layer in x, y
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int y = y0 + r0 + i;
      const int dyl = y < A.ny ? layer_distance(y, A.ny, A.nbl[2], A.nbl[3]) : 0;
      d2xy_a[i] = dyl * dyl + dxa * dxa;
      d2xy_b[i] = dyl * dyl + dxb * dxb;
      xy_free = xy_free && (d2xy_a[i] | d2xy_b[i]) == 0;
    }
    xy_free = __all_sync(0xffffffffu, xy_free);
    // damping coefficients of the warp's nodes on planes outside the z layer
    // (the same for every such plane of the segment): ca0 = 1/(1+e), e0 = e
    float2 ca0[PPT], e0[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      ca0[i] = make_float2(1.f, 1.f);
      e0[i] = make_float2(0.f, 0.f);
      if (!xy_free) {
        const float2 da = __ldg(&A.damp[d2xy_a[i]]), db = __ldg(&A.damp[d2xy_b[i]]);
        ca0[i] = make_float2(da.x, db.x);
        e0[i] = make_float2(da.y, db.y);
      }
    }
    const int rowoff0 = (y0 + r0) * int(A.sy) + x;  // in-plane offsets fit 32 bits (checked on the host)
    const int nb = len + W;
    bool zl_held = false;  // ca0/e0 hold a z-layer plane's coefficients
#pragma unroll 1
    for (int j = 0; j < nb; ++j) {
      // damping coefficients of this plane's nodes: per segment outside the
      // z layer, else fetched here, before the wait, so that their latency
      // hides behind it
      const int z = zb + j - W;
      const int dzl = layer_distance(z, A.nz, A.nbl[0], A.nbl[1]);
      const int dz2 = dzl * dzl;
      const bool zlayer = !IMG && j >= W && dz2 != 0;
      const bool damped = !IMG && (zlayer || (j >= W && !xy_free));
      // one set of coefficient registers: a plane of the z layer overwrites
      // ca0/e0 with its nodes' (1/(1+e), e), the first plane after the layer
      // puts the x/y values back (a separate set held for the z layer's
      // planes cost 3% of the launch)
      if (zlayer) {
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          const float2 da = __ldg(&A.damp[dz2 + d2xy_a[i]]), db = __ldg(&A.damp[dz2 + d2xy_b[i]]);
          ca0[i] = make_float2(da.x, db.x);
          e0[i] = make_float2(da.y, db.y);
        }
        zl_held = true;
      } else if (zl_held && j >= W) {
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          ca0[i] = make_float2(1.f, 1.f);
          e0[i] = make_float2(0.f, 0.f);
          if (!xy_free) {
            const float2 da = __ldg(&A.damp[d2xy_a[i]]), db = __ldg(&A.damp[d2xy_b[i]]);
            ca0[i] = make_float2(da.x, db.x);
            e0[i] = make_float2(da.y, db.y);
          }
        }
        zl_held = false;
      }
      // the decision to go on is taken by the whole warp, so its lanes never
      // split.  The abort flag is not read here (a shared-memory load on the
      // path of every plane, measured 2% of the kernel's time): once a warp
      // gives up, no bundle is issued any more and the other warps' next
      // bounded waits run out too.
      const bool bad = !mbar_wait_bounded(full0 + 8u * s, ph, limit_ns);
      if (__any_sync(0xffffffffu, bad)) {
        give_up(k);
        return;
      }
      const float* S = slots + s * C::SLOT_FLOATS;
      if (j < W) {  // warm-up: the planes of the box that lie below zb + R enter the queue
        const float2* F = reinterpret_cast<const float2*>(S) + r0 * (TX / 2) + lane;
#pragma unroll
        for (int pp = 0; pp < WP; ++pp) {
          if (j * WP + pp < 2 * R) {
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
#pragma unroll
              for (int kk = 0; kk < QL - 1; ++kk) qz[i][kk] = qz[i][kk + 1];
              qz[i][QL - 1] = F[pp * (C::I_FLOATS / 2) + i * (TX / 2)];
            }
          }
        }
      } else {
        const float2* F = reinterpret_cast<const float2*>(S + C::C_FLOATS) + r0 * (TX / 2) + lane;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
#pragma unroll
          for (int kk = 0; kk < QL - 1; ++kk) qz[i][kk] = qz[i][kk + 1];
          qz[i][QL - 1] = F[i * (TX / 2)];
        }
      }
      if (j >= W) {
        const float* cc = S + (r0 + R) * PW + C::XH + 2 * lane;  // centre of output row 0
        const float2* O = reinterpret_cast<const float2*>(S + C::C_FLOATS + C::I_FLOATS) + r0 * (TX / 2) + lane;
        const float2* K = O + C::I_FLOATS / 2;
        // y window: rows -R .. PPT-1+R around the warp's first row
        float2 yw[C::YW];
#pragma unroll
        for (int q = 0; q < C::YW; ++q) yw[q] = *reinterpret_cast<const float2*>(cc + (q - R) * PW);
        float2 kl[PPT];  // kappa L, then p[n+1]
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          const float* c = cc + i * PW;
          float2 w[2 * H + 1];  // columns x-2H .. x+1+2H of this row, as pairs
#pragma unroll
          for (int mm = -H; mm <= H; ++mm)
            w[mm + H] = (mm == 0) ? yw[i + R] : *reinterpret_cast<const float2*>(c + 2 * mm);
          const float2 pc = qz[i][R];
          const float2 p2 = f2_add(pc, pc);
          if constexpr (ISO) {
            // one coefficient per offset on all three axes: the six
            // neighbours at offset jj are summed first, less 6p (the form
            // still annihilates constants); two chains (even / odd jj)
            const float2 p6 = f2_add(p2, f2_add(p2, p2));
            float2 le = make_float2(0.f, 0.f), lo = le;
#pragma unroll
            for (int jj = 1; jj <= R; ++jj) {
              float2 xs;  // (x+jj) + (x-jj) for both columns
              if (jj % 2 == 0) {
                xs = f2_add(w[H + jj / 2], w[H - jj / 2]);
              } else {  // odd offsets straddle the pairs: two scalar adds into one pair
                xs = make_float2(w[H + (jj - 1) / 2].y + w[H - (jj + 1) / 2].y,
                                 w[H + (jj + 1) / 2].x + w[H - (jj - 1) / 2].x);
              }
              const float2 zy = f2_add(f2_add(qz[i][R + jj], qz[i][R - jj]), f2_add(yw[i + R + jj], yw[i + R - jj]));
              const float2 t = f2_sub(f2_add(zy, xs), p6);
              if (jj % 2) lo = f2_fma(cx2[jj], t, lo);
              else le = f2_fma(cx2[jj], t, le);
            }
            kl[i] = f2_add(le, lo);
          } else {
            // three independent accumulation chains (one per axis) for latency
            float2 lz = make_float2(0.f, 0.f), lx = lz, ly = lz;
#pragma unroll
            for (int jj = 1; jj <= R; ++jj) {
              lz = f2_fma(cz2[jj], f2_sub(f2_add(qz[i][R + jj], qz[i][R - jj]), p2), lz);
              float2 xs;  // (x+jj) + (x-jj) for both columns
              if (jj % 2 == 0) {
                xs = f2_add(w[H + jj / 2], w[H - jj / 2]);
              } else {  // odd offsets straddle the pairs: two scalar adds into one pair
                xs = make_float2(w[H + (jj - 1) / 2].y + w[H - (jj + 1) / 2].y,
                                 w[H + (jj + 1) / 2].x + w[H - (jj - 1) / 2].x);
              }
              lx = f2_fma(cx2[jj], f2_sub(xs, p2), lx);
              ly = f2_fma(cy2[jj], f2_sub(f2_add(yw[i + R + jj], yw[i + R - jj]), p2), ly);
            }
            kl[i] = f2_add(f2_add(lz, lx), ly);
          }
          if constexpr (VD) {
            // - grad(ln rho) . grad(p): first derivatives of p from the same
            // neighbours (Eq. 10), ln rho's from the gradient boxes
            float2 dz = make_float2(0.f, 0.f), dx = dz, dy = dz;
#pragma unroll
            for (int jj = 1; jj <= R; ++jj) {
              dz = f2_fma(gz2[jj], f2_sub(qz[i][R + jj], qz[i][R - jj]), dz);
              float2 xd;  // (x+jj) - (x-jj) for both columns
              if (jj % 2 == 0) {
                xd = f2_sub(w[H + jj / 2], w[H - jj / 2]);
              } else {
                xd = make_float2(w[H + (jj - 1) / 2].y - w[H - (jj + 1) / 2].y,
                                 w[H + (jj + 1) / 2].x - w[H - (jj - 1) / 2].x);
              }
              dx = f2_fma(gx2[jj], xd, dx);
              dy = f2_fma(gy2[jj], f2_sub(yw[i + R + jj], yw[i + R - jj]), dy);
            }
            const float2* G = reinterpret_cast<const float2*>(S + C::C_FLOATS + 3 * C::I_FLOATS) + r0 * (TX / 2) + lane;
            const float2 lgz = G[i * (TX / 2)], lgy = G[C::I_FLOATS / 2 + i * (TX / 2)],
                         lgx = G[C::I_FLOATS + i * (TX / 2)];
            const float2 adv = f2_fma(lgy, dy, f2_fma(lgx, dx, f2_mul(lgz, dz)));
            kl[i] = f2_sub(kl[i], adv);
          }
        }
        if constexpr (IMG) {
          // gk + psi (L p), psi from the p[n-1] box, gk from the kappa box
#pragma unroll
          for (int i = 0; i < PPT; ++i) kl[i] = f2_fma(O[i * (TX / 2)], kl[i], K[i * (TX / 2)]);
        } else if (!damped) {
          // outside the absorbing layer: a = 1, e = 0
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            const float2 pc = qz[i][R], po = O[i * (TX / 2)], kp = K[i * (TX / 2)];
            kl[i] = f2_add(pc, f2_fma(kp, kl[i], f2_sub(pc, po)));
          }
        } else {
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            const float2 pc = qz[i][R], po = O[i * (TX / 2)], kp = K[i * (TX / 2)];
            // p[n+1] = a (p + (kappa L + ((p - p[n-1]) + e p[n-1])))
            kl[i] = f2_mul(ca0[i], f2_add(pc, f2_fma(kp, kl[i], f2_fma(e0[i], po, f2_sub(pc, po)))));
          }
        }
        float* plane = A.pout + int64_t(z) * A.sz + rowoff0;
        if (!ragged) {
#pragma unroll
          for (int i = 0; i < PPT; ++i) __stcs(reinterpret_cast<float2*>(plane + i * int(A.sy)), kl[i]);  // streaming
        } else {
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            if (y0 + r0 + i >= A.ny) break;
            float* dst = plane + i * int(A.sy);
            if (vb_ok) {
              *reinterpret_cast<float2*>(dst) = kl[i];
            } else if (va_ok) {
              dst[0] = kl[i].x;
            }
          }
        }
      }
      // release the slot; the last warp to do so refills it with bundle k+NB
      __syncwarp();
      if (lane == 0) {
        asm volatile("fence.acq_rel.cta;" ::: "memory");  // this warp's reads of the slot come first
        if (atomicAdd(&cnt[s], 1) == NCW - 1) {
          cnt[s] = 0;
          asm volatile("fence.acq_rel.cta;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          if (!*abort_flag) issue(s, u, len, j + NB, k + NB + 1);
        }
      }
      ++k;
      if (++s == NB) {
        s = 0;
        ph ^= 1u;
      }
    }
    u += len;
  }
}

}  // namespace sw
