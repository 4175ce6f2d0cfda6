// Leapfrog stencil step for 3D grids, TMA-pipelined persistent version.
//
// Same arithmetic as stencil_plain.cuh (Eq. 7 with the damped coefficients,
// Eq. 9 Laplacian in constant-annihilating form, fused face mirroring), but
// the data movement is built for B300:
//   - persistent grid (SMs x resident CTAs); CTA b owns the contiguous range
//     [total*b/G, total*(b+1)/G) of (xy-tile, z-plane) work items, so every
//     CTA gets the same number of planes to within one;
//   - p[n] tile planes with an R-row / XH-column halo are fetched by TMA
//     (cp.async.bulk.tensor.3d) into a ring of NP = R+1+D shared-memory slots,
//     D+1 planes ahead of use; p[n-1] and kappa tiles come the same way into a
//     second ring of NQ slots; each slot completes on its own mbarrier;
//   - each thread keeps its column's 2R+1 planes of p[n] in a register queue,
//     so a plane is read from shared memory once for z and once per in-plane
//     neighbour;
//   - one block barrier per plane releases the slots of the plane that left
//     the window, after which one thread issues the next loads.
// Every mbarrier wait is bounded (wall clock); on timeout the CTA raises the
// device error flag, drains its own outstanding copies with bounded waits and
// exits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "layout.h"
#include "stencil_plain.cuh"
#include "tma.cuh"

namespace sw {

struct TmaWork {
  int tiles_x;       // tiles along x
  int nz;            // planes per tile column
  long long total;   // tiles * nz work items
};

// Walks the (tile, plane) segments of one CTA's work range.  `extra` is the
// number of planes a segment needs beyond its own (2R warm-up planes for the
// p[n] stream, 0 for the p[n-1] / kappa stream).
struct SegCursor {
  long long u, u1;
  int nz, len, j, extra;
  __device__ void init(long long a, long long b, int nz_, int extra_) {
    u = a;
    u1 = b;
    nz = nz_;
    extra = extra_;
    j = 0;
    len = (u < u1) ? seg_len() : 0;
  }
  __device__ int seg_len() const {
    const int zb = int(u % nz);
    const long long rem = u1 - u;
    return int(rem < (long long)(nz - zb) ? rem : (long long)(nz - zb));
  }
  __device__ bool valid() const { return u < u1; }
  __device__ int tile() const { return int(u / nz); }
  __device__ int zb() const { return int(u % nz); }
  __device__ void advance() {
    if (++j >= len + extra) {
      u += len;
      j = 0;
      len = (u < u1) ? seg_len() : 0;
    }
  }
};

template <int R, int TX, int TY, int PPT, int D, int NQ>
struct TmaConfig {
  static constexpr int XH = (R + 3) / 4 * 4;  // x halo rounded to 16 bytes (TMA x alignment)
  static constexpr int PW = TX + 2 * XH;
  static constexpr int PH = TY + 2 * R;
  static constexpr int NP = R + 1 + D;
  static constexpr int NT = TX * (TY / PPT);
  static constexpr uint32_t P_BYTES = uint32_t(PH * PW) * 4u;  // bytes one p[n] box delivers
  static constexpr uint32_t Q_BYTES = uint32_t(TY * TX) * 4u;   // bytes one p[n-1] / kappa box delivers
  // Slot strides are padded to 128 bytes: a tensor copy's shared-memory
  // destination must be 128-byte aligned.
  static constexpr int P_FLOATS = int((P_BYTES + 127u) / 128u * 128u) / 4;
  static constexpr int Q_FLOATS = int((Q_BYTES + 127u) / 128u * 128u) / 4;
  static constexpr size_t SMEM = size_t(NP) * P_FLOATS * 4 + 2 * size_t(NQ) * Q_FLOATS * 4 + size_t(NP + NQ) * 8 + 16;
  static_assert((P_FLOATS * 4) % 128 == 0 && (Q_FLOATS * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");
  static_assert(TX % 32 == 0 && kTileXMax % TX == 0 && kTileYMax % TY == 0 && TY % PPT == 0, "tile shape");
  static_assert(PW <= 256 && PH <= 256, "TMA box extent");
};

template <int R, int TX, int TY, int PPT, int D, int NQ>
__global__ void __launch_bounds__(TX*(TY / PPT)) stencil_tma_kernel(const __grid_constant__ CUtensorMap map_p,
                                                                     const __grid_constant__ CUtensorMap map_q,
                                                                     const __grid_constant__ CUtensorMap map_k,
                                                                     const StencilArgs a, const TmaWork wk,
                                                                     int* err_flag, unsigned long long limit_ns) {
  using C = TmaConfig<R, TX, TY, PPT, D, NQ>;
  extern __shared__ __align__(128) unsigned char smem[];
  float* sp = reinterpret_cast<float*>(smem);
  float* sq = sp + C::NP * C::P_FLOATS;
  float* sk = sq + NQ * C::Q_FLOATS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sk + NQ * C::Q_FLOATS);
  int* s_abort = reinterpret_cast<int*>(bars + C::NP + NQ);

  const int tid = threadIdx.x;
  const int tx = tid % TX;
  const int ty = tid / TX;
  const long long u0 = wk.total * blockIdx.x / gridDim.x;
  const long long u1 = wk.total * (blockIdx.x + 1) / gridDim.x;
  if (u0 >= u1) return;
  if (smem_addr(smem) & 127u) {  // tensor copies need 128-byte aligned destinations
    if (tid == 0) atomicOr(err_flag, 2);
    return;
  }

  const uint32_t bar_p0 = smem_addr(bars);
  const uint32_t bar_q0 = smem_addr(bars + C::NP);
  SegCursor cp, cq;  // producer cursors (meaningful in thread 0 only)
  long long p_issued = 0, q_issued = 0;

  auto issue_p = [&]() {
    const int t = cp.tile();
    const int x0 = (t % wk.tiles_x) * TX, y0 = (t / wk.tiles_x) * TY;
    const int z = cp.zb() - R + cp.j;
    const int slot = int(p_issued % C::NP);
    const uint32_t bar = bar_p0 + 8u * slot;
    mbar_arrive_expect_tx(bar, C::P_BYTES);
    tma_load_3d(smem_addr(sp + slot * C::P_FLOATS), &map_p, x0 + kXOff - C::XH, y0, z + R, bar);
    ++p_issued;
    cp.advance();
  };
  auto issue_q = [&]() {
    const int t = cq.tile();
    const int x0 = (t % wk.tiles_x) * TX, y0 = (t / wk.tiles_x) * TY;
    const int z = cq.zb() + cq.j;
    const int slot = int(q_issued % NQ);
    const uint32_t bar = bar_q0 + 8u * slot;
    mbar_arrive_expect_tx(bar, 2u * C::Q_BYTES);
    tma_load_3d(smem_addr(sq + slot * C::Q_FLOATS), &map_q, x0 + kXOff, y0 + R, z + R, bar);
    tma_load_3d(smem_addr(sk + slot * C::Q_FLOATS), &map_k, x0 + kXOff, y0 + R, z + R, bar);
    ++q_issued;
    cq.advance();
  };

  if (tid == 0) {
    *s_abort = 0;
    for (int i = 0; i < C::NP; ++i) mbar_init(bar_p0 + 8u * i, 1);
    for (int i = 0; i < NQ; ++i) mbar_init(bar_q0 + 8u * i, 1);
    fence_barrier_init();
    prefetch_tensormap(&map_p);
    prefetch_tensormap(&map_q);
    prefetch_tensormap(&map_k);
    cp.init(u0, u1, wk.nz, 2 * R);
    cq.init(u0, u1, wk.nz, 0);
    for (int i = 0; i <= D && cp.valid(); ++i) issue_p();
    for (int i = 0; i < NQ && cq.valid(); ++i) issue_q();
  }
  __syncthreads();

  volatile int* abort_flag = s_abort;
  float q[PPT][2 * R + 1];
  long long m = 0, qi = 0;  // planes consumed from each ring
  long long u = u0;
  bool aborted = false;
  while (u < u1 && !aborted) {
    const int t = int(u / wk.nz);
    const int zb = int(u % wk.nz);
    const int len = int((u1 - u) < (long long)(wk.nz - zb) ? (u1 - u) : (long long)(wk.nz - zb));
    const int x0 = (t % wk.tiles_x) * TX, y0 = (t / wk.tiles_x) * TY;
    const int x = x0 + tx;
    for (int j = 0; j < len + 2 * R; ++j) {
      const bool compute = j >= 2 * R;
      const int slot = int(m % C::NP);
      bool ok = mbar_wait_bounded(bar_p0 + 8u * slot, uint32_t((m / C::NP) & 1), limit_ns);
      if (ok && compute) ok = mbar_wait_bounded(bar_q0 + 8u * int(qi % NQ), uint32_t((qi / NQ) & 1), limit_ns);
      if (!ok) {
        *abort_flag = 1;
      } else {
        const float* P = sp + slot * C::P_FLOATS;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
#pragma unroll
          for (int k = 0; k < 2 * R; ++k) q[i][k] = q[i][k + 1];
          q[i][2 * R] = P[(ty * PPT + i + R) * C::PW + tx + C::XH];
        }
        if (compute) {
          const int z = zb + j - 2 * R;
          const float* Pc = sp + int((m - R) % C::NP) * C::P_FLOATS;
          const float* Qs = sq + int(qi % NQ) * C::Q_FLOATS;
          const float* Ks = sk + int(qi % NQ) * C::Q_FLOATS;
          const int64_t zoff = int64_t(z) * a.sz;
          const int dz = layer_distance(z, a.nz, a.nbl[0], a.nbl[1]);
          const int dx = layer_distance(x, a.nx, a.nbl[4], a.nbl[5]);
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            const int row = ty * PPT + i;
            const float* c = Pc + (row + R) * C::PW + tx + C::XH;  // centre node in the slot
            const float pc = q[i][R];
            const float p2 = 2.f * pc;
            float lap = 0.f;
#pragma unroll
            for (int jj = 1; jj <= R; ++jj) {
              lap = fmaf(a.cz[jj], (q[i][R + jj] + q[i][R - jj]) - p2, lap);
              lap = fmaf(a.cx[jj], (c[jj] + c[-jj]) - p2, lap);
              lap = fmaf(a.cy[jj], (c[jj * C::PW] + c[-jj * C::PW]) - p2, lap);
            }
            const float po = Qs[row * TX + tx];
            const float kp = Ks[row * TX + tx];
            const int y = y0 + row;
            if (x < a.nx && y < a.ny) {
              const int dy = layer_distance(y, a.ny, a.nbl[2], a.nbl[3]);
              const int d2 = dz * dz + dy * dy + dx * dx;
              float ca = 1.f, e = 0.f;
              if (d2 != 0) {
                const float2 cc = __ldg(&a.damp[d2]);
                ca = cc.x;
                e = cc.y;
              }
              const float dp = pc - po;
              float pnew = ca * (pc + fmaf(kp, lap, fmaf(e, po, dp)));
              const bool dir = (z == 0 && a.bc[0] == kBcDirichlet) || (z == a.nz - 1 && a.bc[1] == kBcDirichlet) ||
                               (y == 0 && a.bc[2] == kBcDirichlet) || (y == a.ny - 1 && a.bc[3] == kBcDirichlet) ||
                               (x == 0 && a.bc[4] == kBcDirichlet) || (x == a.nx - 1 && a.bc[5] == kBcDirichlet);
              if (dir) pnew = 0.f;
              const int64_t idx = zoff + int64_t(y) * a.sy + x;
              a.pnm1[idx] = pnew;
              mirror_ghosts<R>(a.pnm1, idx, z, a.nz, a.sz, a.bc[0], a.bc[1], pnew);
              mirror_ghosts<R>(a.pnm1, idx, y, a.ny, a.sy, a.bc[2], a.bc[3], pnew);
              mirror_ghosts<R>(a.pnm1, idx, x, a.nx, 1, a.bc[4], a.bc[5], pnew);
            }
          }
        }
      }
      __syncthreads();  // slot m-R of the p ring and slot qi of the q ring are free
      if (*abort_flag) {
        aborted = true;
        break;
      }
      if (compute) ++qi;
      ++m;
      if (tid == 0) {
        if (cp.valid()) issue_p();
        if (compute && cq.valid()) issue_q();
      }
    }
    u += len;
  }

  if (aborted && tid == 0) {
    atomicOr(err_flag, 1);
    // drain this CTA's outstanding copies (bounded) before its shared memory goes away
    for (long long k = m; k < p_issued; ++k)
      mbar_wait_bounded(bar_p0 + 8u * int(k % C::NP), uint32_t((k / C::NP) & 1), limit_ns);
    for (long long k = qi; k < q_issued; ++k)
      mbar_wait_bounded(bar_q0 + 8u * int(k % NQ), uint32_t((k / NQ) & 1), limit_ns);
  }
}

}  // namespace sw
