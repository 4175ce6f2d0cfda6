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
//   - each thread keeps its columns' 2R+1 planes of p[n] in a register queue
//     (shifted once per plane), so a plane is read from shared memory once for
//     z and once per in-plane neighbour;
//   - per-slot "empty" mbarriers, which each warp signals when it is done
//     with a plane, gate the refills; only the issuing lane waits on them, so
//     there is no block-wide barrier inside the loop;
//   - each lane computes two adjacent columns with 64-bit shared loads and
//     packed FP32x2 arithmetic, the Laplacian in three per-axis chains;
//   - boundary work (Dirichlet nodes, face mirroring, ragged tails) only runs
//     for nodes within R of a face, decided per lane, row and plane;
//     per-segment and per-plane invariants are computed once.
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

template <int R, int TY, int PPT, int D, int NQ>
struct TmaConfig {
  static constexpr int TX = 64;               // 32 lanes x 2 adjacent columns
  static constexpr int XH = (R + 3) / 4 * 4;  // x halo rounded to 16 bytes (TMA x alignment)
  static constexpr int PW = TX + 2 * XH;
  static constexpr int PH = TY + 2 * R;
  static constexpr int NP = R + 1 + D;       // p[n] ring: R+1 live planes + D prefetched
  static constexpr int NCW = TY / PPT;       // warps, PPT rows each
  static constexpr int NT = 32 * NCW;
  static constexpr int QL = 2 * R + 1;       // register z-queue length
  static constexpr int H = (R + 1) / 2;      // float2 loads each side for the x neighbours
  static constexpr uint32_t P_BYTES = uint32_t(PH * PW) * 4u;  // bytes one p[n] box delivers
  static constexpr uint32_t Q_BYTES = uint32_t(TY * TX) * 4u;  // bytes one p[n-1] / kappa box delivers
  // Slot strides are padded to 128 bytes: a tensor copy's shared-memory
  // destination must be 128-byte aligned.
  static constexpr int P_FLOATS = int((P_BYTES + 127u) / 128u * 128u) / 4;
  static constexpr int Q_FLOATS = int((Q_BYTES + 127u) / 128u * 128u) / 4;
  static constexpr size_t SMEM = size_t(NP) * P_FLOATS * 4 + 2 * size_t(NQ) * Q_FLOATS * 4 +
                                 size_t(2 * NP + 2 * NQ) * 8 + 16 + 128;  // + abort flag, producer state
  static_assert((P_FLOATS * 4) % 128 == 0 && (Q_FLOATS * 4) % 128 == 0, "TMA destinations must stay 128-byte aligned");
  static_assert(kTileXMax % TX == 0 && kTileYMax % TY == 0 && TY % PPT == 0, "tile shape");
  static_assert(PW <= 256 && PH <= 256 && XH % 2 == 0, "TMA box extent / float2 alignment");
};

// Boundary work for one node of a tile that touches a face: Dirichlet face
// nodes are held at zero, the node itself is stored, and its mirror images go
// into the ghost layers of p[n+1].
template <int R>
__device__ __forceinline__ void store_near_face(const StencilArgs& a, int64_t idx, int x, int y, int z, float v) {
  if (x >= a.nx || y >= a.ny) return;
  const bool dir = (z == 0 && a.bc[0] == kBcDirichlet) || (z == a.nz - 1 && a.bc[1] == kBcDirichlet) ||
                   (y == 0 && a.bc[2] == kBcDirichlet) || (y == a.ny - 1 && a.bc[3] == kBcDirichlet) ||
                   (x == 0 && a.bc[4] == kBcDirichlet) || (x == a.nx - 1 && a.bc[5] == kBcDirichlet);
  if (dir) v = 0.f;
  a.pnm1[idx] = v;
  mirror_ghosts<R>(a.pnm1, idx, z, a.nz, a.sz, a.bc[0], a.bc[1], v);
  mirror_ghosts<R>(a.pnm1, idx, y, a.ny, a.sy, a.bc[2], a.bc[3], v);
  mirror_ghosts<R>(a.pnm1, idx, x, a.nx, 1, a.bc[4], a.bc[5], v);
}

// Warp w owns tile rows w*PPT..w*PPT+PPT-1; lane l owns columns 2l and 2l+1,
// handled as a float2 with packed FP32x2 arithmetic.  Lane 0 of the last warp
// also issues every tensor copy.
// Ring protocol per slot: full[s] (1 arrival + transaction bytes) completes when
// a copy lands; empty[s] (NCW arrivals) completes when every consumer warp has
// finished with the plane in it.  p[n] plane index m is used by a consumer
// warp as the queue front at its iteration m and as the in-plane centre at
// iteration m+R, so the warp releases index m-R at the end of iteration m.
// Face treatment of node index i along one axis of length n: whether it is a
// Dirichlet face node (held at zero) and where its mirror image goes in the
// ghost layer (offset in nodes along the axis, 0 = none) with which sign.
// Assumes n > 2R+1, so a node is within R of at most one face.
struct FaceTreat {
  bool zero;
  int mirror;
  float sign;
};

template <int R>
__device__ __forceinline__ FaceTreat face_treat(int i, int n, int bc_lo, int bc_hi) {
  FaceTreat f;
  f.zero = (i == 0 && bc_lo == kBcDirichlet) || (i == n - 1 && bc_hi == kBcDirichlet);
  f.mirror = 0;
  f.sign = 1.f;
  if (bc_lo != kBcNone && i >= 1 && i <= R) {
    f.mirror = -2 * i;
    f.sign = (bc_lo == kBcDirichlet) ? -1.f : 1.f;
  } else if (bc_hi != kBcNone && n - 1 - i >= 1 && n - 1 - i <= R) {
    f.mirror = 2 * (n - 1 - i);
    f.sign = (bc_hi == kBcDirichlet) ? -1.f : 1.f;
  }
  return f;
}

// Producer bookkeeping, kept in shared memory because one lane uses it.
struct ProducerState {
  SegCursor cp, cq;
  long long kp, kq;  // copies issued into each ring
};

// ISO: all three spacings are equal, so one coefficient per j serves every
// axis (fewer registers; same arithmetic).
template <int R, int TY, int PPT, int D, int NQ, int MINB, bool ISO>
__global__ void __launch_bounds__(TmaConfig<R, TY, PPT, D, NQ>::NT)
    stencil_tma_kernel(const __grid_constant__ CUtensorMap map_p, const __grid_constant__ CUtensorMap map_q,
                       const __grid_constant__ CUtensorMap map_k, const StencilArgs a, const TmaWork wk,
                       int* err_flag, unsigned long long limit_ns) {
  using C = TmaConfig<R, TY, PPT, D, NQ>;
  constexpr int TX = C::TX, QL = C::QL, H = C::H, PW = C::PW;
  extern __shared__ __align__(128) unsigned char smem[];
  float* sp = reinterpret_cast<float*>(smem);
  float* sq = sp + C::NP * C::P_FLOATS;
  float* sk = sq + NQ * C::Q_FLOATS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sk + NQ * C::Q_FLOATS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * C::NP + 2 * NQ);
  ProducerState* st = reinterpret_cast<ProducerState*>(bars + 2 * C::NP + 2 * NQ + 2);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long u0 = wk.total * blockIdx.x / gridDim.x;
  const long long u1 = wk.total * (blockIdx.x + 1) / gridDim.x;
  if (u0 >= u1) return;
  if (smem_addr(smem) & 127u) {  // tensor copies need 128-byte aligned destinations
    if (threadIdx.x == 0) atomicOr(err_flag, 2);
    return;
  }
  const uint32_t full_p = smem_addr(bars);
  const uint32_t empty_p = full_p + 8u * C::NP;
  const uint32_t full_q = empty_p + 8u * C::NP;
  const uint32_t empty_q = full_q + 8u * NQ;
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int i = 0; i < C::NP; ++i) {
      mbar_init(full_p + 8u * i, 1);
      mbar_init(empty_p + 8u * i, C::NCW);
    }
    for (int i = 0; i < NQ; ++i) {
      mbar_init(full_q + 8u * i, 1);
      mbar_init(empty_q + 8u * i, C::NCW);
    }
    fence_barrier_init();
  }
  __syncthreads();

  // The last warp's lane 0 is also the producer: it issues the first copies
  // up front and then, at the end of each of its iterations, the copy into the
  // slot every warp has just released (waiting on that slot's "empty"
  // barrier).  The other warps never wait for it except through data: they
  // can run up to D planes ahead.
  const bool producer = (warp == C::NCW - 1) && lane == 0;
  // issue the next p[n] copy; false if a bounded wait gave up
  auto issue_p = [&]() -> bool {
    const long long k = st->kp;
    const int slot = int(k % C::NP);
    if (k >= C::NP && !mbar_wait_bounded(empty_p + 8u * slot, uint32_t(((k / C::NP) - 1) & 1), limit_ns))
      return false;
    const int t = st->cp.tile();
    const int x0 = (t % wk.tiles_x) * TX, y0 = (t / wk.tiles_x) * TY;
    const uint32_t bar = full_p + 8u * slot;
    mbar_arrive_expect_tx(bar, C::P_BYTES);
    tma_load_3d(smem_addr(sp + slot * C::P_FLOATS), &map_p, x0 + kXOff - C::XH, y0, st->cp.zb() + st->cp.j, bar);
    st->kp = k + 1;
    st->cp.advance();
    return true;
  };
  auto issue_q = [&]() -> bool {
    const long long k = st->kq;
    const int slot = int(k % NQ);
    if (k >= NQ && !mbar_wait_bounded(empty_q + 8u * slot, uint32_t(((k / NQ) - 1) & 1), limit_ns)) return false;
    const int t = st->cq.tile();
    const int x0 = (t % wk.tiles_x) * TX, y0 = (t / wk.tiles_x) * TY;
    const int z = st->cq.zb() + st->cq.j;
    const uint32_t bar = full_q + 8u * slot;
    mbar_arrive_expect_tx(bar, 2u * C::Q_BYTES);
    tma_load_3d(smem_addr(sq + slot * C::Q_FLOATS), &map_q, x0 + kXOff, y0 + R, z + R, bar);
    tma_load_3d(smem_addr(sk + slot * C::Q_FLOATS), &map_k, x0 + kXOff, y0 + R, z + R, bar);
    st->kq = k + 1;
    st->cq.advance();
    return true;
  };
  // on a failed wait: raise the flags and let this CTA's issued copies land
  auto give_up = [&]() {
    *abort_flag = 1;
    atomicOr(err_flag, 1);
    if (producer) {
      const long long kp = st->kp, kq = st->kq;
      for (long long i = (kp > C::NP ? kp - C::NP : 0); i < kp; ++i)
        mbar_wait_bounded(full_p + 8u * int(i % C::NP), uint32_t((i / C::NP) & 1), limit_ns);
      for (long long i = (kq > NQ ? kq - NQ : 0); i < kq; ++i)
        mbar_wait_bounded(full_q + 8u * int(i % NQ), uint32_t((i / NQ) & 1), limit_ns);
    }
  };
  if (producer) {
    prefetch_tensormap(&map_p);
    prefetch_tensormap(&map_q);
    prefetch_tensormap(&map_k);
    st->cp.init(u0, u1, wk.nz, 2 * R);
    st->cq.init(u0, u1, wk.nz, 0);
    st->kp = 0;
    st->kq = 0;
    for (int i = 0; i <= D && st->cp.valid(); ++i) issue_p();  // slots still free: no waits
    for (int i = 0; i < NQ && st->cq.valid(); ++i) issue_q();
  }

  // --------------------------------------------------------------- consumers
  float2 cz2[R + 1], cy2[R + 1], cx2[R + 1];  // coefficient pairs (ISO: one set)
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    cx2[j] = make_float2(a.cx[j], a.cx[j]);
    cy2[j] = ISO ? cx2[j] : make_float2(a.cy[j], a.cy[j]);
    cz2[j] = ISO ? cx2[j] : make_float2(a.cz[j], a.cz[j]);
  }
  const int r0 = warp * PPT;  // first tile row of this warp
  float2 qz[PPT][QL];         // z-queue, shifted once per plane
  // ring positions (32-bit): front slot and phase, centre slot, q slot and phase
  int ps = 0, cs = C::NP - R;
  uint32_t pph = 0;
  int qs = 0;
  uint32_t qph = 0;
  int consumed = 0;  // p[n] planes consumed, saturating at R
  long long u = u0;
  while (u < u1) {
    const int t = int(u / wk.nz);
    const int zb = int(u % wk.nz);
    const int len = int((u1 - u) < (long long)(wk.nz - zb) ? (u1 - u) : (long long)(wk.nz - zb));
    const int x0 = (t % wk.tiles_x) * TX, y0 = (t / wk.tiles_x) * TY;
    const int x = x0 + 2 * lane;
    // per-segment invariants; a node is "near" when it is a Dirichlet face
    // node, has a ghost mirror image, or lies past the last node (ragged tile)
    const bool small = a.nx <= 2 * R + 1 || a.ny <= 2 * R + 1 || a.nz <= 2 * R + 1;
    const bool va_ok = x < a.nx, vb_ok = x + 1 < a.nx;
    const FaceTreat fxa = face_treat<R>(x, a.nx, a.bc[4], a.bc[5]);
    const FaceTreat fxb = face_treat<R>(x + 1, a.nx, a.bc[4], a.bc[5]);
    const bool lane_near = !va_ok || !vb_ok || fxa.zero || fxb.zero || fxa.mirror || fxb.mirror;
    bool seg_near = small || __any_sync(0xffffffffu, lane_near);
    const int dxa = layer_distance(x, a.nx, a.nbl[4], a.nbl[5]);
    const int dxb = layer_distance(x + 1, a.nx, a.nbl[4], a.nbl[5]);
    int d2xy_a[PPT], d2xy_b[PPT];
    int rowoff[PPT];  // in-plane offsets fit 32 bits (checked on the host)
    FaceTreat fy[PPT];
    bool row_ok[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int y = y0 + r0 + i;
      const int dyl = layer_distance(y, a.ny, a.nbl[2], a.nbl[3]);
      d2xy_a[i] = dyl * dyl + dxa * dxa;
      d2xy_b[i] = dyl * dyl + dxb * dxb;
      rowoff[i] = y * int(a.sy) + x;
      fy[i] = face_treat<R>(y, a.ny, a.bc[2], a.bc[3]);
      row_ok[i] = y < a.ny;
      seg_near = seg_near || !row_ok[i] || fy[i].zero || fy[i].mirror != 0;  // warp-uniform
    }
    const int nplanes = len + 2 * R;
    for (int j = 0; j < nplanes; ++j) {
      if (*abort_flag) return;
      const bool compute = j >= 2 * R;
      bool ok = mbar_wait_bounded(full_p + 8u * ps, pph, limit_ns);
      if (ok && compute) ok = mbar_wait_bounded(full_q + 8u * qs, qph, limit_ns);
      if (!ok) {
        give_up();
        return;
      }
      {
        const float* P = sp + ps * C::P_FLOATS + (r0 + R) * PW + C::XH + 2 * lane;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
#pragma unroll
          for (int kk = 0; kk < QL - 1; ++kk) qz[i][kk] = qz[i][kk + 1];
          qz[i][QL - 1] = *reinterpret_cast<const float2*>(P + i * PW);
        }
      }
      if (compute) {
        const int z = zb + j - 2 * R;
        const float* c0 = sp + cs * C::P_FLOATS + (r0 + R) * PW + C::XH + 2 * lane;
        const float2* Qs = reinterpret_cast<const float2*>(sq + qs * C::Q_FLOATS + r0 * TX + 2 * lane);
        const float2* Ks = reinterpret_cast<const float2*>(sk + qs * C::Q_FLOATS + r0 * TX + 2 * lane);
        float* plane = a.pnm1 + int64_t(z) * a.sz;
        const int dzl = layer_distance(z, a.nz, a.nbl[0], a.nbl[1]);
        const int dz2 = dzl * dzl;
        const FaceTreat fz = face_treat<R>(z, a.nz, a.bc[0], a.bc[1]);
        const bool near = seg_near || fz.zero || fz.mirror != 0;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          const float* c = c0 + i * PW;
          float2 w[2 * H + 1];  // columns x-2H .. x+1+2H of this row, as pairs
#pragma unroll
          for (int mm = -H; mm <= H; ++mm) w[mm + H] = *reinterpret_cast<const float2*>(c + 2 * mm);
          const float2 pc = qz[i][R];
          const float2 p2 = f2_add(pc, pc);
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
            const float2 ys = f2_add(*reinterpret_cast<const float2*>(c + jj * PW),
                                     *reinterpret_cast<const float2*>(c - jj * PW));
            ly = f2_fma(cy2[jj], f2_sub(ys, p2), ly);
          }
          const float2 lap = f2_add(f2_add(lz, lx), ly);
          const float2 po = Qs[i * (TX / 2)];
          const float2 kp = Ks[i * (TX / 2)];
          // damping coefficients (entry 0 of the table is (1, 0): no branch needed)
          const float2 da = __ldg(&a.damp[dz2 + d2xy_a[i]]);
          const float2 db = __ldg(&a.damp[dz2 + d2xy_b[i]]);
          const float2 ca = make_float2(da.x, db.x), e = make_float2(da.y, db.y);
          // p[n+1] = a (p + (kappa L + ((p - p[n-1]) + e p[n-1])))
          const float2 pnew = f2_mul(ca, f2_add(pc, f2_fma(kp, lap, f2_fma(e, po, f2_sub(pc, po)))));
          float* dst = plane + rowoff[i];
          if (!near) {
            *reinterpret_cast<float2*>(dst) = pnew;
          } else if (small) {
            const int y = y0 + r0 + i;
            const int64_t idx = int64_t(z) * a.sz + rowoff[i];
            store_near_face<R>(a, idx, x, y, z, pnew.x);
            store_near_face<R>(a, idx + 1, x + 1, y, z, pnew.y);
          } else if (row_ok[i]) {
            // Dirichlet face nodes are held at zero; mirror images go to the ghosts
            const bool zrow = fz.zero || fy[i].zero;
            const float va = (zrow || fxa.zero) ? 0.f : pnew.x;
            const float vb = (zrow || fxb.zero) ? 0.f : pnew.y;
            if (va_ok && vb_ok) {
              *reinterpret_cast<float2*>(dst) = make_float2(va, vb);
            } else if (va_ok) {
              dst[0] = va;
            }
            if (va_ok && fxa.mirror) dst[fxa.mirror] = fxa.sign * va;
            if (vb_ok && fxb.mirror) dst[1 + fxb.mirror] = fxb.sign * vb;
            if (fy[i].mirror) {
              float* g = dst + fy[i].mirror * int(a.sy);
              if (va_ok) g[0] = fy[i].sign * va;
              if (vb_ok) g[1] = fy[i].sign * vb;
            }
            if (fz.mirror) {
              float* g = dst + int64_t(fz.mirror) * a.sz;
              if (va_ok) g[0] = fz.sign * va;
              if (vb_ok) g[1] = fz.sign * vb;
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        if (consumed >= R) mbar_arrive(empty_p + 8u * cs);
        if (compute) mbar_arrive(empty_q + 8u * qs);
      }
      if (producer) {
        bool fine = true;
        if (st->cp.valid()) fine = issue_p();
        if (fine && compute && st->cq.valid()) fine = issue_q();
        if (!fine) {
          give_up();
          return;
        }
      }
      // advance ring positions
      if (++ps == C::NP) {
        ps = 0;
        pph ^= 1u;
      }
      if (++cs == C::NP) cs = 0;  // centre slot tracks index m-R every iteration
      if (consumed < R) ++consumed;
      if (compute) {
        if (++qs == NQ) {
          qs = 0;
          qph ^= 1u;
        }
      }
    }
    u += len;
  }
}

}  // namespace sw
