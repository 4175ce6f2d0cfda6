// Batched shots: one launch per time step advances every shot of a batch of
// 2D grids of uneven sizes (constant density, one space order).
//
// The paper's solver runs one shot at a time; full-waveform inversion runs
// many shots over one model (Sec. 1 and 6 name it as the solver's use).
// Shots over the same model form a group that shares its model reads: a
// tile of the group's kappa field comes from memory once per step and serves
// every shot of the group, so the update streams 12 B per node and shot plus
// 4 B per node and group instead of 16 B per node and shot.
//
// Work list: every group is cut into tiles of kBatchTX columns by ZB rows
// (ZB = 16, 32 or 64, picked per batch by timing each, see sw_create_batch); a work item is one tile of one shot.  Items are numbered group after
// group, tile-major with the shot fastest (so the shots of a tile run side by
// side and read its kappa once from memory, then from L2), and a persistent
// grid walks them.  One warp copies the item's p[n] rows (with both halos)
// into shared memory with 1D bulk copies, one mbarrier per chunk of kBatchU
// rows, and every thread computes a chunk as soon as its barrier completes,
// so that an item's reads are all in flight at once; p[n-1] and kappa are
// loaded into registers a chunk ahead (across items too).  A thread owns two
// adjacent columns, handled as a pair with packed FP32x2 arithmetic, and
// keeps their z-neighbours in a register queue; the x-neighbours come from
// the shared image as 64-bit pairs.  Per column the arithmetic is the
// single-grid 2D kernel's (laplacian_2d, leapfrog_update: the same IEEE
// operations in the same order), so a batched shot reproduces its
// single-grid run bit for bit.
#pragma once

#include "aux_kernels.cuh"
#include "layout.h"
#include "stencil_plain.cuh"
#include "tma.cuh"

namespace sw {

constexpr int kBatchTX = 128;      // columns per tile
constexpr int kBatchThreads = 64;  // two adjacent columns per thread
constexpr int kBatchZBs[3] = {16, 32, 64};  // tile heights the tuner tries
constexpr int kBatchU = 4;     // rows per register-queue chunk

// One model shared by the shots [first, first + count) of the shot table.
struct BatchGroup {
  const float* kappa;  // node (0, 0) of the padded (c dt)^2 field
  const float2* damp;  // (a, e) by squared distance to the physical box
  int64_t sz;          // row stride of the padded layout
  int nz, nx;
  int nbl[4];  // absorbing cells: z low, z high, x low, x high
  int bc[4];   // face conditions in the same order
  float cz[kMaxR + 1], cx[kMaxR + 1];  // v_j / h^2 per axis
  int first, count;
  int tiles_x;    // tiles along x
  int item_base;  // number of the group's first work item (tile x shot)
};

// One shot: its two wavefield buffers, its sources and receivers.
struct BatchShot {
  float* u[2];  // node (0, 0) of the two levels; step n reads u[n & 1], writes u[(n + 1) & 1]
  PointSet src, rec;
  const float* kappa;
  const float2* damp;
  FaceInfo f;
  const float* wavelet;
  int sig_stride;
  float* seis;  // [n_steps][rec.count] on the device, or nullptr
};

// Shared-memory image of one work item: p[n] rows z0 - R .. z0 + ZB + R - 1
// over columns x0 - RH .. x0 + TX + RH - 1 (RH = R rounded up to 4 floats, so
// that every row starts on a 16-byte boundary).  p[n-1] and kappa, read once
// and without neighbours, go straight to registers, a chunk ahead.
template <int R, int ZB>
struct BatchSmem {
  static constexpr int RH = (R + 3) / 4 * 4;
  static constexpr int TXP = kBatchTX + 2 * RH;
  static constexpr int PROWS = ZB + 2 * R;
  static constexpr int BYTES = PROWS * TXP * 4;
};
constexpr int kBatchMaxChunks = 16;  // one mbarrier per chunk: ZB / kBatchU of them

// 1D bulk copy global -> shared, completing `bytes` on the mbarrier `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

// Where a work item lies: its group, shot, first column and row range.
struct BatchItem {
  int g, s, x0, z0, z1, nch;
};

template <int ZB>
__device__ __forceinline__ BatchItem batch_item(const BatchGroup* __restrict__ groups, int n_groups, int t) {
  int lo = 0, hi = n_groups - 1;  // last group whose first item is <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (groups[mid].item_base <= t) lo = mid;
    else hi = mid - 1;
  }
  const BatchGroup& G = groups[lo];
  // items of a group: tile-major, shot fastest, so that the shots of one
  // tile run at about the same time and share its kappa reads through L2
  const int local = t - G.item_base;
  const int tile = local / G.count;
  const int strip = tile / G.tiles_x;
  BatchItem it;
  it.g = lo;
  it.s = G.first + (local - tile * G.count);
  it.x0 = (tile - strip * G.tiles_x) * kBatchTX;
  it.z0 = strip * ZB;
  it.z1 = min(it.z0 + ZB, G.nz);
  it.nch = (it.z1 - it.z0 + kBatchU - 1) / kBatchU;
  return it;
}

// Radii up to 4: at most 128 registers, so that eight CTAs fit an SM (229
// against 208 Gpts/s for the uncapped 140 registers and seven CTAs on the
// order-8 batch; a few bytes spill); larger radii run uncapped.
template <int R, int ZB>
__global__ void __launch_bounds__(kBatchThreads, R <= 4 ? 8 : 1) batch_stencil_2d_kernel(
    const BatchGroup* __restrict__ groups, int n_groups, const BatchShot* __restrict__ shots, int total_items,
    int parity, int* err_flag, unsigned long long limit_ns) {
  static_assert(ZB % kBatchU == 0 && ZB / kBatchU <= kBatchMaxChunks, "tile height");
  constexpr int NCH = ZB / kBatchU;
  using S = BatchSmem<R, ZB>;
  constexpr int TXP = S::TXP, RH = S::RH;
  extern __shared__ __align__(128) float batch_smem[];  // the image [PROWS][TXP]
  __shared__ __align__(8) uint64_t bars[NCH];          // one per chunk
  __shared__ int abort_s;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int k = 0; k < NCH; ++k) mbar_init(smem_addr(&bars[k]), 1);
    abort_s = 0;
    fence_barrier_init();
  }
  __syncthreads();
  unsigned phases = 0;   // parity of the next phase of every barrier
  unsigned pending = 0;  // barriers armed and not yet seen complete

  // p[n-1] and kappa of a thread's column pair for one chunk (rows past z1
  // are not read; columns past nx lie in the row padding and are not stored)
  auto load_ok = [&](const BatchItem& it, int k, float2* dpo, float2* dkp) {
    const BatchGroup& G = groups[it.g];
    const int sz = int(G.sz);
    const float* ob = shots[it.s].u[parity ^ 1] + it.x0 + 2 * tid;
    const float* kb = G.kappa + it.x0 + 2 * tid;
    const int z = it.z0 + k * kBatchU;
#pragma unroll
    for (int u = 0; u < kBatchU; ++u) {
      const bool in = z + u < it.z1;
      dpo[u] = in ? *reinterpret_cast<const float2*>(ob + (z + u) * sz) : make_float2(0.f, 0.f);
      dkp[u] = in ? __ldg(reinterpret_cast<const float2*>(kb + (z + u) * sz)) : make_float2(0.f, 0.f);
    }
  };

  constexpr int H = (R + 1) / 2;  // float2 loads each side for the x neighbours
  float2 po[kBatchU], kp[kBatchU], npo[kBatchU] = {}, nkp[kBatchU] = {};
  int t = blockIdx.x;
  BatchItem cur;
  if (t < total_items) {
    cur = batch_item<ZB>(groups, n_groups, t);
    load_ok(cur, 0, po, kp);
  }
  for (; t < total_items; t += gridDim.x) {
    const int tn = t + gridDim.x;
    const BatchItem nxt = tn < total_items ? batch_item<ZB>(groups, n_groups, tn) : cur;
    const BatchGroup& G = groups[cur.g];
    const int nz = G.nz, nx = G.nx, x0 = cur.x0, z0 = cur.z0, z1 = cur.z1, nch = cur.nch;
    const int sz = int(G.sz);  // a padded field holds fewer than 2^31 elements (checked on the host)
    float* pout = shots[cur.s].u[parity ^ 1] + x0;  // holds p[n-1] until overwritten

    // warp 0 issues the item's bulk copies of p[n]: chunk 0 = the rows of the
    // first chunk with both halos, then per chunk its R-ahead rows
    if (tid < 32 && !abort_s) {
      const float* pn = shots[cur.s].u[parity] + x0;
      for (int k = 0; k < nch; ++k) {
        const int ra = k == 0 ? 0 : 2 * R + k * kBatchU;  // image rows (row r is z0 - R + r)
        const int rb = min(2 * R + (k + 1) * kBatchU, z1 - z0 + 2 * R);
        const uint32_t bar = smem_addr(&bars[k]);
        if (tid == 0) mbar_arrive_expect_tx(bar, uint32_t((rb - ra) * TXP * 4));
        __syncwarp();
        for (int r = ra + tid; r < rb; r += 32)
          bulk_load(smem_addr(batch_smem + r * TXP), pn + (z0 - R + r) * sz - RH, TXP * 4, bar);
        pending |= 1u << k;
      }
    }

    const int x = x0 + 2 * tid;  // columns x (.x of a pair) and x + 1 (.y)
    const bool act_a = x < nx, act_b = x + 1 < nx;
    float2 cz[R + 1], cx[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) {
      cz[j] = make_float2(G.cz[j], G.cz[j]);
      cx[j] = make_float2(G.cx[j], G.cx[j]);
    }
    // per-column constants: damping distance (0 past the grid, where the
    // damping table ends), Dirichlet column, x-face images
    const int dxa = act_a ? layer_distance(x, nx, G.nbl[2], G.nbl[3]) : 0;
    const int dxb = act_b ? layer_distance(x + 1, nx, G.nbl[2], G.nbl[3]) : 0;
    const int dx2a = dxa * dxa, dx2b = dxb * dxb;
    const int bz0 = G.bc[0], bz1 = G.bc[1], bx0 = G.bc[2], bx1 = G.bc[3];
    const bool xdir_a = (x == 0 && bx0 == kBcDirichlet) || (x == nx - 1 && bx1 == kBcDirichlet);
    const bool xdir_b = x + 1 == nx - 1 && bx1 == kBcDirichlet;
    const int xra = nx - 1 - x, xrb = xra - 1;
    const bool xm_lo_a = bx0 != kBcNone && x >= 1 && x <= R, xm_lo_b = bx0 != kBcNone && x + 1 <= R;
    const bool xm_hi_a = bx1 != kBcNone && xra >= 1 && xra <= R, xm_hi_b = bx1 != kBcNone && xrb >= 1 && xrb <= R;
    const bool xm_any = (xm_lo_a || xm_lo_b || xm_hi_a || xm_hi_b) && act_a;
    const float xs_lo = bx0 == kBcDirichlet ? -1.f : 1.f, xs_hi = bx1 == kBcDirichlet ? -1.f : 1.f;
    const int nbz0 = G.nbl[0], nbz1 = G.nbl[1];
    const float2* damp = G.damp;
    // damping of these columns on rows outside the z layers
    float2 ca_x = make_float2(1.f, 1.f), e_x = make_float2(0.f, 0.f);
    if (dx2a != 0) {
      const float2 c = __ldg(&damp[dx2a]);
      ca_x.x = c.x;
      e_x.x = c.y;
    }
    if (dx2b != 0) {
      const float2 c = __ldg(&damp[dx2b]);
      ca_x.y = c.x;
      e_x.y = c.y;
    }
    // node values of a row pair into p[n+1]: the pair, or column x alone at a
    // ragged edge, then the x-face images of the columns that have one
    auto put = [&](float* o, float2 v) {
      if (act_b) *reinterpret_cast<float2*>(o) = v;
      else if (act_a) o[0] = v.x;
      if (xm_any) {
        if (xm_lo_a) o[-2 * x] = xs_lo * v.x;
        if (xm_lo_b) o[1 - 2 * (x + 1)] = xs_lo * v.y;
        if (xm_hi_a) o[2 * xra] = xs_hi * v.x;
        if (xm_hi_b && act_b) o[1 + 2 * xrb] = xs_hi * v.y;
      }
    };
    // the Eq. 9 Laplacian of row u of the chunk for both columns, in the
    // order of laplacian_2d: z and x terms alternate in one FMA chain
    const float* col = batch_smem + RH + 2 * tid;  // this thread's columns of the image
    float2 q[2 * R + kBatchU];  // p[n] of rows z - R .. z + R + U - 1 of the two columns
    auto lap_row = [&](int rz, int u) {
      const float* row = col + (rz + u + R) * TXP;
      float2 w[2 * H + 1];  // columns x-2H .. x+1+2H, as pairs
#pragma unroll
      for (int mm = -H; mm <= H; ++mm)
        w[mm + H] = (mm == 0) ? q[u + R] : *reinterpret_cast<const float2*>(row + 2 * mm);
      const float2 pc = q[u + R];
      const float2 p2 = f2_add(pc, pc);  // 2 p, exactly
      float2 lap = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        lap = f2_fma(cz[j], f2_sub(f2_add(q[u + R + j], q[u + R - j]), p2), lap);
        float2 xs;  // (x+j) + (x-j) for both columns
        if (j % 2 == 0) {
          xs = f2_add(w[H + j / 2], w[H - j / 2]);
        } else {  // odd offsets straddle the pairs: two scalar adds into one pair
          xs = make_float2(w[H + (j - 1) / 2].y + w[H - (j + 1) / 2].y, w[H + (j + 1) / 2].x + w[H - (j - 1) / 2].x);
        }
        lap = f2_fma(cx[j], f2_sub(xs, p2), lap);
      }
      return lap;
    };
    // rows with nothing special along z: no z-face image, not a Dirichlet
    // face, outside the z absorbing layers
    const int plain_lo = max(R + 1, nbz0), plain_hi = min(nz - 2 - R, nz - 1 - nbz1);
    float* out = pout + 2 * tid;
    for (int k = 0; k < nch; ++k) {
      // the next chunk's p[n-1] and kappa (the next item's first chunk after the last)
      if (k + 1 < nch) load_ok(cur, k + 1, npo, nkp);
      else if (tn < total_items) load_ok(nxt, 0, npo, nkp);
      bool ok = false;
      if (!abort_s) ok = mbar_wait_bounded(smem_addr(&bars[k]), (phases >> k) & 1u, limit_ns);
      if (ok) {
        phases ^= 1u << k;
        pending &= ~(1u << k);
      } else {
        if (!abort_s) atomicOr(err_flag, 1);
        abort_s = 1;
      }
      if (ok) {
        const int z = z0 + k * kBatchU;
        const int rz = k * kBatchU;  // image row of p for z - R
        if (k == 0) {
#pragma unroll
          for (int j = 0; j < 2 * R; ++j) q[j] = *reinterpret_cast<const float2*>(col + j * TXP);
        }
#pragma unroll
        for (int u = 0; u < kBatchU; ++u)  // rows past z1 + R unused
          q[2 * R + u] = *reinterpret_cast<const float2*>(col + (rz + 2 * R + u) * TXP);
        if (act_a) {
          if (z >= plain_lo && z + kBatchU - 1 <= plain_hi && z + kBatchU <= z1) {
            // the common case: a whole chunk of plain rows
            float* o = out + z * sz;
#pragma unroll
            for (int u = 0; u < kBatchU; ++u) {
              const float2 lap = lap_row(rz, u);
              const float2 pc = q[u + R];
              // leapfrog_update for both columns
              float2 pnew = f2_mul(ca_x, f2_add(pc, f2_fma(kp[u], lap, f2_fma(e_x, po[u], f2_sub(pc, po[u])))));
              if (xdir_a) pnew.x = 0.f;
              if (xdir_b) pnew.y = 0.f;
              put(o, pnew);
              o += sz;
            }
          } else {
#pragma unroll
            for (int u = 0; u < kBatchU; ++u) {
              const int zu = z + u;
              if (zu >= z1) break;
              const float2 lap = lap_row(rz, u);
              const int dz = layer_distance(zu, nz, nbz0, nbz1);
              const int d2a = dz * dz + dx2a, d2b = dz * dz + dx2b;
              float2 ca = make_float2(1.f, 1.f), e = make_float2(0.f, 0.f);
              if (d2a != 0) {
                const float2 c = __ldg(&damp[d2a]);
                ca.x = c.x;
                e.x = c.y;
              }
              if (d2b != 0) {
                const float2 c = __ldg(&damp[d2b]);
                ca.y = c.x;
                e.y = c.y;
              }
              const float2 pc = q[u + R];
              float2 pnew = f2_mul(ca, f2_add(pc, f2_fma(kp[u], lap, f2_fma(e, po[u], f2_sub(pc, po[u])))));
              const bool zdir = (zu == 0 && bz0 == kBcDirichlet) || (zu == nz - 1 && bz1 == kBcDirichlet);
              if (xdir_a || zdir) pnew.x = 0.f;
              if (xdir_b || zdir) pnew.y = 0.f;
              float* o = out + zu * sz;
              put(o, pnew);
              if (zu <= R || zu >= nz - 1 - R) {
                mirror_ghosts<R>(o, 0, zu, nz, sz, bz0, bz1, pnew.x);
                if (act_b) mirror_ghosts<R>(o, 1, zu, nz, sz, bz0, bz1, pnew.y);
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) q[j] = q[j + kBatchU];
      }
#pragma unroll
      for (int u = 0; u < kBatchU; ++u) {
        po[u] = npo[u];
        kp[u] = nkp[u];
      }
    }
    __syncthreads();  // the next item's copies overwrite the image; abort_s is settled
    if (abort_s) break;
    cur = nxt;
  }
  // after a failed wait: let this CTA's own copies land (bounded) before it exits
  if (abort_s && tid == 0)
    for (int k = 0; k < NCH; ++k)
      if (pending & (1u << k)) mbar_wait_bounded(smem_addr(&bars[k]), (phases >> k) & 1u, limit_ns);
}

// Eq. 11 for every shot of the batch (blockIdx.y = shot), into p[n+1].
__global__ void batch_inject_kernel(const BatchShot* __restrict__ shots, int step, int parity, int R) {
  const BatchShot& S = shots[blockIdx.y];
  inject_source_tap(S.u[parity ^ 1], S.kappa, S.damp, S.src, S.wavelet, S.sig_stride, step, S.f, 2, R,
                    blockIdx.x * blockDim.x + threadIdx.x);
}

// Eq. 12 for every shot of the batch (blockIdx.y = shot), several receivers
// per warp (sample_receivers_grouped, as the single-grid 2D path).
__global__ void batch_receivers_kernel(const BatchShot* __restrict__ shots, int step, int parity) {
  const BatchShot& S = shots[blockIdx.y];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= grouped_receiver_warps(S.rec) || !S.seis) return;  // whole warps leave together
  sample_receivers_grouped(S.u[parity ^ 1], S.rec, S.f, S.seis, step, warp, threadIdx.x & 31);
}

}  // namespace sw
