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
// Work list: every group is cut into tiles of kBatchTX columns by kBatchZB
// rows; a work item is one tile of one shot.  Items are numbered group after
// group, tile-major with the shot fastest (so the shots of a tile run side by
// side and read its kappa once from memory, then from L2), and a persistent
// grid walks them.  A CTA copies the whole item (p[n] with its halo, p[n-1],
// kappa) into shared memory with asynchronous 16-byte copies, one copy group
// per chunk of kBatchU rows, and computes each chunk as soon as its group has
// landed, so that an item's reads are all in flight at once.  One thread
// owns one column and keeps its z-neighbours in a register queue; the
// x-neighbours come from the shared image.  The arithmetic is the same
// sequence of operations as the single-grid 2D kernel (laplacian_2d,
// leapfrog_update), so a batched shot reproduces its single-grid run bit for
// bit.
#pragma once

#include "aux_kernels.cuh"
#include "layout.h"
#include "stencil_plain.cuh"

namespace sw {

constexpr int kBatchTX = 128;  // columns per tile, one per thread
constexpr int kBatchZB = 32;   // rows per tile
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
// that every row starts on a 16-byte boundary), p[n-1] and kappa of rows
// z0 .. z0 + ZB - 1 over the tile's columns.
template <int R>
struct BatchSmem {
  static constexpr int RH = (R + 3) / 4 * 4;
  static constexpr int TXP = kBatchTX + 2 * RH;
  static constexpr int PROWS = kBatchZB + 2 * R;
  static constexpr int BYTES = (PROWS * TXP + 2 * kBatchZB * kBatchTX) * 4;
};

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most n of this thread's copy groups are still in flight
__device__ __forceinline__ void cp_async_wait(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
  }
}
static_assert(kBatchZB / kBatchU <= 8, "at most 8 copy groups per work item");

template <int R>
__global__ void __launch_bounds__(kBatchTX) batch_stencil_2d_kernel(const BatchGroup* __restrict__ groups,
                                                                   int n_groups, const BatchShot* __restrict__ shots,
                                                                   int total_items, int parity) {
  using S = BatchSmem<R>;
  extern __shared__ __align__(16) float batch_smem[];
  float* P = batch_smem;                         // [PROWS][TXP]
  float* O = batch_smem + S::PROWS * S::TXP;     // [ZB][TX]
  float* K = O + kBatchZB * kBatchTX;            // [ZB][TX]
  const int tid = threadIdx.x;
  for (int t = blockIdx.x; t < total_items; t += gridDim.x) {
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
    const int s = G.first + (local - tile * G.count);
    const int strip = tile / G.tiles_x;
    const int x0 = (tile - strip * G.tiles_x) * kBatchTX;
    const int nz = G.nz, nx = G.nx;
    const int z0 = strip * kBatchZB;
    const int z1 = min(z0 + kBatchZB, nz);
    const int sz = int(G.sz);  // a padded field holds fewer than 2^31 elements (checked on the host)
    const float* pn = shots[s].u[parity] + x0;
    float* pout = shots[s].u[parity ^ 1] + x0;  // holds p[n-1] until overwritten
    const float* kap = G.kappa + x0;

    // copies: group 0 = p rows of the first chunk with both halos, then one
    // group per chunk (its R-ahead p rows, its p[n-1] and kappa rows)
    const int nch = (z1 - z0 + kBatchU - 1) / kBatchU;
    for (int k = 0; k < nch; ++k) {
      const int ra = k == 0 ? 0 : 2 * R + k * kBatchU;   // smem rows of p (row r is z0 - R + r)
      const int rb = min(2 * R + (k + 1) * kBatchU, z1 - z0 + 2 * R);
      constexpr int CPR = S::TXP / 4;
      for (int i = tid; i < (rb - ra) * CPR; i += kBatchTX) {
        const int r = ra + i / CPR, c = (i - (i / CPR) * CPR) * 4;
        cp_async16(P + r * S::TXP + c, pn + (z0 - R + r) * sz + (c - S::RH));
      }
      const int oa = k * kBatchU, ob = min(oa + kBatchU, z1 - z0);
      constexpr int CPO = kBatchTX / 4;
      for (int i = tid; i < (ob - oa) * CPO; i += kBatchTX) {
        const int r = oa + i / CPO, c = (i - (i / CPO) * CPO) * 4;
        cp_async16(O + r * kBatchTX + c, pout + (z0 + r) * sz + c);
        cp_async16(K + r * kBatchTX + c, kap + (z0 + r) * sz + c);
      }
      cp_async_commit();
    }

    const int x = x0 + tid;
    const bool act = x < nx;
    float cz[R + 1], cx[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) {
      cz[j] = G.cz[j];
      cx[j] = G.cx[j];
    }
    // per-column constants: damping distance, Dirichlet column, x-mirror images
    const int dx = layer_distance(x, nx, G.nbl[2], G.nbl[3]);
    const int dx2 = dx * dx;
    const int bz0 = G.bc[0], bz1 = G.bc[1], bx0 = G.bc[2], bx1 = G.bc[3];
    const bool xdir = (x == 0 && bx0 == kBcDirichlet) || (x == nx - 1 && bx1 == kBcDirichlet);
    const int xr = nx - 1 - x;
    const bool xm_lo = bx0 != kBcNone && x >= 1 && x <= R;
    const bool xm_hi = bx1 != kBcNone && xr >= 1 && xr <= R;
    const float xs_lo = bx0 == kBcDirichlet ? -1.f : 1.f, xs_hi = bx1 == kBcDirichlet ? -1.f : 1.f;
    const int nbz0 = G.nbl[0], nbz1 = G.nbl[1];
    const float2* damp = G.damp;
    const float* col = P + S::RH + tid;  // this thread's column of the p image
    float* out = pout + tid;
    float q[2 * R + kBatchU];  // p[n] of rows z - R .. z + R + U - 1 of this column
    for (int k = 0; k < nch; ++k) {
      cp_async_wait(nch - 1 - k);
      __syncthreads();
      const int z = z0 + k * kBatchU;
      const int rz = k * kBatchU;  // smem row of p for z - R
      if (k == 0) {
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) q[j] = col[j * S::TXP];
      }
#pragma unroll
      for (int u = 0; u < kBatchU; ++u) q[2 * R + u] = col[(rz + 2 * R + u) * S::TXP];  // rows past z1 + R unused
#pragma unroll
      for (int u = 0; u < kBatchU; ++u) {
        const int zu = z + u;
        if (act && zu < z1) {
          const float* row = col + (rz + u + R) * S::TXP;
          float qx[2 * R + 1];
          qx[R] = q[u + R];
#pragma unroll
          for (int j = 1; j <= R; ++j) {
            qx[R + j] = row[j];
            qx[R - j] = row[-j];
          }
          const float lap = laplacian_2d<R>(q + u, qx, cz, cx);
          const int dz = layer_distance(zu, nz, nbz0, nbz1);
          const int d2 = dz * dz + dx2;
          float ca = 1.f, e = 0.f;
          if (d2 != 0) {
            const float2 c = __ldg(&damp[d2]);
            ca = c.x;
            e = c.y;
          }
          const int ro = (rz + u) * kBatchTX + tid;
          float pnew = leapfrog_update(q[u + R], O[ro], K[ro], lap, ca, e);
          if (xdir || (zu == 0 && bz0 == kBcDirichlet) || (zu == nz - 1 && bz1 == kBcDirichlet)) pnew = 0.f;
          float* o = out + zu * sz;
          o[0] = pnew;
          if (xm_lo) o[-2 * x] = xs_lo * pnew;
          if (xm_hi) o[2 * xr] = xs_hi * pnew;
          if (zu <= R || zu >= nz - 1 - R) mirror_ghosts<R>(o, 0, zu, nz, sz, bz0, bz1, pnew);
        }
      }
#pragma unroll
      for (int j = 0; j < 2 * R; ++j) q[j] = q[j + kBatchU];
    }
    __syncthreads();  // the next item's copies overwrite the image
  }
}

// Eq. 11 for every shot of the batch (blockIdx.y = shot), into p[n+1].
__global__ void batch_inject_kernel(const BatchShot* __restrict__ shots, int step, int parity, int R) {
  const BatchShot& S = shots[blockIdx.y];
  inject_source_tap(S.u[parity ^ 1], S.kappa, S.damp, S.src, S.wavelet, S.sig_stride, step, S.f, 2, R,
                    blockIdx.x * blockDim.x + threadIdx.x);
}

// Eq. 12 for every shot of the batch (blockIdx.y = shot): one warp per receiver.
__global__ void batch_receivers_kernel(const BatchShot* __restrict__ shots, int step, int parity) {
  const BatchShot& S = shots[blockIdx.y];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= S.rec.count || !S.seis) return;
  sample_receiver(S.u[parity ^ 1], S.rec, S.f, S.seis, step, warp, threadIdx.x & 31, false);
}

}  // namespace sw
