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
// rows; the tiles of all groups are numbered consecutively (group after group,
// rows of tiles along x) and a persistent grid walks them.  One thread owns
// one column of a tile and marches down its rows with the z-neighbours in a
// register queue (kBatchU new rows per chunk, so several row loads are in
// flight at once); x-neighbours come through L1.  The arithmetic is the same
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
  int tile_base;  // number of the group's first tile
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

template <int R>
__global__ void __launch_bounds__(kBatchTX) batch_stencil_2d_kernel(const BatchGroup* __restrict__ groups,
                                                                   int n_groups, const BatchShot* __restrict__ shots,
                                                                   int total_tiles, int parity) {
  // kappa of the current tile; every thread reads back only its own column,
  // so the array needs no barrier
  __shared__ float ks[kBatchZB][kBatchTX];
  const int tid = threadIdx.x;
  for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    int lo = 0, hi = n_groups - 1;  // last group whose first tile is <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (groups[mid].tile_base <= t) lo = mid;
      else hi = mid - 1;
    }
    const BatchGroup& G = groups[lo];
    const int local = t - G.tile_base;
    const int strip = local / G.tiles_x;
    const int x = (local - strip * G.tiles_x) * kBatchTX + tid;
    if (x >= G.nx) continue;
    const int nz = G.nz, nx = G.nx;
    const int z0 = strip * kBatchZB;
    const int z1 = min(z0 + kBatchZB, nz);
    const int64_t sz = G.sz;
    for (int r = 0; r < z1 - z0; ++r) ks[r][tid] = __ldg(&G.kappa[int64_t(z0 + r) * sz + x]);
    float cz[R + 1], cx[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) {
      cz[j] = G.cz[j];
      cx[j] = G.cx[j];
    }
    const int dx = layer_distance(x, nx, G.nbl[2], G.nbl[3]);
    const bool xdir = (x == 0 && G.bc[2] == kBcDirichlet) || (x == nx - 1 && G.bc[3] == kBcDirichlet);
    const int bz0 = G.bc[0], bz1 = G.bc[1], bx0 = G.bc[2], bx1 = G.bc[3];
    const int nbz0 = G.nbl[0], nbz1 = G.nbl[1];
    const float2* damp = G.damp;
    for (int s = G.first; s < G.first + G.count; ++s) {
      const float* __restrict__ pn = shots[s].u[parity];
      float* pout = shots[s].u[parity ^ 1];  // holds p[n-1] until overwritten
      float q[2 * R + kBatchU];              // p[n] of rows z - R .. z + R + U - 1 in this column
#pragma unroll
      for (int j = 0; j < 2 * R; ++j) q[j] = __ldg(&pn[int64_t(z0 - R + j) * sz + x]);
      for (int z = z0; z < z1; z += kBatchU) {
        float po[kBatchU];
#pragma unroll
        for (int u = 0; u < kBatchU; ++u) {
          const int zr = z + R + u;  // rows past nz - 1 + R feed only rows past the grid
          q[2 * R + u] = zr < nz + R ? __ldg(&pn[int64_t(zr) * sz + x]) : 0.f;
          po[u] = z + u < z1 ? pout[int64_t(z + u) * sz + x] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kBatchU; ++u) {
          const int zu = z + u;
          if (zu < z1) {
            const int64_t idx = int64_t(zu) * sz + x;
            float qx[2 * R + 1];
            qx[R] = q[u + R];
#pragma unroll
            for (int j = 1; j <= R; ++j) {
              qx[R + j] = __ldg(&pn[idx + j]);
              qx[R - j] = __ldg(&pn[idx - j]);
            }
            const float lap = laplacian_2d<R>(q + u, qx, cz, cx);
            const int dz = layer_distance(zu, nz, nbz0, nbz1);
            const int d2 = dz * dz + dx * dx;
            float ca = 1.f, e = 0.f;
            if (d2 != 0) {
              const float2 c = __ldg(&damp[d2]);
              ca = c.x;
              e = c.y;
            }
            float pnew = leapfrog_update(q[u + R], po[u], ks[zu - z0][tid], lap, ca, e);
            if (xdir || (zu == 0 && bz0 == kBcDirichlet) || (zu == nz - 1 && bz1 == kBcDirichlet)) pnew = 0.f;
            pout[idx] = pnew;
            mirror_ghosts<R>(pout, idx, zu, nz, sz, bz0, bz1, pnew);
            mirror_ghosts<R>(pout, idx, x, nx, 1, bx0, bx1, pnew);
          }
        }
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) q[j] = q[j + kBatchU];
      }
    }
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
