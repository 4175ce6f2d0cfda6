// Two leapfrog steps per pass over memory for 2D grids of constant density
// (temporal blocking).
//
// The per-step 2D kernels stream p[n], p[n-1] and kappa and write p[n+1]
// for every step: 16 bytes per node update.  This kernel advances a tile by
// two steps per launch: tensor copies stage p[n] on the tile plus a 2R-node
// ring and p[n-1], kappa on the tile plus an R-node ring in shared memory
// (the next tile's copies in flight while the CTA works), it computes
// p[n+1] (Eq. 7, with step n's source taps of Eq. 11 and the face images of
// the ghost nodes) on the tile plus its R-node ring, and from that p[n+2]
// on the tile.  It writes both new levels: 20 bytes per two node updates
// plus the halo rows read twice.  The first step's ring is computed by
// both neighbouring tiles (recomputation instead of communication).
//
// Every node value is formed by the operations of the per-step kernels in
// the same order (laplacian_2d, leapfrog_update, the tap increment of
// inject_source_node), so the levels equal theirs bit for bit when no two
// source taps share a node.  The new levels go to two other buffers than
// the two it reads (neighbouring tiles still read p[n] and p[n-1]); the
// ghost nodes of both new levels, step n+1's sources and the receivers are
// left to the launches that follow it.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "aux_kernels.cuh"
#include "layout.h"
#include "stencil_plain.cuh"
#include "tma.cuh"

namespace sw {

constexpr int kTb2TZ = 32;        // tile rows (z)
constexpr int kTb2TX = 64;        // tile columns (x)
constexpr int kTb2Threads = 256;

struct Tb2Args {
  float* out1;       // p[n+1] at node (0, 0) (node values)
  float* out2;       // p[n+2] (node values, without step n+1's sources)
  const float2* damp;
  int64_t sz;        // row stride
  int nz, nx;
  int nbl[4];        // absorbing cells: z low, z high, x low, x high
  int bc[4];         // face conditions in the same order
  float cz[kMaxR + 1], cx[kMaxR + 1];  // v_j / h^2
  PointSet src;      // source windows (1/prod(h) folded into the x weights)
  const float* sig;
  int sig_stride;
  int step;          // n
  int tiles_x, tiles;
};

// Shared-memory images of one tile: p[n] over the tile and a 2R ring (rows),
// p[n-1] and kappa over the tile and an R ring; their x halos are rounded up
// to 4 floats so that every tensor copy starts on a 16-byte boundary.  Two
// slots of the three images (the next tile's copies land in one while the
// CTA works on the other) and one image of p[n+1].
template <int R>
struct Tb2Cfg {
  static constexpr int XA0 = (2 * R + 3) / 4 * 4, XA1 = (R + 3) / 4 * 4;
  static constexpr int W0 = kTb2TX + 2 * XA0, H0 = kTb2TZ + 4 * R;
  static constexpr int W1 = kTb2TX + 2 * XA1, H1 = kTb2TZ + 2 * R;
  static constexpr int F0 = (H0 * W0 + 31) / 32 * 32, F1 = (H1 * W1 + 31) / 32 * 32;  // 128-byte multiples
  static constexpr int SLOT = F0 + 2 * F1;
  static constexpr uint32_t TX_BYTES = uint32_t(H0 * W0 + 2 * H1 * W1) * 4u;
  static constexpr size_t BYTES = (size_t(2) * SLOT + F1) * sizeof(float) + 2 * sizeof(uint64_t) + 16;
  static_assert(W0 <= 256 && H0 <= 256, "tensor copy box extent");
};

// Box extents of the tensor maps of a radius (host side, for the maps).
inline void tb2_boxes(int R, int* w0, int* h0, int* w1, int* h1) {
  const int xa0 = (2 * R + 3) / 4 * 4, xa1 = (R + 3) / 4 * 4;
  *w0 = kTb2TX + 2 * xa0;
  *h0 = kTb2TZ + 4 * R;
  *w1 = kTb2TX + 2 * xa1;
  *h1 = kTb2TZ + 2 * R;
}

__device__ __forceinline__ bool tb2_dirichlet(const Tb2Args& a, int z, int x) {
  return (z == 0 && a.bc[0] == kBcDirichlet) || (z == a.nz - 1 && a.bc[1] == kBcDirichlet) ||
         (x == 0 && a.bc[2] == kBcDirichlet) || (x == a.nx - 1 && a.bc[3] == kBcDirichlet);
}

// Maps (3D over the padded field with a y extent of 1): map_n boxes of
// W0 x 1 x H0 over p[n], map_m and map_k boxes of W1 x 1 x H1 over p[n-1] and
// kappa.  A persistent grid walks the tiles (CTA b: tiles b, b + G, ...).
template <int R>
__global__ void __launch_bounds__(kTb2Threads) tb2_2d_kernel(const __grid_constant__ CUtensorMap map_n,
                                                             const __grid_constant__ CUtensorMap map_m,
                                                             const __grid_constant__ CUtensorMap map_k,
                                                             const Tb2Args a, int* err_flag,
                                                             unsigned long long limit_ns) {
  using C = Tb2Cfg<R>;
  constexpr int W0 = C::W0, W1 = C::W1, H1 = C::H1, XA0 = C::XA0, XA1 = C::XA1;
  extern __shared__ __align__(128) float tb2_smem[];
  float* P1 = tb2_smem + 2 * C::SLOT;  // p[n+1]: rows z0 - R .., columns x0 - XA1 ..
  uint64_t* bars = reinterpret_cast<uint64_t*>(P1 + C::F1);
  griddep_launch_dependents();
  griddep_wait();  // the previous launches' levels
  const int tid = threadIdx.x;
  if (int(blockIdx.x) >= a.tiles) return;
  if (smem_addr(tb2_smem) & 127u) {  // tensor copies need 128-byte aligned destinations
    if (tid == 0) atomicOr(err_flag, 2);
    return;
  }
  const uint32_t bar0 = smem_addr(bars);
  const int64_t sz = a.sz;
  // the three images of tile t into slot s (one thread)
  auto issue = [&](int t, int s) {
    const int z0 = (t / a.tiles_x) * kTb2TZ, x0 = (t % a.tiles_x) * kTb2TX;
    float* sl = tb2_smem + s * C::SLOT;
    const uint32_t bar = bar0 + 8u * s;
    mbar_arrive_expect_tx(bar, C::TX_BYTES);
    // padded coordinates: x + kXOff, z + R (rows before -R read as zeros, never used)
    tma_load_3d(smem_addr(sl), &map_n, x0 - XA0 + kXOff, 0, z0 - R, bar);
    tma_load_3d(smem_addr(sl + C::F0), &map_m, x0 - XA1 + kXOff, 0, z0, bar);
    tma_load_3d(smem_addr(sl + C::F0 + C::F1), &map_k, x0 - XA1 + kXOff, 0, z0, bar);
  };
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8u, 1);
    fence_barrier_init();
    prefetch_tensormap(&map_n);
    prefetch_tensormap(&map_m);
    prefetch_tensormap(&map_k);
    issue(blockIdx.x, 0);
  }
  __syncthreads();

  int i = 0;
  for (int t = blockIdx.x; t < a.tiles; t += gridDim.x, ++i) {
    const int s = i & 1;
    const bool more = t + int(gridDim.x) < a.tiles;
    if (tid == 0 && more) {  // the other slot was last read in the previous tile, before its final barrier
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + gridDim.x, s ^ 1);
    }
    const bool bad = !mbar_wait_bounded(bar0 + 8u * s, uint32_t((i >> 1) & 1), limit_ns);
    if (__syncthreads_or(bad)) {  // the copies never arrived: raise the flag, let ours land, leave
      if (tid == 0) {
        atomicOr(err_flag, 1);
        mbar_wait_bounded(bar0 + 8u * s, uint32_t((i >> 1) & 1), limit_ns);
        if (more) mbar_wait_bounded(bar0 + 8u * (s ^ 1), uint32_t(((i + 1) >> 1) & 1), limit_ns);
      }
      return;
    }
    const float* P0 = tb2_smem + s * C::SLOT;  // p[n]:   rows z0 - 2R .., columns x0 - XA0 ..
    const float* PM = P0 + C::F0;              // p[n-1]: rows z0 - R ..,  columns x0 - XA1 ..
    const float* KP = PM + C::F1;              // kappa
    const int z0 = (t / a.tiles_x) * kTb2TZ, x0 = (t % a.tiles_x) * kTb2TX;

    // step n: p[n+1] at the in-grid nodes of the tile and its ring; thread
    // groups take a column each and slide down a share of its rows with the
    // column's 2R+1 values of p[n] in registers
    {
      constexpr int NC = kTb2TX + 2 * R;  // ring columns x0 - R .. x0 + TX + R - 1
      constexpr int G = kTb2Threads / NC, RPG = (H1 + G - 1) / G;
      const int c = tid % NC, grp = tid / NC;
      const int x = x0 - R + c;
      if (grp < G && x >= 0 && x < a.nx) {
        const int r0 = grp * RPG, r1 = min(H1, r0 + RPG);
        const int dx = layer_distance(x, a.nx, a.nbl[2], a.nbl[3]);
        const float* col = P0 + (c - R + XA0);  // column x of the p[n] image
        const int c1 = c - R + XA1;              // column x of the ring images
        float qz[2 * R + 1], qx[2 * R + 1];
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) qz[j + 1] = col[(r0 + j) * W0];  // rows z(r0) - R .. z(r0) + R - 1
        for (int r = r0; r < r1; ++r) {
#pragma unroll
          for (int j = 0; j < 2 * R; ++j) qz[j] = qz[j + 1];
          qz[2 * R] = col[(r + 2 * R) * W0];
          const int z = z0 - R + r;
          if (z < 0 || z >= a.nz) continue;
          const float* row = col + (r + R) * W0;
#pragma unroll
          for (int j = -R; j <= R; ++j) qx[j + R] = j == 0 ? qz[R] : row[j];
          const float lap = laplacian_2d<R>(qz, qx, a.cz, a.cx);
          const int dz = layer_distance(z, a.nz, a.nbl[0], a.nbl[1]);
          const int d2 = dz * dz + dx * dx;
          const float2 d = d2 != 0 ? __ldg(&a.damp[d2]) : make_float2(1.f, 0.f);
          const int e = r * W1 + c1;
          float pnew = leapfrog_update(qz[R], PM[e], KP[e], lap, d.x, d.y);
          if (tb2_dirichlet(a, z, x)) pnew = 0.f;
          P1[e] = pnew;
        }
      }
    }
    __syncthreads();
    // step n's sources: the taps on in-grid, non-Dirichlet nodes of the tile and its ring
    {
      const PointSet& sp = a.src;
      const int taps = sp.lz * sp.ly * sp.lx;
      for (int q = tid; q < sp.count * taps; q += kTb2Threads) {
        const int p = q / taps;
        const int rem = q - p * taps;
        const int ix = rem % sp.lx;
        const int iz = rem / (sp.ly * sp.lx);
        const int z = sp.first[3 * p] + iz, x = sp.first[3 * p + 2] + ix;
        if (z < z0 - R || z >= z0 + kTb2TZ + R || x < x0 - R || x >= x0 + kTb2TX + R) continue;
        const float* w = sp.w + int64_t(p) * 3 * sp.L;
        const float wgt = w[iz] * w[sp.L] * w[2 * sp.L + ix];  // the y weight of a 2D window is 1
        if (wgt == 0.f || tb2_dirichlet(a, z, x)) continue;
        const int e = (z - z0 + R) * W1 + (x - x0 + XA1);
        const int dz = layer_distance(z, a.nz, a.nbl[0], a.nbl[1]), dx = layer_distance(x, a.nx, a.nbl[2], a.nbl[3]);
        const int d2 = dz * dz + dx * dx;
        const float ca = d2 != 0 ? __ldg(&a.damp[d2]).x : 1.f;
        atomicAdd(&P1[e], KP[e] * ca * wgt * a.sig[int64_t(p) * a.sig_stride + a.step]);
      }
    }
    __syncthreads();
    // face images of p[n+1] in the ring's ghost nodes (within R of a face;
    // the mirrored node always lies in the ring or the tile)
    for (int e = tid; e < H1 * (kTb2TX + 2 * R); e += kTb2Threads) {
      const int r = e / (kTb2TX + 2 * R), c = e - r * (kTb2TX + 2 * R);
      const int z = z0 - R + r, x = x0 - R + c;
      const bool zin = z >= 0 && z < a.nz, xin = x >= 0 && x < a.nx;
      if (zin == xin) continue;  // a node, or a corner (never read)
      int bc, mz = z, mx = x;
      if (!zin) {
        if (z < -R || z >= a.nz + R) continue;
        bc = z < 0 ? a.bc[0] : a.bc[1];
        mz = z < 0 ? -z : 2 * (a.nz - 1) - z;
      } else {
        if (x < -R || x >= a.nx + R) continue;
        bc = x < 0 ? a.bc[2] : a.bc[3];
        mx = x < 0 ? -x : 2 * (a.nx - 1) - x;
      }
      const float v = P1[(mz - z0 + R) * W1 + (mx - x0 + XA1)];
      P1[r * W1 + (c - R + XA1)] = bc == kBcNone ? 0.f : (bc == kBcDirichlet ? -v : v);
    }
    __syncthreads();
    // step n+1: p[n+2] on the tile (a column of kTb2TZ / G rows per thread,
    // sliding down p[n+1]); both levels' node values to memory
    {
      constexpr int G = kTb2Threads / kTb2TX, RPG = kTb2TZ / G;
      static_assert(kTb2Threads % kTb2TX == 0 && kTb2TZ % G == 0, "tile shape");
      const int c = tid % kTb2TX, grp = tid / kTb2TX;
      const int x = x0 + c;
      if (x < a.nx) {
        const int r0 = grp * RPG;
        const int dx = layer_distance(x, a.nx, a.nbl[2], a.nbl[3]);
        const float* col = P1 + (c + XA1);  // column x of the p[n+1] image (rows from z0 - R)
        float qz[2 * R + 1], qx[2 * R + 1];
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) qz[j + 1] = col[(r0 + j) * W1];
        for (int r = r0; r < r0 + RPG; ++r) {
#pragma unroll
          for (int j = 0; j < 2 * R; ++j) qz[j] = qz[j + 1];
          qz[2 * R] = col[(r + 2 * R) * W1];
          const int z = z0 + r;
          if (z >= a.nz) break;
          const float* row = col + (r + R) * W1;
#pragma unroll
          for (int j = -R; j <= R; ++j) qx[j + R] = j == 0 ? qz[R] : row[j];
          const float lap = laplacian_2d<R>(qz, qx, a.cz, a.cx);
          const int dz = layer_distance(z, a.nz, a.nbl[0], a.nbl[1]);
          const int d2 = dz * dz + dx * dx;
          const float2 d = d2 != 0 ? __ldg(&a.damp[d2]) : make_float2(1.f, 0.f);
          float pnew = leapfrog_update(qz[R], P0[(r + 2 * R) * W0 + (c + XA0)], KP[(r + R) * W1 + (c + XA1)], lap,
                                       d.x, d.y);
          if (tb2_dirichlet(a, z, x)) pnew = 0.f;
          const int64_t k = int64_t(z) * sz + x;
          a.out1[k] = qz[R];
          a.out2[k] = pnew;
        }
      }
    }
    __syncthreads();  // this slot and the p[n+1] image are free again
  }
}

}  // namespace sw
