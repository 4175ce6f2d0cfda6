// Two leapfrog steps per pass over memory for 2D grids of constant density
// (temporal blocking).
//
// The per-step 2D kernels stream p[n], p[n-1] and kappa and write p[n+1]
// for every step: 16 bytes per node update.  This kernel advances a tile by
// two steps per launch: it stages p[n] on the tile plus a 2R-node ring and
// p[n-1], kappa on the tile plus an R-node ring in shared memory, computes
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

namespace sw {

constexpr int kTb2TZ = 32;        // tile rows (z)
constexpr int kTb2TX = 64;        // tile columns (x)
constexpr int kTb2Threads = 256;

struct Tb2Args {
  const float* pn;   // p[n] at node (0, 0) (ghost rows and columns current)
  const float* pm;   // p[n-1]
  float* out1;       // p[n+1] (node values)
  float* out2;       // p[n+2] (node values, without step n+1's sources)
  const float* kappa;
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
  int tiles_x;
};

template <int R>
struct Tb2Smem {
  static constexpr int W0 = kTb2TX + 4 * R, H0 = kTb2TZ + 4 * R;  // p[n]: tile + 2R ring
  static constexpr int W1 = kTb2TX + 2 * R, H1 = kTb2TZ + 2 * R;  // p[n-1], kappa, p[n+1]: tile + R ring
  static constexpr size_t BYTES = (size_t(H0) * W0 + 3 * size_t(H1) * W1) * sizeof(float);
};

__device__ __forceinline__ float2 tb2_damping(const Tb2Args& a, int z, int x) {
  const int dz = layer_distance(z, a.nz, a.nbl[0], a.nbl[1]);
  const int dx = layer_distance(x, a.nx, a.nbl[2], a.nbl[3]);
  const int d2 = dz * dz + dx * dx;
  return d2 != 0 ? __ldg(&a.damp[d2]) : make_float2(1.f, 0.f);
}

__device__ __forceinline__ bool tb2_dirichlet(const Tb2Args& a, int z, int x) {
  return (z == 0 && a.bc[0] == kBcDirichlet) || (z == a.nz - 1 && a.bc[1] == kBcDirichlet) ||
         (x == 0 && a.bc[2] == kBcDirichlet) || (x == a.nx - 1 && a.bc[3] == kBcDirichlet);
}

template <int R>
__global__ void __launch_bounds__(kTb2Threads) tb2_2d_kernel(const Tb2Args a) {
  using S = Tb2Smem<R>;
  constexpr int W0 = S::W0, H0 = S::H0, W1 = S::W1, H1 = S::H1;
  extern __shared__ __align__(16) float tb2_smem[];
  float* P0 = tb2_smem;        // p[n],   rows z0-2R.., columns x0-2R..
  float* PM = P0 + H0 * W0;    // p[n-1], rows z0-R..,  columns x0-R..
  float* KP = PM + H1 * W1;    // kappa
  float* P1 = KP + H1 * W1;    // p[n+1]
  griddep_launch_dependents();
  griddep_wait();  // the previous launches' levels
  const int tid = threadIdx.x;
  const int tz = blockIdx.x / a.tiles_x, tx = blockIdx.x - tz * a.tiles_x;
  const int z0 = tz * kTb2TZ, x0 = tx * kTb2TX;
  const int64_t sz = a.sz;

  // p[n] where some in-grid node of the ring reads it: nodes and ghosts,
  // rows and columns -R .. n-1+R (inside the padded allocation)
  for (int e = tid; e < H0 * W0; e += kTb2Threads) {
    const int r = e / W0, c = e - (e / W0) * W0;
    const int z = z0 - 2 * R + r, x = x0 - 2 * R + c;
    if (z >= -R && z < a.nz + R && x >= -R && x < a.nx + R) P0[e] = a.pn[int64_t(z) * sz + x];
  }
  // p[n-1] and kappa at the in-grid nodes of the tile and its ring
  for (int e = tid; e < H1 * W1; e += kTb2Threads) {
    const int r = e / W1, c = e - (e / W1) * W1;
    const int z = z0 - R + r, x = x0 - R + c;
    if (z >= 0 && z < a.nz && x >= 0 && x < a.nx) {
      const int64_t k = int64_t(z) * sz + x;
      PM[e] = a.pm[k];
      KP[e] = __ldg(&a.kappa[k]);
    }
  }
  __syncthreads();

  // step n: p[n+1] at the in-grid nodes of the tile and its ring; thread
  // groups of W1 threads take a column each and slide down a share of its
  // rows with the column's 2R+1 values of p[n] in registers
  {
    constexpr int G = kTb2Threads / W1, RPG = (H1 + G - 1) / G;  // groups, rows per group
    const int c = tid % W1, grp = tid / W1;
    const int x = x0 - R + c;
    if (grp < G && x >= 0 && x < a.nx) {
      const int r0 = grp * RPG, r1 = min(H1, r0 + RPG);
      const int dx = layer_distance(x, a.nx, a.nbl[2], a.nbl[3]);
      const float* col = P0 + R + c;  // column x of the p[n] image
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
        const int e = r * W1 + c;
        float pnew = leapfrog_update(qz[R], PM[e], KP[e], lap, d.x, d.y);
        if (tb2_dirichlet(a, z, x)) pnew = 0.f;
        P1[e] = pnew;
      }
    }
  }
  __syncthreads();
  // step n's sources: the taps on in-grid, non-Dirichlet nodes of the tile and its ring
  {
    const PointSet& s = a.src;
    const int taps = s.lz * s.ly * s.lx;
    for (int t = tid; t < s.count * taps; t += kTb2Threads) {
      const int p = t / taps;
      int rem = t - p * taps;
      const int ix = rem % s.lx;
      const int iz = rem / (s.ly * s.lx);
      const int z = s.first[3 * p] + iz, x = s.first[3 * p + 2] + ix;
      if (z < z0 - R || z >= z0 + kTb2TZ + R || x < x0 - R || x >= x0 + kTb2TX + R) continue;
      const float* w = s.w + int64_t(p) * 3 * s.L;
      const float wgt = w[iz] * w[s.L] * w[2 * s.L + ix];  // the y weight of a 2D window is 1
      if (wgt == 0.f || tb2_dirichlet(a, z, x)) continue;
      const int e = (z - z0 + R) * W1 + (x - x0 + R);
      const float2 d = tb2_damping(a, z, x);
      atomicAdd(&P1[e], KP[e] * d.x * wgt * a.sig[int64_t(p) * a.sig_stride + a.step]);
    }
  }
  __syncthreads();
  // face images of p[n+1] in the ring's ghost nodes (within R of a face;
  // the mirrored node always lies in the ring or the tile)
  for (int e = tid; e < H1 * W1; e += kTb2Threads) {
    const int r = e / W1, c = e - (e / W1) * W1;
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
    const float v = P1[(mz - z0 + R) * W1 + (mx - x0 + R)];
    P1[e] = bc == kBcNone ? 0.f : (bc == kBcDirichlet ? -v : v);
  }
  __syncthreads();

  // step n+1: p[n+2] on the tile (a column of kTb2TZ / 4 rows per thread,
  // sliding down p[n+1]); both levels' node values to memory
  {
    constexpr int G = kTb2Threads / kTb2TX, RPG = kTb2TZ / G;
    static_assert(kTb2Threads % kTb2TX == 0 && kTb2TZ % G == 0, "tile shape");
    const int c = tid % kTb2TX, grp = tid / kTb2TX;
    const int x = x0 + c;
    if (x < a.nx) {
      const int r0 = grp * RPG;
      const int dx = layer_distance(x, a.nx, a.nbl[2], a.nbl[3]);
      const float* col = P1 + R + c;  // column x of the p[n+1] image (rows from z0 - R)
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
        float pnew = leapfrog_update(qz[R], P0[(r + 2 * R) * W0 + (c + 2 * R)], KP[(r + R) * W1 + (c + R)], lap, d.x,
                                     d.y);
        if (tb2_dirichlet(a, z, x)) pnew = 0.f;
        const int64_t k = int64_t(z) * sz + x;
        a.out1[k] = qz[R];
        a.out2[k] = pnew;
      }
    }
  }
}

}  // namespace sw
