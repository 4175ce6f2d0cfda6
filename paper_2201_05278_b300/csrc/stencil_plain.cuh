// Leapfrog stencil step, shared-memory plane + register z-queue version.
//
// One CTA owns a TX x TY column of the grid (TX x 1 in 2D) and marches along z
// over a chunk of planes.  Each thread keeps the 2R+1 values of p[n] it needs
// along z in registers (a queue shifted once per plane) and takes the in-plane
// neighbours from a shared-memory copy of the current plane with an R-wide
// halo.  p[n-1] and kappa are read once per node; p[n+1] overwrites p[n-1].
//
// Per node (Sec. 2.2, Eq. 7 with every term divided by 1 + eta dt):
//   p[n+1] = a (p[n] + kappa L p[n] + (p[n] - p[n-1]) + e p[n-1]),  a = 1/(1+e)
//   L = sum_axes h^-2 sum_j v_j ((p+j + p-j) - 2p)   (Eq. 9, v0 = -2 sum_j v_j)
//       - sum_axes D(ln rho) D(p),  D = (2h)^-1 sum_j w_j (.+j - .-j) (Eq. 10)
// e = alpha d^p dt from a table indexed by the squared cell distance to the
// physical domain (Eq. 4).  Face conditions are kept in ghost nodes: the
// thread that writes a node within R of a mirrored face also writes its
// mirror image into the ghost layer of p[n+1]; Dirichlet face nodes are 0.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "layout.h"
#include "tma.cuh"

namespace sw {

struct StencilArgs {
  const float* pn;      // p[n] at node (0,0,0) of the padded layout
  const float* pnm1;    // p[n-1]
  float* pout;          // p[n+1] (== pnm1 for the in-place update of the time loop)
  const float* kappa;   // (c dt)^2
  const float* lnrho;   // ln(rho) with mirrored ghosts, or nullptr
  const float2* damp;   // (a, e) = (1/(1+eta dt), eta dt) by squared distance (cells^2)
  int64_t sz, sy;
  int nz, ny, nx;
  int nbl[6];
  int bc[6];
  int zchunk;
  float cz[kMaxR + 1], cy[kMaxR + 1], cx[kMaxR + 1];  // v_j / h^2
  float gz[kMaxR + 1], gy[kMaxR + 1], gx[kMaxR + 1];  // w_j / (2h)
};

__device__ __forceinline__ int layer_distance(int i, int n, int lo, int hi) {
  return max(max(lo - i, i - (n - 1 - hi)), 0);
}

// Writes the face-mirror images of a freshly computed node value into the
// ghost layers of p[n+1] along one axis.  `i` is the node index along the
// axis, `n` its length, `stride` the axis stride.
template <int R>
__device__ __forceinline__ void mirror_ghosts(float* p, int64_t idx, int i, int n, int64_t stride,
                                              int bc_lo, int bc_hi, float v) {
  if (bc_lo != kBcNone && i >= 1 && i <= R)
    p[idx - int64_t(2 * i) * stride] = (bc_lo == kBcDirichlet) ? -v : v;
  const int m = n - 1 - i;  // distance to the high face node
  if (bc_hi != kBcNone && m >= 1 && m <= R)
    p[idx + int64_t(2 * m) * stride] = (bc_hi == kBcDirichlet) ? -v : v;
}

template <int R, int NDIM, bool VD, int TX, int TY, int PPT>
__global__ void __launch_bounds__(TX*(TY / PPT)) stencil_plain_kernel(const StencilArgs a) {
  constexpr int NT = TX * (TY / PPT);
  constexpr int SW = TX + 2 * R;
  constexpr int SH = (NDIM == 3) ? TY + 2 * R : 1;
  __shared__ float sp[SH][SW];
  __shared__ float sl[VD ? SH : 1][VD ? SW : 1];

  const int tid = threadIdx.x;
  const int tx = tid % TX;
  const int ty = tid / TX;
  const int x0 = blockIdx.x * TX;
  const int y0 = (NDIM == 3) ? blockIdx.y * TY : 0;
  const int zb = blockIdx.z * a.zchunk;
  const int ze = min(zb + a.zchunk, a.nz);
  const int x = x0 + tx;
  const int64_t sz = a.sz, sy = a.sy;

  int yrow[PPT];
  int64_t col[PPT];  // offset of (0, y, x) for each of the thread's rows
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    yrow[i] = (NDIM == 3) ? y0 + ty * PPT + i : 0;
    col[i] = int64_t(yrow[i]) * sy + x;
  }

  float q[PPT][2 * R + 1];
  float ql[VD ? PPT : 1][VD ? 2 * R + 1 : 1];
#pragma unroll
  for (int k = 0; k < 2 * R; ++k) {
    const int64_t zoff = int64_t(zb - R + k) * sz;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      q[i][k + 1] = a.pn[zoff + col[i]];
      if constexpr (VD) ql[i][k + 1] = a.lnrho[zoff + col[i]];
    }
  }

  for (int z = zb; z < ze; ++z) {
    const int64_t zoff = int64_t(z) * sz;
    const int64_t zf = int64_t(z + R) * sz;
    float po[PPT], kp[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
#pragma unroll
      for (int k = 0; k < 2 * R; ++k) q[i][k] = q[i][k + 1];
      q[i][2 * R] = a.pn[zf + col[i]];
      if constexpr (VD) {
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) ql[i][k] = ql[i][k + 1];
        ql[i][2 * R] = a.lnrho[zf + col[i]];
      }
      po[i] = a.pnm1[zoff + col[i]];
      kp[i] = a.kappa[zoff + col[i]];
    }

    __syncthreads();  // the previous plane's readers are done with sp / sl
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int row = (NDIM == 3) ? ty * PPT + i + R : 0;
      sp[row][tx + R] = q[i][R];
      if constexpr (VD) sl[row][tx + R] = ql[i][R];
    }
    // x halo: R columns on each side of every row of the tile
    for (int e = tid; e < (NDIM == 3 ? TY : 1) * 2 * R; e += NT) {
      const int r = e / (2 * R);
      const int c = e % (2 * R);
      const int scol = (c < R) ? c : TX + c;
      const int gxx = x0 - R + scol;
      const int64_t off = zoff + int64_t((NDIM == 3) ? y0 + r : 0) * sy + gxx;
      const int srow = (NDIM == 3) ? r + R : 0;
      sp[srow][scol] = a.pn[off];
      if constexpr (VD) sl[srow][scol] = a.lnrho[off];
    }
    if constexpr (NDIM == 3) {
      // y halo: R rows above and below, TX columns
      for (int e = tid; e < 2 * R * TX; e += NT) {
        const int r = e / TX;
        const int c = e % TX;
        const int srow = (r < R) ? r : TY + r;
        const int gyy = y0 - R + srow;
        const int64_t off = zoff + int64_t(gyy) * sy + x0 + c;
        sp[srow][c + R] = a.pn[off];
        if constexpr (VD) sl[srow][c + R] = a.lnrho[off];
      }
    }
    __syncthreads();

#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int row = (NDIM == 3) ? ty * PPT + i + R : 0;
      const float pc = q[i][R];
      const float p2 = 2.f * pc;
      // sum_j c_j ((p+j + p-j) - 2p): the FP32 operator annihilates constants exactly
      // (a separate v0 p term would leave the FP32 rounding of sum(v) as a spurious
      // mass term that shifts the phase of long runs).
      float lap = 0.f;
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        lap = fmaf(a.cz[j], (q[i][R + j] + q[i][R - j]) - p2, lap);
        lap = fmaf(a.cx[j], (sp[row][tx + R + j] + sp[row][tx + R - j]) - p2, lap);
        if constexpr (NDIM == 3) lap = fmaf(a.cy[j], (sp[row + j][tx + R] + sp[row - j][tx + R]) - p2, lap);
      }
      if constexpr (VD) {
        float dpz = 0.f, dlz = 0.f, dpx = 0.f, dlx = 0.f, dpy = 0.f, dly = 0.f;
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          dpz = fmaf(a.gz[j], q[i][R + j] - q[i][R - j], dpz);
          dlz = fmaf(a.gz[j], ql[i][R + j] - ql[i][R - j], dlz);
          dpx = fmaf(a.gx[j], sp[row][tx + R + j] - sp[row][tx + R - j], dpx);
          dlx = fmaf(a.gx[j], sl[row][tx + R + j] - sl[row][tx + R - j], dlx);
          if constexpr (NDIM == 3) {
            dpy = fmaf(a.gy[j], sp[row + j][tx + R] - sp[row - j][tx + R], dpy);
            dly = fmaf(a.gy[j], sl[row + j][tx + R] - sl[row - j][tx + R], dly);
          }
        }
        float adv = dlz * dpz + dlx * dpx;
        if constexpr (NDIM == 3) adv = fmaf(dly, dpy, adv);
        lap -= adv;
      }
      const int y = yrow[i];
      if (x < a.nx && y < a.ny) {
        const int dz = layer_distance(z, a.nz, a.nbl[0], a.nbl[1]);
        const int dy = (NDIM == 3) ? layer_distance(y, a.ny, a.nbl[2], a.nbl[3]) : 0;
        const int dx = layer_distance(x, a.nx, a.nbl[4], a.nbl[5]);
        const int d2 = dz * dz + dy * dy + dx * dx;
        float ca = 1.f, e = 0.f;
        if (d2 != 0) {
          const float2 c = __ldg(&a.damp[d2]);
          ca = c.x;
          e = c.y;
        }
        // (1+e) p[n+1] = kappa L + 2p - (1-e) p[n-1], evaluated as
        // p[n+1] = a (p + (kappa L + (p - p[n-1]) + e p[n-1])): p - p[n-1] is small and
        // (for a smooth field) exact, so only the last add rounds at the scale of p.
        const float dp = pc - po[i];
        float pnew = ca * (pc + fmaf(kp[i], lap, fmaf(e, po[i], dp)));
        const bool dir = (z == 0 && a.bc[0] == kBcDirichlet) || (z == a.nz - 1 && a.bc[1] == kBcDirichlet) ||
                         (x == 0 && a.bc[4] == kBcDirichlet) || (x == a.nx - 1 && a.bc[5] == kBcDirichlet) ||
                         (NDIM == 3 && ((y == 0 && a.bc[2] == kBcDirichlet) ||
                                        (y == a.ny - 1 && a.bc[3] == kBcDirichlet)));
        if (dir) pnew = 0.f;
        const int64_t idx = zoff + col[i];
        a.pout[idx] = pnew;
        mirror_ghosts<R>(a.pout, idx, z, a.nz, sz, a.bc[0], a.bc[1], pnew);
        mirror_ghosts<R>(a.pout, idx, x, a.nx, 1, a.bc[4], a.bc[5], pnew);
        if constexpr (NDIM == 3) mirror_ghosts<R>(a.pout, idx, y, a.ny, sy, a.bc[2], a.bc[3], pnew);
      }
    }
  }
}

// 2D: one thread per node, every neighbour read from global memory (the
// fields of a 2D grid are a few MB and stay in L2; marching along z with a
// shared plane would leave most SMs idle on such grids).  Same arithmetic
// and face handling as stencil_plain_kernel; one block row of 128 nodes
// per (x tile, z) pair.
// Eq. 9 in 2D from the 2R+1 values along z and along x around a node (centre
// at index R), each pair as (p[+j] + p[-j]) - 2p.
template <int R>
__device__ __forceinline__ float laplacian_2d(const float* qz, const float* qx, const float* cz, const float* cx) {
  const float p2 = 2.f * qz[R];
  float lap = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    lap = fmaf(cz[j], (qz[R + j] + qz[R - j]) - p2, lap);
    lap = fmaf(cx[j], (qx[R + j] + qx[R - j]) - p2, lap);
  }
  return lap;
}

// Eq. 7 divided by (1 + e): p[n+1] = a (p + (kappa L + (p - p[n-1]) + e p[n-1])).
__device__ __forceinline__ float leapfrog_update(float pc, float po, float kp, float lap, float ca, float e) {
  return ca * (pc + fmaf(kp, lap, fmaf(e, po, pc - po)));
}

template <int R, bool VD>
__device__ __forceinline__ void stencil_2d_node(const StencilArgs& a, int z, int x) {
  const int64_t sz = a.sz;
  const int64_t idx = int64_t(z) * sz + x;
  const float* p = a.pn;
  float qz[2 * R + 1], qx[2 * R + 1];
#pragma unroll
  for (int j = -R; j <= R; ++j) {
    qz[j + R] = __ldg(&p[idx + j * sz]);
    qx[j + R] = __ldg(&p[idx + j]);
  }
  const float po = a.pnm1[idx];
  const float kp = __ldg(&a.kappa[idx]);
  const float pc = qz[R];
  float lap = laplacian_2d<R>(qz, qx, a.cz, a.cx);
  if constexpr (VD) {
    const float* l = a.lnrho;
    float dpz = 0.f, dlz = 0.f, dpx = 0.f, dlx = 0.f;
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      dpz = fmaf(a.gz[j], qz[R + j] - qz[R - j], dpz);
      dlz = fmaf(a.gz[j], __ldg(&l[idx + j * sz]) - __ldg(&l[idx - j * sz]), dlz);
      dpx = fmaf(a.gx[j], qx[R + j] - qx[R - j], dpx);
      dlx = fmaf(a.gx[j], __ldg(&l[idx + j]) - __ldg(&l[idx - j]), dlx);
    }
    lap -= dlz * dpz + dlx * dpx;
  }
  const int dz = layer_distance(z, a.nz, a.nbl[0], a.nbl[1]);
  const int dx = layer_distance(x, a.nx, a.nbl[4], a.nbl[5]);
  const int d2 = dz * dz + dx * dx;
  float ca = 1.f, e = 0.f;
  if (d2 != 0) {
    const float2 c = __ldg(&a.damp[d2]);
    ca = c.x;
    e = c.y;
  }
  float pnew = leapfrog_update(pc, po, kp, lap, ca, e);
  const bool dir = (z == 0 && a.bc[0] == kBcDirichlet) || (z == a.nz - 1 && a.bc[1] == kBcDirichlet) ||
                   (x == 0 && a.bc[4] == kBcDirichlet) || (x == a.nx - 1 && a.bc[5] == kBcDirichlet);
  if (dir) pnew = 0.f;
  a.pout[idx] = pnew;
  mirror_ghosts<R>(a.pout, idx, z, a.nz, sz, a.bc[0], a.bc[1], pnew);
  mirror_ghosts<R>(a.pout, idx, x, a.nx, 1, a.bc[4], a.bc[5], pnew);
}

template <int R, bool VD>
__global__ void __launch_bounds__(128) stencil_2d_kernel(const StencilArgs a) {
  // may be launched as a programmatic dependent of the previous step's last
  // kernel: wait for it before touching the fields
  griddep_launch_dependents();
  griddep_wait();
  const int x = blockIdx.x * 128 + threadIdx.x;
  if (x >= a.nx) return;
  for (int z = blockIdx.y; z < a.nz; z += gridDim.y) stencil_2d_node<R, VD>(a, z, x);
}

}  // namespace sw
