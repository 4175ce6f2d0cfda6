// Source injection, receiver sampling and model set-up kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "layout.h"

namespace sw {

struct PointSet {
  const int* first;  // [count][3] first window node per axis (z, y, x)
  const float* w;    // [count][3][L] per-axis weights (y: single 1 in 2D)
  int count;
  int L;             // row length of w
  int lz, ly, lx;    // window lengths per axis
};

struct FaceInfo {
  int64_t sz, sy;
  int nz, ny, nx;
  int nbl[6];
  int bc[6];
};

__device__ __forceinline__ int face_distance(int i, int n, int lo, int hi) {
  return max(max(lo - i, i - (n - 1 - hi)), 0);
}

__device__ __forceinline__ void add_with_mirrors(float* p, int64_t idx, int i, int n, int64_t stride,
                                                 int bc_lo, int bc_hi, int R, float d) {
  if (bc_lo != kBcNone && i >= 1 && i <= R)
    atomicAdd(&p[idx - int64_t(2 * i) * stride], bc_lo == kBcDirichlet ? -d : d);
  const int m = n - 1 - i;
  if (bc_hi != kBcNone && m >= 1 && m <= R)
    atomicAdd(&p[idx + int64_t(2 * m) * stride], bc_hi == kBcDirichlet ? -d : d);
}

// Eq. 11: p[n+1]_k += kappa_k a_k S_s(t_n) d_k / prod(h) for every window node
// of every source (1/prod(h) is folded into the x weights).  The ghost images
// of nodes near mirrored faces get the same increment (with the face's sign),
// so the ghost layer stays consistent with p[n+1].  Dirichlet face nodes stay 0.
__global__ void inject_sources_kernel(float* p, const float* kappa, const float2* damp, PointSet src,
                                      const float* sig, int sig_stride, int step, FaceInfo f, int ndim,
                                      int R) {
  const int taps = src.lz * src.ly * src.lx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= src.count * taps) return;
  const int s = t / taps;
  int rem = t % taps;
  const int ix = rem % src.lx;
  rem /= src.lx;
  const int iy = rem % src.ly;
  const int iz = rem / src.ly;
  const float* w = src.w + int64_t(s) * 3 * src.L;
  const float wgt = w[iz] * w[src.L + iy] * w[2 * src.L + ix];
  if (wgt == 0.f) return;
  const int z = src.first[3 * s] + iz;
  const int y = src.first[3 * s + 1] + iy;
  const int x = src.first[3 * s + 2] + ix;
  const bool dir = (z == 0 && f.bc[0] == kBcDirichlet) || (z == f.nz - 1 && f.bc[1] == kBcDirichlet) ||
                   (x == 0 && f.bc[4] == kBcDirichlet) || (x == f.nx - 1 && f.bc[5] == kBcDirichlet) ||
                   (ndim == 3 && ((y == 0 && f.bc[2] == kBcDirichlet) ||
                                  (y == f.ny - 1 && f.bc[3] == kBcDirichlet)));
  if (dir) return;
  const int64_t idx = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
  const int dz = face_distance(z, f.nz, f.nbl[0], f.nbl[1]);
  const int dy = ndim == 3 ? face_distance(y, f.ny, f.nbl[2], f.nbl[3]) : 0;
  const int dx = face_distance(x, f.nx, f.nbl[4], f.nbl[5]);
  const int d2 = dz * dz + dy * dy + dx * dx;
  const float ca = d2 ? damp[d2].x : 1.f;
  const float d = kappa[idx] * ca * wgt * sig[int64_t(s) * sig_stride + step];
  atomicAdd(&p[idx], d);
  add_with_mirrors(p, idx, z, f.nz, f.sz, f.bc[0], f.bc[1], R, d);
  add_with_mirrors(p, idx, x, f.nx, 1, f.bc[4], f.bc[5], R, d);
  if (ndim == 3) add_with_mirrors(p, idx, y, f.ny, f.sy, f.bc[2], f.bc[3], R, d);
}

// Eq. 12: rec[step][r] = sum_k d_k p[n+1]_k.  One warp per receiver.
__global__ void sample_receivers_kernel(const float* p, PointSet rec, FaceInfo f, float* out, int step) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= rec.count) return;
  const int taps = rec.lz * rec.ly * rec.lx;
  const float* w = rec.w + int64_t(warp) * 3 * rec.L;
  const int z0 = rec.first[3 * warp], y0 = rec.first[3 * warp + 1], x0 = rec.first[3 * warp + 2];
  float acc = 0.f;
  for (int t = lane; t < taps; t += 32) {
    int rem = t;
    const int ix = rem % rec.lx;
    rem /= rec.lx;
    const int iy = rem % rec.ly;
    const int iz = rem / rec.ly;
    const float wgt = w[iz] * w[rec.L + iy] * w[2 * rec.L + ix];
    acc = fmaf(wgt, p[int64_t(z0 + iz) * f.sz + int64_t(y0 + iy) * f.sy + (x0 + ix)], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[int64_t(step) * rec.count + warp] = acc;
}

// ---- model set-up -----------------------------------------------------------

// Maximum and minimum of a positive field through the float bit pattern
// (order-preserving for non-negative floats); flags non-finite or <= 0 values.
__global__ void field_range_kernel(const float* v, int64_t n, unsigned* vmax, unsigned* vmin, int* bad) {
  unsigned lmax = 0u, lmin = 0x7f800000u;
  int lbad = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float x = v[i];
    if (!(x > 0.f) || !(x < 3.0e38f)) lbad = 1;
    const unsigned b = __float_as_uint(x);
    lmax = max(lmax, b);
    lmin = min(lmin, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    lbad |= __shfl_xor_sync(0xffffffffu, lbad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(vmax, lmax);
    atomicMin(vmin, lmin);
    if (lbad) atomicOr(bad, 1);
  }
}

// kappa = (c dt)^2 written into the padded layout (node origin pointer).
__global__ void kappa_kernel(const float* vel, float* kappa, FaceInfo f, double dt) {
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    const double c = double(vel[i]) * dt;
    kappa[int64_t(z) * f.sz + int64_t(y) * f.sy + x] = float(c * c);
  }
}

// ln(rho) into the padded layout.
__global__ void lnrho_kernel(const float* rho, float* lr, FaceInfo f) {
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    lr[int64_t(z) * f.sz + int64_t(y) * f.sy + x] = float(log(double(rho[i])));
  }
}

// Even mirror of a padded field into its R ghost layers along one axis
// (axis 0 = z, 1 = y, 2 = x), over the node range of the two other axes.
__global__ void mirror_even_kernel(float* f_, FaceInfo f, int axis, int R) {
  const int n[3] = {f.nz, f.ny, f.nx};
  const int64_t st[3] = {f.sz, f.sy, 1};
  const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
  const int64_t face = int64_t(n[o1]) * n[o2];
  const int64_t total = face * 2 * R;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = t % face;
    const int k = int(t / face);  // 0..2R-1
    const int side = k / R;
    const int j = k % R + 1;
    const int i1 = int(e / n[o2]), i2 = int(e % n[o2]);
    const int g = side == 0 ? -j : n[axis] - 1 + j;
    const int m = side == 0 ? j : n[axis] - 1 - j;
    const int64_t base = int64_t(i1) * st[o1] + int64_t(i2) * st[o2];
    f_[base + int64_t(g) * st[axis]] = f_[base + int64_t(m) * st[axis]];
  }
}

// Dense copy of the nodes of a padded field.
__global__ void extract_kernel(const float* p, float* out, FaceInfo f) {
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    out[i] = p[int64_t(z) * f.sz + int64_t(y) * f.sy + x];
  }
}

}  // namespace sw
