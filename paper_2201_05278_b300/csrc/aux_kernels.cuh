// Source injection, receiver sampling and model set-up kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "layout.h"
#include "tma.cuh"

namespace sw {

struct PointSet {
  const int* first;  // [count][3] first window node per axis (z, y, x)
  const float* w;    // [count][3][L] per-axis weights (y: single 1 in 2D)
  int count;
  int L;             // row length of w
  int lz, ly, lx;    // window lengths per axis
  const int4* span;  // optional [count]: (first row, rows) along z and y with non-zero weight
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
__device__ __forceinline__ void inject_source_node(float* p, const float* kappa, const float2* damp,
                                                   const PointSet& src, const float* sig, int sig_stride, int step,
                                                   const FaceInfo& f, int ndim, int R, int s, int iz, int iy, int ix) {
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

__device__ __forceinline__ void inject_source_tap(float* p, const float* kappa, const float2* damp,
                                                  const PointSet& src, const float* sig, int sig_stride, int step,
                                                  const FaceInfo& f, int ndim, int R, int t) {
  const int taps = src.lz * src.ly * src.lx;
  if (t >= src.count * taps) return;
  const int s = t / taps;
  int rem = t % taps;
  const int ix = rem % src.lx;
  rem /= src.lx;
  const int iy = rem % src.ly;
  const int iz = rem / src.ly;
  inject_source_node(p, kappa, damp, src, sig, sig_stride, step, f, ndim, R, s, iz, iy, ix);
}

// The same increments over only the window rows with a non-zero weight along
// z and y (src.span set; max_rows = the largest such row count): one thread
// per (point, row, column).
__device__ __forceinline__ void inject_row_node(float* p, const float* kappa, const float2* damp, const PointSet& src,
                                                int max_rows, const float* sig, int sig_stride, int step,
                                                const FaceInfo& f, int ndim, int R, int t) {
  const int per = max_rows * src.lx;
  if (t >= src.count * per) return;
  const int s = t / per;
  const int rem = t - s * per;
  const int row = rem / src.lx, ix = rem - (rem / src.lx) * src.lx;
  const int4 sp = src.span[s];
  if (row >= sp.y * sp.w) return;
  inject_source_node(p, kappa, damp, src, sig, sig_stride, step, f, ndim, R, s, sp.x + row / sp.w, sp.z + row % sp.w,
                     ix);
}


__global__ void inject_sources_kernel(float* p, const float* kappa, const float2* damp, PointSet src,
                                      const float* sig, int sig_stride, int step, FaceInfo f, int ndim,
                                      int R) {
  griddep_launch_dependents();
  griddep_wait();  // p[n+1] of the stencil launched before (when launched as its dependent)
  inject_source_tap(p, kappa, damp, src, sig, sig_stride, step, f, ndim, R, blockIdx.x * blockDim.x + threadIdx.x);
}

// Tap table of the sources for the pipelined path, built once per forward
// run: for every window node the offset of the node and kappa_k a_k d_k /
// prod(h), the step-independent part of the Eq. 11 increment, as
// inject_sources_kernel forms it.  Dirichlet face nodes get offset -1 (never
// incremented).  No ghost images: the face conditions follow the injection.
// With tap_pre, also the coefficients of the pre-injection (PreInject).
__global__ void source_taps_kernel(const float* kappa, const float2* damp, PointSet src, FaceInfo f,
                                   int64_t* tap_off, float* tap_coef, float* tap_pre) {
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
  const int z = src.first[3 * s] + iz, y = src.first[3 * s + 1] + iy, x = src.first[3 * s + 2] + ix;
  const bool dir = (z == 0 && f.bc[0] == kBcDirichlet) || (z == f.nz - 1 && f.bc[1] == kBcDirichlet) ||
                   (y == 0 && f.bc[2] == kBcDirichlet) || (y == f.ny - 1 && f.bc[3] == kBcDirichlet) ||
                   (x == 0 && f.bc[4] == kBcDirichlet) || (x == f.nx - 1 && f.bc[5] == kBcDirichlet);
  const int64_t idx = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
  const int dz = face_distance(z, f.nz, f.nbl[0], f.nbl[1]);
  const int dy = face_distance(y, f.ny, f.nbl[2], f.nbl[3]);
  const int dx = face_distance(x, f.nx, f.nbl[4], f.nbl[5]);
  const int d2 = dz * dz + dy * dy + dx * dx;
  const float ca = d2 ? damp[d2].x : 1.f;
  const float e = d2 ? damp[d2].y : 0.f;
  tap_off[t] = (dir || wgt == 0.f) ? -1 : idx;
  tap_coef[t] = kappa[idx] * ca * wgt;
  if (tap_pre) tap_pre[t] = -(kappa[idx] * wgt) / (1.f - e);  // see PreInject (used where e < 1/2 at every tap)
}

// Eq. 11 from the tap table: p[n+1]_k += coef_k S_s(t_n), one thread per tap.
__global__ void inject_taps_kernel(float* p, const int64_t* tap_off, const float* tap_coef, int taps, int count,
                                   const float* sig, int sig_stride, int step) {
  griddep_launch_dependents();
  griddep_wait();  // p[n+1] of the stencil launched before
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count * taps) return;
  const int64_t k = tap_off[t];
  if (k < 0) return;
  atomicAdd(&p[k], tap_coef[t] * sig[int64_t(t / taps) * sig_stride + step]);
}

// Eq. 12: rec[step][r] = sum_k d_k p[n+1]_k, receiver r by one warp: lanes
// run along x within a window row (lx <= 32 lanes per row, 32 / lx rows per
// pass), so each load instruction reads a few contiguous row pieces, and the
// row loop is unrolled so that several loads are in flight per lane.  With
// `dirichlet_zero` a node on a Dirichlet face counts as zero whatever is
// stored there (for sampling while the face conditions are being applied).
__device__ __forceinline__ void sample_receiver(const float* p, const PointSet& rec, const FaceInfo& f, float* out,
                                                int step, int r, int lane, bool dirichlet_zero) {
  const float* w = rec.w + int64_t(r) * 3 * rec.L;
  // only the window rows with a non-zero weight along z and y contribute (a
  // receiver on a grid plane has a single one along that axis)
  int za = 0, lz = rec.lz, ya = 0, ly = rec.ly;
  if (rec.span) {
    const int4 sp = rec.span[r];
    za = sp.x;
    lz = sp.y;
    ya = sp.z;
    ly = sp.w;
  }
  const int z0 = rec.first[3 * r] + za, y0 = rec.first[3 * r + 1] + ya, x0 = rec.first[3 * r + 2];
  const float* wz = w + za;
  const float* wy = w + rec.L + ya;
  const int rows = lz * ly, rpp = 32 / rec.lx;
  const int ix = lane % rec.lx, rs = lane / rec.lx;
  float acc = 0.f;
  if (rs < rows && rs < rpp) {
    const int x = x0 + ix;
    const bool xd = dirichlet_zero && ((x == 0 && f.bc[4] == kBcDirichlet) || (x == f.nx - 1 && f.bc[5] == kBcDirichlet));
    // window rows rs, rs + rpp, ... as (iz, iy), stepped without divisions
    const int dz = rpp / ly, dy = rpp - dz * ly;
    int iz = rs / ly, iy = rs - (rs / ly) * ly;
    const float* q = p + int64_t(z0) * f.sz + int64_t(y0) * f.sy + x;
    float s = 0.f;
#pragma unroll 4
    while (iz < lz) {
      float v = q[int64_t(iz) * f.sz + int64_t(iy) * f.sy];
      if (dirichlet_zero) {
        const int z = z0 + iz, y = y0 + iy;
        if (xd || (z == 0 && f.bc[0] == kBcDirichlet) || (z == f.nz - 1 && f.bc[1] == kBcDirichlet) ||
            (y == 0 && f.bc[2] == kBcDirichlet) || (y == f.ny - 1 && f.bc[3] == kBcDirichlet))
          v = 0.f;
      }
      s = fmaf(wz[iz] * wy[iy], v, s);
      iz += dz;
      iy += dy;
      if (iy >= ly) {
        iy -= ly;
        ++iz;
      }
    }
    acc = w[2 * rec.L + ix] * s;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[int64_t(step) * rec.count + r] = acc;
}

// Eq. 12 with several receivers per warp, for windows of at most 32 columns
// (lx): a group of G lanes (lx rounded up to a power of two) per receiver,
// lane i of the group on window column i, the window rows (those with a
// non-zero weight along z and y) summed in turn, then the group's lanes
// reduced.  2D grids use it on both the single-grid and the batched path.
__device__ __forceinline__ void sample_receivers_grouped(const float* p, const PointSet& rec, const FaceInfo& f,
                                                         float* out, int step, int warp, int lane) {
  const int G = rec.lx <= 8 ? 8 : (rec.lx <= 16 ? 16 : 32);
  const int r = warp * (32 / G) + lane / G;
  const int ix = lane % G;
  float acc = 0.f;
  if (r < rec.count && ix < rec.lx) {
    const float* w = rec.w + int64_t(r) * 3 * rec.L;
    int za = 0, lz = rec.lz, ya = 0, ly = rec.ly;
    if (rec.span) {
      const int4 sp = rec.span[r];
      za = sp.x;
      lz = sp.y;
      ya = sp.z;
      ly = sp.w;
    }
    const float* q = p + int64_t(rec.first[3 * r] + za) * f.sz + int64_t(rec.first[3 * r + 1] + ya) * f.sy +
                     (rec.first[3 * r + 2] + ix);
    float s = 0.f;
    for (int iz = 0; iz < lz; ++iz)
      for (int iy = 0; iy < ly; ++iy)
        s = fmaf(w[za + iz] * w[rec.L + ya + iy], q[int64_t(iz) * f.sz + int64_t(iy) * f.sy], s);
    acc = w[2 * rec.L + ix] * s;
  }
  for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (r < rec.count && ix == 0) out[int64_t(step) * rec.count + r] = acc;
}

__global__ void sample_receivers_grouped_kernel(const float* p, PointSet rec, FaceInfo f, float* out, int step) {
  griddep_launch_dependents();
  griddep_wait();  // the level it samples (when launched as a dependent)
  sample_receivers_grouped(p, rec, f, out, step, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31);
}

__host__ __device__ inline int grouped_receiver_warps(const PointSet& rec) {
  const int per = rec.lx <= 8 ? 4 : (rec.lx <= 16 ? 2 : 1);
  return (rec.count + per - 1) / per;
}

__global__ void sample_receivers_kernel(const float* p, PointSet rec, FaceInfo f, float* out, int step) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= rec.count) return;
  sample_receiver(p, rec, f, out, step, warp, threadIdx.x & 31, false);
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

// First-derivative weights w_j / (2 h) per axis (FP64), for the ln(rho)
// gradient fields of the pipelined variable-density stencil.
struct GradWeights {
  double z[kMaxR + 1], y[kMaxR + 1], x[kMaxR + 1];
};

// g_axis = D_axis ln(rho) = sum_j w_j / (2 h) (lnrho(+j) - lnrho(-j)) (Eq. 10)
// at every node of a 3D grid, from ln(rho) with its even-mirrored ghosts,
// summed in FP64 and stored in FP32 in the padded layout.  Computed once per
// model; the pipelined stencil then reads the three gradients instead of
// differentiating ln(rho) every step.
__global__ void lnrho_gradient_kernel(const float* lr, float* gz, float* gy, float* gx, FaceInfo f, GradWeights w,
                                      int R) {
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    const int64_t k = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
    double dz = 0.0, dy = 0.0, dx = 0.0;
    for (int j = 1; j <= R; ++j) {
      dz += w.z[j] * (double(lr[k + j * f.sz]) - double(lr[k - j * f.sz]));
      dy += w.y[j] * (double(lr[k + j * f.sy]) - double(lr[k - j * f.sy]));
      dx += w.x[j] * (double(lr[k + j]) - double(lr[k - j]));
    }
    gz[k] = float(dz);
    gy[k] = float(dy);
    gx[k] = float(dx);
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

// Face conditions of a freshly computed 3D p[n+1], for the pipelined stencil
// kernel, which writes node values only (Sec. 2.3): nodes on a Dirichlet face
// are set to zero, and every node within R of a Dirichlet (odd) or Neumann
// (even) face gets its mirror image in that face's ghost layer; a node on any
// Dirichlet face is mirrored as zero.  z and y faces: one thread per (side,
// position on the face), consecutive threads at consecutive x, walking the R
// nodes next to the face; a block covers 256 consecutive x of one line of
// the face, so a thread finds its position without a division.  x faces:
// kFaceLanes lanes per row, lane l writing ghost column l + 1 of its side, so
// that each row's ghosts go out as one whole 32- or 64-byte run; the columns
// past R get zeros (nothing reads them: the stencils use R ghost columns, and
// the x pad holds zeros there from the allocation on).  Ghost layers of
// different axes are disjoint, and a node read for mirroring while another
// thread zeroes it is taken as zero either way.  Needs every axis longer than
// 2R+1 (a node is within R of one face only).
template <int AX, int R>
__device__ __forceinline__ void face_line(float* p, const FaceInfo& f, int side, int ia, int ib) {
  // ia: position along the slower axis spanning the face (y for z faces, z
  // for y faces), ib: x
  const int n = AX == 0 ? f.nz : f.ny;
  const int64_t sa = AX == 0 ? f.sy : f.sz;
  const int64_t s = AX == 0 ? f.sz : f.sy;
  const int bc = side ? f.bc[2 * AX + 1] : f.bc[2 * AX];
  if (bc == kBcNone) return;
  // is the line on a Dirichlet face of another axis? (then every node of it is zero)
  const int cz = AX == 1 ? ia : 0, cy = AX == 0 ? ia : 0;
  const bool zero = (AX != 0 && ((cz == 0 && f.bc[0] == kBcDirichlet) || (cz == f.nz - 1 && f.bc[1] == kBcDirichlet))) ||
                    (AX != 1 && ((cy == 0 && f.bc[2] == kBcDirichlet) || (cy == f.ny - 1 && f.bc[3] == kBcDirichlet))) ||
                    ((ib == 0 && f.bc[4] == kBcDirichlet) || (ib == f.nx - 1 && f.bc[5] == kBcDirichlet));
  float* q = p + ia * sa + ib + (side ? int64_t(n - 1) * s : 0);  // the face node
  const int64_t in = side ? -s : s;                                // inwards
  const float sign = (bc == kBcDirichlet) ? -1.f : 1.f;
  float v[R + 1];
#pragma unroll
  for (int j = 1; j <= R; ++j) v[j] = q[j * in];
  if (bc == kBcDirichlet || zero) q[0] = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j) q[-j * in] = zero ? 0.f : sign * v[j];
}

template <int R>
constexpr int face_lanes() { return R <= 8 ? 8 : 16; }

// Ghost column j (1 .. face_lanes<R>()) of the row (side, z, y) on an x face.
template <int R>
__device__ __forceinline__ void face_x(float* p, const FaceInfo& f, int side, int z, int y, int j) {
  const int bc = side ? f.bc[5] : f.bc[4];
  if (bc == kBcNone) return;
  const bool zero = (z == 0 && f.bc[0] == kBcDirichlet) || (z == f.nz - 1 && f.bc[1] == kBcDirichlet) ||
                    (y == 0 && f.bc[2] == kBcDirichlet) || (y == f.ny - 1 && f.bc[3] == kBcDirichlet);
  float* q = p + int64_t(z) * f.sz + int64_t(y) * f.sy + (side ? f.nx - 1 : 0);  // the face node
  const int in = side ? -1 : 1;
  float v = 0.f;
  if (j <= R && !zero) {
    v = q[j * in];
    if (bc == kBcDirichlet) v = -v;
  }
  q[-j * in] = v;
  if (j == 1 && (bc == kBcDirichlet || zero)) q[0] = 0.f;
}

// One launch per step after the pipelined stencil: the receiver samples of
// the step (Eq. 12; receiver windows hold nodes only, and Dirichlet face
// nodes are read as zero) and the face conditions.  The 1D grid is cut into
// consecutive block ranges: receivers (8 per block) first, so that their
// longer load chains start early, then z faces, y faces and x faces.
struct FaceGrid {
  int rec, z, y, x, pre;  // blocks per part
  int bxz;                // blocks per face line along x (z and y faces)
  int bxx;                // blocks per z plane of an x face
  int flat = 0;           // z, y and x faces numbered across lines (small faces: no idle lanes per line)
  int total() const { return rec + z + y + x + pre; }
};

// Source injection of the next step, applied to the level it reads as
// p[n-1]: the update reads p[n-1] at the node only, through
// p[n+1] = a (2 p - (1 - e) p[n-1] + kappa L), so adding
// d = kappa_k d_k S(t) / (1 - e_k) there before the step adds
// kappa_k a_k d_k S(t) to p[n+1]_k, the Eq. 11 term, up to rounding.
// `coef` holds -kappa_k d_k / (1 - e_k) (tap table order, offsets as the
// tap table's); count = 0: nothing to do.
struct PreInject {
  float* p;  // the level stored as p[n-1] of the next step (node values)
  const int64_t* off;
  const float* coef;
  const float* sig;
  int taps, count, sig_stride, step;
};

// Block b of the face launch of one grid (the parts in the order of FaceGrid).
template <int R>
__device__ __forceinline__ void face_block(float* p, const FaceInfo& f, const PointSet& rec, float* out, int step,
                                           const FaceGrid& fg, const PreInject& pi, int b) {
  if (b < fg.pre) {  // a different level from the one the other parts touch
    const int t = b * blockDim.x + threadIdx.x;
    if (t < pi.count * pi.taps) {
      const int64_t k = pi.off[t];
      if (k >= 0) atomicAdd(&pi.p[k], pi.coef[t] * pi.sig[int64_t(t / pi.taps) * pi.sig_stride + pi.step]);
    }
    return;
  }
  b -= fg.pre;
  if (b < fg.rec) {
    const int r = b * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r < rec.count) sample_receiver(p, rec, f, out, step, r, threadIdx.x & 31, true);
    return;
  }
  b -= fg.rec;
  if (b < fg.z + fg.y) {  // block: 256 consecutive x of one (side, y) or (side, z) line
    const bool zf = b < fg.z;
    if (!zf) b -= fg.z;
    const int na = zf ? f.ny : f.nz;
    int line, ib;
    if (fg.flat) {  // 256 consecutive (line, x) positions
      const int t = b * 256 + int(threadIdx.x);
      if (t >= 2 * na * f.nx) return;
      line = t / f.nx;
      ib = t - line * f.nx;
    } else {
      line = b / fg.bxz;
      ib = (b - line * fg.bxz) * 256 + threadIdx.x;
      if (ib >= f.nx) return;
    }
    const int side = line >= na ? 1 : 0;
    if (zf)
      face_line<0, R>(p, f, side, line - side * na, ib);
    else
      face_line<1, R>(p, f, side, line - side * na, ib);
    return;
  }
  b -= fg.z + fg.y;
  // block: 256 / kFaceLanes consecutive rows of one (side, z) plane of an x face
  constexpr int LPR = face_lanes<R>();
  int plane, y;
  if (fg.flat) {  // 256 / LPR consecutive (side, z, y) rows
    const int r = b * (256 / LPR) + int(threadIdx.x) / LPR;
    if (r >= 2 * f.nz * f.ny) return;
    plane = r / f.ny;
    y = r - plane * f.ny;
  } else {
    plane = b / fg.bxx;
    y = (b - plane * fg.bxx) * (256 / LPR) + int(threadIdx.x) / LPR;
    if (y >= f.ny) return;
  }
  const int side = plane >= f.nz ? 1 : 0;
  face_x<R>(p, f, side, plane - side * f.nz, y, int(threadIdx.x) % LPR + 1);
}

template <int R>
__global__ void face_conditions_kernel(float* p, FaceInfo f, PointSet rec, float* out, int step, FaceGrid fg,
                                       PreInject pi) {
  griddep_launch_dependents();
  griddep_wait();  // p[n+1] of the stencil and the injection launched before
  face_block<R>(p, f, rec, out, step, fg, pi, blockIdx.x);
}

// The face launches of a batch of 3D grids in one launch: grid i owns the
// blocks [block0, block0 + fg.total()) and runs its own face launch there
// (face conditions of p[n+1], receiver samples, the next step's sources
// into p[n]).
struct FaceBatchDesc {
  float* lv[2];  // the two levels (node (0, 0, 0)); p[n+1] of step n is lv[(n + 1) & 1]
  FaceInfo f;
  PointSet rec;
  float* seis;  // [n_steps][n_rec] receiver samples
  FaceGrid fg;
  const int64_t* tap_off;  // source tap table and pre-injection coefficients (PreInject)
  const float* tap_pre;
  const float* sig;
  const unsigned char* live;  // per step: some source sample is non-zero
  int taps, n_src, sig_stride;
  int block0;
};

template <int R>
__global__ void face_batch_kernel(const FaceBatchDesc* __restrict__ d, int n, int total, int step, int n_steps) {
  griddep_launch_dependents();
  griddep_wait();  // the batch's stencil launch
  // the blocks of all grids' face launches, walked by a persistent grid
  for (int b = blockIdx.x; b < total; b += gridDim.x) {
    int gi = 0;
    for (int i = 1; i < n && d[i].block0 <= b; ++i) gi = i;
    const FaceBatchDesc& D = d[gi];
    PreInject pi{};
    if (step + 1 < n_steps && D.n_src > 0 && D.live[step + 1])
      pi = PreInject{D.lv[step & 1], D.tap_off, D.tap_pre, D.sig, D.taps, D.n_src, D.sig_stride, step + 1};
    face_block<R>(D.lv[(step + 1) & 1], D.f, D.rec, D.seis, step, D.fg, pi, b - D.block0);
  }
}

// Launch with programmatic stream serialization: the kernel may start before
// the previous kernel of the stream ends (it calls griddep_wait() first).
template <typename... P, typename... A>
inline void launch_dependent(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Face conditions of p (after the 3D pipelined stencil, the two-step 2D
// kernel and in the gradient's passes) and, if rec.count > 0, the
// receiver samples of this step, and, if pi.count > 0, the pre-injection of
// the next step's sources, in one launch of 256-thread blocks.
// Blocks of each part of a face launch: pre_threads threads of
// pre-injection, rec_count receivers, the face lines of the axes with a
// condition.
inline FaceGrid face_grid(const FaceInfo& f, int R, int rec_count, int pre_threads, bool flat = false) {
  FaceGrid fg;
  fg.pre = (pre_threads + 255) / 256;
  fg.rec = (rec_count + 7) / 8;
  // an axis whose two faces have no condition has nothing to write (its
  // ghosts stay zero): no blocks for it (the y axis of a 2D grid)
  const bool zf = f.bc[0] != kBcNone || f.bc[1] != kBcNone, yf = f.bc[2] != kBcNone || f.bc[3] != kBcNone,
             xf = f.bc[4] != kBcNone || f.bc[5] != kBcNone;
  const int lpr = R <= 8 ? 8 : 16;  // face_lanes<R>()
  fg.bxz = (f.nx + 255) / 256;
  fg.bxx = (f.ny + 256 / lpr - 1) / (256 / lpr);
  fg.z = zf ? 2 * f.ny * fg.bxz : 0;
  fg.y = yf ? 2 * f.nz * fg.bxz : 0;
  fg.x = xf ? 2 * f.nz * fg.bxx : 0;
  if (flat) {
    fg.flat = 1;
    fg.z = zf ? int((2 * int64_t(f.ny) * f.nx + 255) / 256) : 0;
    fg.y = yf ? int((2 * int64_t(f.nz) * f.nx + 255) / 256) : 0;
    fg.x = xf ? int((2 * int64_t(f.nz) * f.ny + 256 / lpr - 1) / (256 / lpr)) : 0;
  }
  return fg;
}

inline void launch_face_conditions(float* p, const FaceInfo& f, int R, const PointSet& rec, float* out, int step,
                                   cudaStream_t st, const PreInject& pi = PreInject{}) {
  // faces narrower than a block (a 2D grid's x faces are one row per plane)
  // are numbered across lines, so that no block runs with idle lanes
  const bool narrow = f.nx < 256 || f.ny < 256 / (R <= 8 ? 8 : 16);
  const FaceGrid fg = face_grid(f, R, rec.count, pi.count * pi.taps, narrow);
  const unsigned grid = unsigned(fg.total());
  switch (R) {
    case 1: launch_dependent(face_conditions_kernel<1>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 2: launch_dependent(face_conditions_kernel<2>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 3: launch_dependent(face_conditions_kernel<3>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 4: launch_dependent(face_conditions_kernel<4>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 5: launch_dependent(face_conditions_kernel<5>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 6: launch_dependent(face_conditions_kernel<6>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 7: launch_dependent(face_conditions_kernel<7>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 8: launch_dependent(face_conditions_kernel<8>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 9: launch_dependent(face_conditions_kernel<9>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    case 10: launch_dependent(face_conditions_kernel<10>, dim3(grid), dim3(256), 0, st, p, f, rec, out, step, fg, pi); break;
    default: break;
  }
}

// ---- misfit gradient (adjoint-state method) ---------------------------------
//
// Extension beyond the paper, which names FWI as the solver's use: the exact
// discrete adjoint of the forward recurrence.  In psi = kappa a lambda
// (lambda the adjoint state, a = 1/(1+e)) one adjoint step is the forward
// update with the transposed Laplacian L^T and the residuals injected
// through the receiver weights; L^T is L with the same ghost mirrors except
// along a Neumann face, where the even mirror makes L non-symmetric.

// L^T psi - L psi along the Neumann faces, scaled as the update uses it:
// out += a kappa (v_k / h^2) psi1[face] at the nodes k = 1..R from the face,
// out -= a kappa sum_k (v_k / h^2) psi1[k] at the face node.  psi1 is the
// level the stencil just read, out the level it wrote (before the face
// conditions).  One thread per (axis, side, face line); nodes near two
// Neumann faces get both corrections (atomics).
struct LapCoef {
  float c[3][kMaxR + 1];  // v_j / h^2 per axis (z, y, x)
};

template <int AX>
__device__ __forceinline__ void neumann_adjoint_axis(const float* psi1, float* out, const float* kappa,
                                                     const float2* damp, const FaceInfo& f, const LapCoef& lc, int R,
                                                     int64_t t) {
  // the two other axes (o1 slower, o2 faster) and their extents and strides
  constexpr int O1 = AX == 0 ? 1 : 0, O2 = AX == 2 ? 1 : 2;
  const int n_ax = AX == 0 ? f.nz : (AX == 1 ? f.ny : f.nx);
  const int n1 = O1 == 0 ? f.nz : f.ny;
  const int n2 = O2 == 1 ? f.ny : f.nx;
  const int64_t s_ax = AX == 0 ? f.sz : (AX == 1 ? f.sy : 1);
  const int64_t s1 = O1 == 0 ? f.sz : f.sy;
  const int64_t s2 = O2 == 1 ? f.sy : 1;
  const int64_t face = int64_t(n1) * n2;
  if (t >= 2 * face) return;
  const int side = int(t / face);
  if ((side ? f.bc[2 * AX + 1] : f.bc[2 * AX]) != kBcNeumann) return;  // constant indices: f stays in registers
  const int64_t e = t - side * face;
  const int c1 = int(e / n2), c2 = int(e - (e / n2) * n2);
  const int64_t base = int64_t(c1) * s1 + int64_t(c2) * s2;
  // squared distance to the physical box along the two other axes
  const int d1 = O1 == 0 ? face_distance(c1, f.nz, f.nbl[0], f.nbl[1]) : face_distance(c1, f.ny, f.nbl[2], f.nbl[3]);
  const int d2o = O2 == 1 ? face_distance(c2, f.ny, f.nbl[2], f.nbl[3]) : face_distance(c2, f.nx, f.nbl[4], f.nbl[5]);
  const int d12 = d1 * d1 + d2o * d2o;
  auto at = [&](int k, float* a) {  // node k in from this face, and its 1/(1+e)
    const int c = side == 0 ? k : n_ax - 1 - k;
    const int da = face_distance(c, n_ax, f.nbl[2 * AX], f.nbl[2 * AX + 1]);
    const int d2 = d12 + da * da;
    *a = d2 ? damp[d2].x : 1.f;
    return base + int64_t(c) * s_ax;
  };
  float a0;
  const int64_t k0 = at(0, &a0);
  const float pf = psi1[k0];
  float back = 0.f;
#pragma unroll
  for (int k = 1; k <= kMaxR; ++k) {  // unrolled to kMaxR so that the weights stay in registers
    if (k > R) break;
    float ak;
    const int64_t kk = at(k, &ak);
    atomicAdd(&out[kk], ak * kappa[kk] * lc.c[AX][k] * pf);
    back = fmaf(lc.c[AX][k], psi1[kk], back);
  }
  atomicAdd(&out[k0], -a0 * kappa[k0] * back);
}

// The source part of the same term: gk += psi s over the source windows
// (s = window weights / prod(h) times S(t_n)), one thread per tap.
__device__ __forceinline__ void image_source_tap(const float* psi, float* gk, const PointSet& src, const float* sig,
                                                 int sig_stride, int step, const FaceInfo& f, int t) {
  const int taps = src.lz * src.ly * src.lx;
  if (t >= src.count * taps) return;
  const int s = t / taps;
  int rem = t % taps;
  const int ix = rem % src.lx;
  rem /= src.lx;
  const int iy = rem % src.ly;
  const int iz = rem / src.ly;
  const float* w = src.w + int64_t(s) * 3 * src.L;
  const float wgt = w[iz] * w[src.L + iy] * w[2 * src.L + ix];
  const int64_t k = int64_t(src.first[3 * s] + iz) * f.sz + int64_t(src.first[3 * s + 1] + iy) * f.sy +
                    (src.first[3 * s + 2] + ix);
  atomicAdd(&gk[k], psi[k] * wgt * sig[int64_t(s) * sig_stride + step]);
}

__global__ void image_sources_kernel(const float* psi, float* gk, PointSet src, const float* sig, int sig_stride,
                                     int step, FaceInfo f) {
  image_source_tap(psi, gk, src, sig, sig_stride, step, f, blockIdx.x * blockDim.x + threadIdx.x);
}

// The source imaging of an earlier adjoint step, folded into the next
// step's additions launch (adjoint_additions_kernel): psi is that step's
// final adjoint state (the next step only reads it); blocks = 0: none.
struct SourceImaging {
  const float* psi;
  float* gk;
  PointSet src;
  const float* sig;
  int sig_stride, step, blocks;
};


// The two additions an adjoint step makes to psi after its stencil, in one
// launch: the Neumann-face correction (nb.x + nb.y + nb.z blocks, after the
// si.blocks of an earlier step's source imaging) and the residuals through
// the receiver windows (the blocks after them).  Both only add to `out`
// with atomics and read other arrays, so their blocks run in any order, as
// do the source imaging's, which add to gk.
// nb: blocks of the Neumann correction per axis (0 for an axis without a
// Neumann face).
__global__ void adjoint_additions_kernel(const float* psi1, float* out, const float* kappa, const float2* damp,
                                         FaceInfo f, LapCoef lc, int R, int3 nb, PointSet rec, int max_rows,
                                         const float* res, int res_stride, int step, int ndim, SourceImaging si) {
  griddep_launch_dependents();
  griddep_wait();  // the adjoint stencil launched before
  int b = blockIdx.x;
  if (b < si.blocks) {  // an earlier step's source imaging (adds to gk, reads other arrays than out)
    image_source_tap(si.psi, si.gk, si.src, si.sig, si.sig_stride, si.step, f, b * blockDim.x + threadIdx.x);
    return;
  }
  b -= si.blocks;
  if (b < nb.x) {
    neumann_adjoint_axis<0>(psi1, out, kappa, damp, f, lc, R, int64_t(b) * blockDim.x + threadIdx.x);
    return;
  }
  b -= nb.x;
  if (b < nb.y) {
    neumann_adjoint_axis<1>(psi1, out, kappa, damp, f, lc, R, int64_t(b) * blockDim.x + threadIdx.x);
    return;
  }
  b -= nb.y;
  if (b < nb.z) {
    neumann_adjoint_axis<2>(psi1, out, kappa, damp, f, lc, R, int64_t(b) * blockDim.x + threadIdx.x);
    return;
  }
  b -= nb.z;
  inject_row_node(out, kappa, damp, rec, max_rows, res, res_stride, step, f, ndim, R, b * blockDim.x + threadIdx.x);
}

// One term of kappa dJ/dkappa per node: gk += psi (L p), L the Eq. 9
// Laplacian of p (whose ghosts hold the face conditions), in the same
// constant-annihilating form as the stencils; the factor 1/kappa, the same
// at every step, is applied once at the end (gradient_velocity_kernel), so
// the pass reads no kappa.  Block (128 x, y, z).
template <int R, int NDIM>
__global__ void image_kernel(const float* p, const float* psi, float* gk, FaceInfo f, LapCoef lc) {
  griddep_launch_dependents();
  griddep_wait();  // psi of the face launch before
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= f.nx) return;
  const int64_t k = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
  const float ps = psi[k];
  if (ps == 0.f) return;
  const float pc = p[k], p2 = 2.f * pc;
  float lap = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    lap = fmaf(lc.c[0][j], (p[k + j * f.sz] + p[k - j * f.sz]) - p2, lap);
    lap = fmaf(lc.c[2][j], (p[k + j] + p[k - j]) - p2, lap);
    if constexpr (NDIM == 3) lap = fmaf(lc.c[1][j], (p[k + j * f.sy] + p[k - j * f.sy]) - p2, lap);
  }
  gk[k] += ps * lap;
}

// Residual r = synthetic - observed, transposed to [receiver][step] (the
// layout inject_sources_kernel reads a per-source signal in), and the misfit
// 1/2 sum r^2 accumulated in FP64.
__global__ void residual_kernel(const float* syn, const float* obs, float* res_t, double* misfit, int n_steps,
                                int n_rec) {
  __shared__ double part[8];
  double acc = 0.0;
  const int64_t total = int64_t(n_steps) * n_rec;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int n = int(i / n_rec), r = int(i % n_rec);
    const float d = syn[i] - obs[i];
    res_t[int64_t(r) * n_steps + n] = d;
    acc += double(d) * double(d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) s += part[i];
    atomicAdd(misfit, 0.5 * s);
  }
}

// dJ/dc = 2 c dt^2 dJ/dkappa with dJ/dkappa = gk / kappa (gk the accumulated
// kappa dJ/dkappa), densely per node.
__global__ void gradient_velocity_kernel(const float* gk, const float* kappa, float* out, FaceInfo f, float dt) {
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    const int64_t k = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
    out[i] = 2.f * dt * gk[k] / sqrtf(kappa[k]);  // 2 c dt^2 gk / kappa, kappa = (c dt)^2
  }
}

// ---- variable-density gradient -------------------------------------------------
//
// With density the forward operator is L_rho p = L p - sum_a G_a D_a p
// (G_a = D_a ln rho, Eq. 10), whose transpose is
// L_rho^T q = L^T q - sum_a D_a^T (G_a q).  D_a^T is the transpose of "fill
// the ghosts from the face conditions, then take the centred difference":
// (D^T q)[m] = sum_j w_j/(2h) (q[m-j] - q[m+j]) with q zero off the nodes,
// plus, for each ghost of a mirrored face, its share folded back onto the
// node it mirrors (sign -1 on a Dirichlet face, +1 on a Neumann face or for
// the even extension of ln rho).

struct VdWeights {
  float w[3][kMaxR + 1];  // w_j / (2h) per axis (z, y, x)
};

// (D^T q) at node m of an axis of n nodes; q(i) reads q at node i of the axis.
template <typename Q>
__device__ __forceinline__ float dt_axis(const Q& q, int m, int n, const float* wh, int R, float s_lo, float s_hi) {
  float acc = 0.f;
  for (int j = 1; j <= R; ++j) {
    if (m - j >= 0) acc = fmaf(wh[j], q(m - j), acc);
    if (m + j < n) acc = fmaf(-wh[j], q(m + j), acc);
  }
  if (s_lo != 0.f && m >= 1 && m <= R)  // ghost -m: gets -sum_{j>=m} w_j q[j-m]
    for (int j = m; j <= R; ++j) acc = fmaf(-s_lo * wh[j], q(j - m), acc);
  const int g = n - 1 - m;
  if (s_hi != 0.f && g >= 1 && g <= R)  // ghost n-1+g: gets sum_{j>=g} w_j q[n-1+g-j]
    for (int j = g; j <= R; ++j) acc = fmaf(s_hi * wh[j], q(n - 1 + g - j), acc);
  return acc;
}

__device__ __forceinline__ float mirror_sign(int bc) {
  return bc == kBcDirichlet ? -1.f : (bc == kBcNeumann ? 1.f : 0.f);
}

// The density part of one adjoint step: out += -a kappa sum_a D_a^T (G_a psi)
// at every node (psi = psi[k+1], G_a = D_a ln rho in the padded layout).
__global__ void vd_adjoint_kernel(const float* psi, const float* gz, const float* gy, const float* gx,
                                  const float* kappa, const float2* damp, float* out, FaceInfo f, VdWeights W, int R,
                                  int ndim) {
  griddep_launch_dependents();
  griddep_wait();  // the adjoint stencil launched before
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    const int64_t k = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
    const int64_t bz = k - int64_t(z) * f.sz, bx = k - x;
    float t = dt_axis([&](int j) { return gz[bz + j * f.sz] * psi[bz + j * f.sz]; }, z, f.nz, W.w[0], R,
                      mirror_sign(f.bc[0]), mirror_sign(f.bc[1]));
    t += dt_axis([&](int j) { return gx[bx + j] * psi[bx + j]; }, x, f.nx, W.w[2], R, mirror_sign(f.bc[4]),
                 mirror_sign(f.bc[5]));
    if (ndim == 3) {
      const int64_t by = k - int64_t(y) * f.sy;
      t += dt_axis([&](int j) { return gy[by + j * f.sy] * psi[by + j * f.sy]; }, y, f.ny, W.w[1], R,
                   mirror_sign(f.bc[2]), mirror_sign(f.bc[3]));
    }
    const int dz = face_distance(z, f.nz, f.nbl[0], f.nbl[1]);
    const int dy = ndim == 3 ? face_distance(y, f.ny, f.nbl[2], f.nbl[3]) : 0;
    const int dx = face_distance(x, f.nx, f.nbl[4], f.nbl[5]);
    const int d2 = dz * dz + dy * dy + dx * dx;
    const float a = d2 ? damp[d2].x : 1.f;
    out[k] -= a * kappa[k] * t;
  }
}

// One term of kappa dJ/dkappa and of dJ/dG_a with density: gk += psi L_rho p
// and A_a -= psi D_a p (p's ghosts hold the face conditions).
template <int R, int NDIM>
__global__ void image_vd_kernel(const float* p, const float* psi, const float* gz,
                                const float* gy, const float* gx, float* gk, float* az, float* ay, float* ax,
                                FaceInfo f, LapCoef lc, VdWeights W) {
  griddep_launch_dependents();
  griddep_wait();  // psi of the face launch before
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= f.nx) return;
  const int64_t k = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
  const float ps = psi[k];
  if (ps == 0.f) return;
  const float pc = p[k], p2 = 2.f * pc;
  float lap = 0.f, dz = 0.f, dy = 0.f, dx = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    const float zp = p[k + j * f.sz], zm = p[k - j * f.sz], xp = p[k + j], xm = p[k - j];
    lap = fmaf(lc.c[0][j], (zp + zm) - p2, lap);
    lap = fmaf(lc.c[2][j], (xp + xm) - p2, lap);
    dz = fmaf(W.w[0][j], zp - zm, dz);
    dx = fmaf(W.w[2][j], xp - xm, dx);
    if constexpr (NDIM == 3) {
      const float yp = p[k + j * f.sy], ym = p[k - j * f.sy];
      lap = fmaf(lc.c[1][j], (yp + ym) - p2, lap);
      dy = fmaf(W.w[1][j], yp - ym, dy);
    }
  }
  float adv = fmaf(gz[k], dz, gx[k] * dx);
  if constexpr (NDIM == 3) adv = fmaf(gy[k], dy, adv);
  gk[k] += ps * (lap - adv);
  az[k] -= ps * dz;
  ax[k] -= ps * dx;
  if constexpr (NDIM == 3) ay[k] -= ps * dy;
}

// dJ/drho = (sum_a D_a^T A_a) / rho with the even extension of ln rho (A_a =
// dJ/dG_a), densely per node.
__global__ void gradient_density_kernel(const float* az, const float* ay, const float* ax, const float* lnrho,
                                        float* out, FaceInfo f, VdWeights W, int R, int ndim) {
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    const int64_t k = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
    const int64_t bz = k - int64_t(z) * f.sz, bx = k - x;
    float t = dt_axis([&](int j) { return az[bz + j * f.sz]; }, z, f.nz, W.w[0], R, 1.f, 1.f);
    t += dt_axis([&](int j) { return ax[bx + j]; }, x, f.nx, W.w[2], R, 1.f, 1.f);
    if (ndim == 3) {
      const int64_t by = k - int64_t(y) * f.sy;
      t += dt_axis([&](int j) { return ay[by + j * f.sy]; }, y, f.ny, W.w[1], R, 1.f, 1.f);
    }
    out[i] = t / expf(lnrho[k]);
  }
}

// ---- compressed checkpoints ---------------------------------------------------
// A checkpointed wavefield is stored as its nodes only, in 16 bits, divided by
// the field's largest magnitude (its per-snapshot scale); restoring
// multiplies back and leaves the ghosts to the face conditions.

// max |p| over the nodes, as the bit pattern of a non-negative float
// (order-preserving as an unsigned integer).
// Node passes over (z, y) rows: blockIdx.x along x (256 threads), blockIdx.y
// striding over the nz * ny rows, so that no thread divides per node.
inline dim3 row_grid(const FaceInfo& f) {
  const int64_t rows = int64_t(f.nz) * f.ny;
  const int64_t cap = 4096 / ((f.nx + 255) / 256) + 1;  // a few thousand CTAs, each walking many rows
  return dim3(unsigned((f.nx + 255) / 256), unsigned(rows < cap ? rows : cap));
}

// max |p - q| over the nodes (q may be NULL: max |p|)
__global__ void absmax_kernel(const float* p, const float* q, FaceInfo f, unsigned* out) {
  unsigned m = 0u;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = int64_t(f.nz) * f.ny;
  if (x < f.nx)
    for (int64_t zy = blockIdx.y; zy < rows; zy += gridDim.y) {
      const int64_t k = (zy / f.ny) * f.sz + (zy % f.ny) * f.sy + x;
      m = max(m, __float_as_uint(fabsf(q ? p[k] - q[k] : p[k])));
    }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__device__ __forceinline__ float snapshot_scale(const unsigned* bits) {
  const float s = __uint_as_float(*bits);
  return s > 0.f ? s : 1.f;
}

template <typename T>
__device__ __forceinline__ T to_half_kind(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_half_kind<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_half_kind<__half>(float v) { return __float2half_rn(v); }

// out = (p - q) / scale per node in 16 bits (q may be NULL: p / scale)
template <typename T>
__global__ void pack_snapshot_kernel(const float* p, const float* q, FaceInfo f, const unsigned* scale_bits, T* out) {
  const float inv = 1.f / snapshot_scale(scale_bits);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = int64_t(f.nz) * f.ny;
  if (x >= f.nx) return;
  for (int64_t zy = blockIdx.y; zy < rows; zy += gridDim.y) {
    const int64_t k = (zy / f.ny) * f.sz + (zy % f.ny) * f.sy + x;
    out[zy * f.nx + x] = to_half_kind<T>((q ? p[k] - q[k] : p[k]) * inv);
  }
}

// p = base - in * scale per node (base may be NULL: p = in * scale)
template <typename T>
__global__ void unpack_snapshot_kernel(const T* in, const unsigned* scale_bits, FaceInfo f, const float* base,
                                       float* p) {
  const float sc = snapshot_scale(scale_bits);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = int64_t(f.nz) * f.ny;
  if (x >= f.nx) return;
  for (int64_t zy = blockIdx.y; zy < rows; zy += gridDim.y) {
    const int64_t k = (zy / f.ny) * f.sz + (zy % f.ny) * f.sy + x;
    const float v = float(in[zy * f.nx + x]) * sc;
    p[k] = base ? base[k] - v : v;
  }
}

// 16-bit fixed point with one scale per (z, y) row of the nodes:
// q = round(v * 32767 / s), s = max |v| over the row, v = p - base (base may
// be NULL: v = p).  Wavefields vary smoothly along a row, so the step
// s / 32767 is small next to the values that matter, where a 16-bit float
// keeps only 8 or 11 bits of every value.  One CTA of 256 threads per row.
__global__ void pack_rows_i16_kernel(const float* p, const float* base, FaceInfo f, float* scales, int16_t* out) {
  griddep_launch_dependents();
  griddep_wait();  // the level of the stencil launched before
  // one warp per (z, y) row; rows of a multiple of 4 nodes in float4 / 4 x int16 pieces
  // (row starts are 128-byte aligned in the padded layout), others one node per lane
  const int lane = threadIdx.x & 31;
  const int64_t rows = int64_t(f.nz) * f.ny;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const bool vec = (f.nx & 3) == 0;
  for (int64_t zy = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; zy < rows; zy += nw) {
    const int64_t off = (zy / f.ny) * f.sz + (zy % f.ny) * f.sy;
    const float* pr = p + off;
    const float* br = base ? base + off : nullptr;
    int16_t* orow = out + zy * f.nx;
    float m = 0.f;
    if (vec) {
      for (int x = 4 * lane; x < f.nx; x += 128) {
        float4 v = *reinterpret_cast<const float4*>(pr + x);
        if (br) {
          const float4 b = *reinterpret_cast<const float4*>(br + x);
          v = make_float4(v.x - b.x, v.y - b.y, v.z - b.z, v.w - b.w);
        }
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
    } else {
      for (int x = lane; x < f.nx; x += 32) m = fmaxf(m, fabsf(br ? pr[x] - br[x] : pr[x]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float sc = m > 0.f ? m : 1.f;
    if (lane == 0) scales[zy] = sc;
    const float inv = 32767.f / sc;
    if (vec) {
      for (int x = 4 * lane; x < f.nx; x += 128) {
        float4 v = *reinterpret_cast<const float4*>(pr + x);
        if (br) {
          const float4 b = *reinterpret_cast<const float4*>(br + x);
          v = make_float4(v.x - b.x, v.y - b.y, v.z - b.z, v.w - b.w);
        }
        short4 q;
        q.x = int16_t(__float2int_rn(v.x * inv));
        q.y = int16_t(__float2int_rn(v.y * inv));
        q.z = int16_t(__float2int_rn(v.z * inv));
        q.w = int16_t(__float2int_rn(v.w * inv));
        *reinterpret_cast<short4*>(orow + x) = q;
      }
    } else {
      for (int x = lane; x < f.nx; x += 32)
        orow[x] = int16_t(__float2int_rn((br ? pr[x] - br[x] : pr[x]) * inv));
    }
  }
}

// p = base - v or p = v with v = q * s / 32767 (row scales s); one warp per
// (z, y) row, in 4-node pieces when the row length allows.
__global__ void unpack_rows_i16_kernel(const int16_t* in, const float* scales, FaceInfo f, const float* base,
                                       float* p) {
  griddep_launch_dependents();
  griddep_wait();  // the kernels launched before
  const int lane = threadIdx.x & 31;
  const int64_t rows = int64_t(f.nz) * f.ny;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const bool vec = (f.nx & 3) == 0;
  for (int64_t zy = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; zy < rows; zy += nw) {
    const int64_t off = (zy / f.ny) * f.sz + (zy % f.ny) * f.sy;
    const float s = scales[zy] * (1.f / 32767.f);
    const int16_t* irow = in + zy * f.nx;
    float* pr = p + off;
    const float* br = base ? base + off : nullptr;
    if (vec) {
      for (int x = 4 * lane; x < f.nx; x += 128) {
        const short4 q = *reinterpret_cast<const short4*>(irow + x);
        float4 v = make_float4(float(q.x) * s, float(q.y) * s, float(q.z) * s, float(q.w) * s);
        if (br) {
          const float4 b = *reinterpret_cast<const float4*>(br + x);
          v = make_float4(b.x - v.x, b.y - v.y, b.z - v.z, b.w - v.w);
        }
        *reinterpret_cast<float4*>(pr + x) = v;
      }
    } else {
      for (int x = lane; x < f.nx; x += 32) {
        const float v = float(irow[x]) * s;
        pr[x] = br ? br[x] - v : v;
      }
    }
  }
}

// Distributed forcing f(x, t_n) = sum_m F_m(x) T_m(t_n), added like a source
// term (Eq. 7 and 11 with a dense source): p[n+1]_k += kappa_k a_k f_k.  The
// nodes are dense ([n_force][nz][ny][nx] fields, [n_force][n_sig] signatures);
// Dirichlet face nodes stay 0; with `mirrors` the ghost images get the same
// increment (the face conditions do not follow on that path).
__global__ void forcing_kernel(float* p, const float* kappa, const float2* damp, const float* F, const float* T,
                               int n_force, int n_sig, int step, FaceInfo f, int ndim, int R, int mirrors) {
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    const bool dir = (z == 0 && f.bc[0] == kBcDirichlet) || (z == f.nz - 1 && f.bc[1] == kBcDirichlet) ||
                     (x == 0 && f.bc[4] == kBcDirichlet) || (x == f.nx - 1 && f.bc[5] == kBcDirichlet) ||
                     (ndim == 3 && ((y == 0 && f.bc[2] == kBcDirichlet) ||
                                    (y == f.ny - 1 && f.bc[3] == kBcDirichlet)));
    if (dir) continue;
    float s = 0.f;
    for (int m = 0; m < n_force; ++m) s = fmaf(F[int64_t(m) * n + i], T[int64_t(m) * n_sig + step], s);
    const int64_t idx = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
    const int dz = face_distance(z, f.nz, f.nbl[0], f.nbl[1]);
    const int dy = ndim == 3 ? face_distance(y, f.ny, f.nbl[2], f.nbl[3]) : 0;
    const int dx = face_distance(x, f.nx, f.nbl[4], f.nbl[5]);
    const int d2 = dz * dz + dy * dy + dx * dx;
    const float d = kappa[idx] * (d2 ? damp[d2].x : 1.f) * s;
    p[idx] += d;
    if (mirrors) {
      add_with_mirrors(p, idx, z, f.nz, f.sz, f.bc[0], f.bc[1], R, d);
      add_with_mirrors(p, idx, x, f.nx, 1, f.bc[4], f.bc[5], R, d);
      if (ndim == 3) add_with_mirrors(p, idx, y, f.ny, f.sy, f.bc[2], f.bc[3], R, d);
    }
  }
}

// Writes a dense field into the nodes of a zeroed padded field, with the
// ghost images the face conditions give (odd mirror on a Dirichlet face, even
// on a Neumann face, none stays 0).  Dirichlet face nodes are set to 0.
__device__ __forceinline__ void set_with_mirrors(float* p, int64_t idx, int i, int n, int64_t stride, int bc_lo,
                                                 int bc_hi, int R, float v) {
  if (bc_lo != kBcNone && i >= 1 && i <= R) p[idx - int64_t(2 * i) * stride] = bc_lo == kBcDirichlet ? -v : v;
  const int m = n - 1 - i;
  if (bc_hi != kBcNone && m >= 1 && m <= R) p[idx + int64_t(2 * m) * stride] = bc_hi == kBcDirichlet ? -v : v;
}

__global__ void insert_kernel(const float* in, float* p, FaceInfo f, int ndim, int R) {
  const int64_t n = int64_t(f.nz) * f.ny * f.nx;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % f.nx);
    const int64_t zy = i / f.nx;
    const int y = int(zy % f.ny);
    const int z = int(zy / f.ny);
    const bool dir = (z == 0 && f.bc[0] == kBcDirichlet) || (z == f.nz - 1 && f.bc[1] == kBcDirichlet) ||
                     (x == 0 && f.bc[4] == kBcDirichlet) || (x == f.nx - 1 && f.bc[5] == kBcDirichlet) ||
                     (ndim == 3 && ((y == 0 && f.bc[2] == kBcDirichlet) ||
                                    (y == f.ny - 1 && f.bc[3] == kBcDirichlet)));
    const float v = dir ? 0.f : in[i];
    const int64_t idx = int64_t(z) * f.sz + int64_t(y) * f.sy + x;
    p[idx] = v;
    set_with_mirrors(p, idx, z, f.nz, f.sz, f.bc[0], f.bc[1], R, v);
    set_with_mirrors(p, idx, x, f.nx, 1, f.bc[4], f.bc[5], R, v);
    if (ndim == 3) set_with_mirrors(p, idx, y, f.ny, f.sy, f.bc[2], f.bc[3], R, v);
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
