// Whole forward run of a small 2D grid in one launch of one thread-block
// cluster, the wavefields resident in the cluster's shared memory.
//
// A 2D grid of a few hundred thousand nodes (the 256 x 256 homogeneous
// workload has 65,536) is far too small to keep HBM busy: one kernel launch
// per time step spends most of its time in launch latency and in the
// dependency between consecutive steps.  Here the cluster's C CTAs (up to
// 16, one per SM) split the rows into bands; CTA c keeps rows
// [c B, min((c+1) B, nz)) of both levels p[n], p[n-1] and of kappa in its
// shared memory for the whole run, with R halo rows above and below and R
// ghost columns each side.  A time step is:
//   1. halo rows of p[n] from the CTAs that own them (distributed shared
//      memory), rows outside the grid as the face condition's image of the
//      rows inside it (Dirichlet: odd, Neumann: even, none: zero); then the
//      ghost columns of every row the same way; the receivers of p[n]
//      (seismogram row n - 1) are sampled from the owners' bands;
//   2. Eq. 7 (laplacian_2d, leapfrog_update: the single-grid 2D kernel's
//      operations in its order) for the band's nodes, written over p[n-1];
//      Dirichlet face nodes are set to zero;
//   3. the Eq. 11 source increments of the band's nodes (the same products
//      as inject_sources_kernel);
//   4. a cluster barrier (release / acquire), after which every CTA's p[n+1]
//      is complete and visible to the others.
// Ghost values are rebuilt from the nodes at every step, so they always hold
// the images of the node values, including the source increments, as the
// single-grid path's mirrored stores and mirrored increments do: the run is
// bit-identical to the single-grid 2D path.  Every thread of every CTA runs
// the same number of cluster barriers (one before the loop, one per step);
// nothing leaves the loop early.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "aux_kernels.cuh"
#include "stencil_plain.cuh"
#include "tma.cuh"

namespace sw {

namespace cg = cooperative_groups;

constexpr int kClusterThreads = 512;  // 16 warps per CTA
constexpr int kClusterMaxCtas = 16;   // non-portable cluster size
constexpr int kClusterRecRows = 8;    // receiver window rows kept in registers

struct ClusterRun {
  float* u[2];          // node (0, 0) of the two levels of the padded layout (in: p[0], p[-1]; out: the last two)
  const float* kappa;   // node (0, 0) of (c dt)^2
  const float2* damp;   // (a, e) by squared distance to the physical box
  FaceInfo f;           // nz, nx, row stride sz, absorbing cells and face conditions (z: 0, 1; x: 4, 5)
  int B;                // rows per band (the last band may be shorter)
  int W;                // shared row length (cluster_row_len)
  float cz[kMaxR + 1], cx[kMaxR + 1];  // v_j / h^2 per axis
  PointSet src, rec;
  const float* sig;  // wavelet samples [n_src or 1][nt]
  int sig_stride;
  float* seis;  // [n_steps][rec.count] on the device, or nullptr
  int n_steps;
  int rec_fast;  // one pass of the cluster's warps covers the receivers (see the kernel)
};

// Shared rows: column x of a row sits at index cluster_col0(R) + x, even so
// that column pairs are 8-byte aligned; the ghost columns -R .. -1 and
// nx .. nx - 1 + R and the columns a column pair's neighbour loads reach
// (up to R + 1 past either end) fit in a row of cluster_row_len floats.
__host__ __device__ inline int cluster_col0(int R) { return (R + 1) / 2 * 2; }
__host__ __device__ inline int cluster_row_len(int nx, int R) { return (cluster_col0(R) + nx + R + 2) / 2 * 2; }
__host__ __device__ inline int cluster_kappa_len(int nx) { return (nx + 1) / 2 * 2; }

// Shared floats of one CTA: two levels of (B + 2R) rows and B rows of kappa.
__host__ __device__ inline int64_t cluster_smem_floats(int B, int nx, int R) {
  return 2 * int64_t(B + 2 * R) * cluster_row_len(nx, R) + int64_t(B) * cluster_kappa_len(nx);
}

// Sign of a face's image: Dirichlet odd, Neumann even, none zero.
__device__ __forceinline__ float face_sign(int bc) {
  return bc == kBcDirichlet ? -1.f : (bc == kBcNeumann ? 1.f : 0.f);
}

template <int R>
__global__ void __launch_bounds__(kClusterThreads) stencil_2d_cluster_kernel(const ClusterRun run) {
  extern __shared__ __align__(16) float csm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int C = int(cluster.num_blocks());
  const FaceInfo& f = run.f;
  const int nz = f.nz, nx = f.nx, B = run.B, W = run.W;
  const int64_t sz = f.sz;
  const int z0 = rank * B;
  const int nb = max(min(B, nz - z0), 0);  // rows of this band
  constexpr int X0 = (R + 1) / 2 * 2;       // cluster_col0(R)
  const int KW = cluster_kappa_len(nx);
  const int lvl = (B + 2 * R) * W;          // floats per level
  auto level = [&](int k) { return csm + k * lvl; };  // level k: [r * W + X0 + x] is row z0 - R + r, column x
  float* K = csm + 2 * lvl;                 // kappa of the band: K[(z - z0) * KW + x]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kClusterThreads / 32;

  // both initial levels and kappa of the band into shared memory
  for (int r = warp; r < nb; r += NW) {
    const int64_t g = int64_t(z0 + r) * sz;
    for (int x = lane; x < nx; x += 32) {
      level(0)[(r + R) * W + X0 + x] = run.u[0][g + x];
      level(1)[(r + R) * W + X0 + x] = run.u[1][g + x];
      K[r * KW + x] = run.kappa[g + x];
    }
  }
  constexpr int H = (R + 1) / 2;  // float2 loads each side for the x neighbours of a column pair
  float2 cz[R + 1], cx[R + 1];
#pragma unroll
  for (int j = 0; j <= R; ++j) {
    cz[j] = make_float2(run.cz[j], run.cz[j]);
    cx[j] = make_float2(run.cx[j], run.cx[j]);
  }
  const float sz_lo = face_sign(f.bc[0]), sz_hi = face_sign(f.bc[1]);
  const float sx_lo = face_sign(f.bc[4]), sx_hi = face_sign(f.bc[5]);
  const bool dir_z0 = f.bc[0] == kBcDirichlet, dir_z1 = f.bc[1] == kBcDirichlet;
  const bool dir_x0 = f.bc[4] == kBcDirichlet, dir_x1 = f.bc[5] == kBcDirichlet;

  // Eq. 12 on level `cur` of every CTA, into seismogram row `row` (the
  // grouped receiver sampler's arithmetic: lanes along x, a group of G lanes
  // per receiver, the window rows with a non-zero weight).  When one pass of
  // the cluster's warps covers every receiver and a window has at most
  // kClusterRecRows such rows, each lane keeps its rows' owners, offsets and
  // weights in registers from the start of the run.
  const PointSet& rec = run.rec;
  const int G = rec.lx <= 8 ? 8 : (rec.lx <= 16 ? 16 : 32);
  const int gw0 = warp * C + rank;  // this warp's first group of receivers, spread over the CTAs
  const int r0 = gw0 * (32 / G) + lane / G, ix0 = lane % G;
  const bool one_pass = run.rec_fast != 0;
  int rz_owner[kClusterRecRows], rz_off[kClusterRecRows];
  float rz_w[kClusterRecRows], rx_w = 0.f;
  int rlz = 0;
  if (one_pass && run.seis && r0 < rec.count && ix0 < rec.lx) {
    const float* w = rec.w + int64_t(r0) * 3 * rec.L;
    int za = 0;
    rlz = rec.lz;
    if (rec.span) {
      const int4 sp = rec.span[r0];
      za = sp.x;
      rlz = sp.y;
    }
    const int x = rec.first[3 * r0 + 2] + ix0;
#pragma unroll
    for (int iz = 0; iz < kClusterRecRows; ++iz) {
      const int z = rec.first[3 * r0] + za + min(iz, rlz - 1);
      rz_owner[iz] = z / B;
      rz_off[iz] = (z - rz_owner[iz] * B + R) * W + X0 + x;
      rz_w[iz] = iz < rlz ? w[za + iz] * w[rec.L] : 0.f;
    }
    rx_w = w[2 * rec.L + ix0];
  }
  auto sample = [&](int cur, int row) {
    if (!run.seis) return;
    if (one_pass) {
      if (gw0 * (32 / G) >= rec.count) return;  // whole warps
      float s = 0.f;
#pragma unroll
      for (int iz = 0; iz < kClusterRecRows; ++iz)
        if (iz < rlz) s = fmaf(rz_w[iz], cluster.map_shared_rank(level(cur), rz_owner[iz])[rz_off[iz]], s);
      float acc = rlz > 0 ? rx_w * s : 0.f;
      for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (r0 < rec.count && ix0 == 0) run.seis[int64_t(row) * rec.count + r0] = acc;
      return;
    }
    for (int gw = gw0; gw * (32 / G) < rec.count; gw += C * NW) {
      const int r = gw * (32 / G) + lane / G;
      const int ix = lane % G;
      float acc = 0.f;
      if (r < rec.count && ix < rec.lx) {
        const float* w = rec.w + int64_t(r) * 3 * rec.L;
        int za = 0, lz = rec.lz;
        if (rec.span) {
          const int4 sp = rec.span[r];
          za = sp.x;
          lz = sp.y;
        }
        const int x = rec.first[3 * r + 2] + ix;
        float s = 0.f;
        for (int iz = 0; iz < lz; ++iz) {
          const int z = rec.first[3 * r] + za + iz;
          const int owner = z / B;
          const float* q = cluster.map_shared_rank(level(cur), owner);
          s = fmaf(w[za + iz] * w[rec.L], q[(z - owner * B + R) * W + X0 + x], s);
        }
        acc = w[2 * rec.L + ix] * s;
      }
      for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (r < rec.count && ix == 0) run.seis[int64_t(row) * rec.count + r] = acc;
    }
  };

  // Eq. 11 taps of this band: thread t owns tap t (the host sends runs with
  // at most kClusterThreads taps here): its offset in a level and
  // kappa a d_k, the step-independent factors in inject_sources_kernel's order
  const PointSet& src = run.src;
  int tap_off = -1, tap_s = 0;
  float tap_coef = 0.f;
  if (tid < src.count * src.lz * src.lx) {
    const int taps = src.lz * src.lx;
    const int s = tid / taps, rem = tid - s * taps;
    const int iz = rem / src.lx, ix = rem - iz * src.lx;
    const int z = src.first[3 * s] + iz, x = src.first[3 * s + 2] + ix;
    const float* w = src.w + int64_t(s) * 3 * src.L;
    const float wgt = w[iz] * w[src.L] * w[2 * src.L + ix];
    const bool dir = (z == 0 && dir_z0) || (z == nz - 1 && dir_z1) || (x == 0 && dir_x0) || (x == nx - 1 && dir_x1);
    if (z >= z0 && z < z0 + nb && wgt != 0.f && !dir) {
      const int dz = face_distance(z, nz, f.nbl[0], f.nbl[1]);
      const int dx = face_distance(x, nx, f.nbl[4], f.nbl[5]);
      const int d2 = dz * dz + dx * dx;
      const float ca = d2 ? run.damp[d2].x : 1.f;
      tap_off = (z - z0 + R) * W + X0 + x;
      tap_coef = K[(z - z0) * KW + x] * ca * wgt;
      tap_s = s;
    }
  }
  cluster.sync();  // every band loaded before any halo is read
  int cur = 0;
  for (int n = 0; n < run.n_steps; ++n) {
    float* Pc = level(cur);
    float* Po = level(cur ^ 1);
    // this step's source signature sample, ahead of its use
    const float sig_n = tap_off >= 0 ? run.sig[int64_t(tap_s) * run.sig_stride + n] : 0.f;
    // 1. halo rows of p[n]: rows z0 - R .. z0 - 1 and z0 + nb .. z0 + nb + R - 1
    for (int h = warp; h < 2 * R; h += NW) {
      const int r = h < R ? h : nb + h;  // shared row
      const int z = z0 - R + r;
      int zs = z;
      float sg = 1.f;
      if (z < 0) {
        zs = -z;
        sg = sz_lo;
      } else if (z >= nz) {
        zs = 2 * (nz - 1) - z;
        sg = sz_hi;
      }
      const int owner = zs / B;
      const float* q = cluster.map_shared_rank(Pc, owner) + (zs - owner * B + R) * W + X0;
      float* d = Pc + r * W + X0;
      // eight remote loads in flight per lane before the stores
      for (int xb = lane; xb < nx; xb += 32 * 8) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = xb + 32 * k < nx ? q[xb + 32 * k] : 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (xb + 32 * k < nx) d[xb + 32 * k] = sg * v[k];
      }
    }
    // ghost columns of the band's rows (the only rows whose x neighbours
    // the step reads), from the band's final values of the previous step
    for (int r = R + warp; r < R + nb; r += NW) {
      float* row = Pc + r * W + X0;
      if (lane < R) {
        const int j = lane + 1;
        row[-j] = sx_lo * row[j];
        row[nx - 1 + j] = sx_hi * row[nx - 1 - j];
      }
    }
    if (n > 0) sample(cur, n - 1);
    __syncthreads();
    // 2. p[n+1] over p[n-1], two adjacent columns per lane with packed
    //    FP32x2 operations (per column laplacian_2d's and leapfrog_update's
    //    operations in their order; a column past nx is computed, not stored)
    for (int r = warp; r < nb; r += NW) {
      const int z = z0 + r;
      const int dz = layer_distance(z, nz, f.nbl[0], f.nbl[1]);
      const bool zdir = (z == 0 && dir_z0) || (z == nz - 1 && dir_z1);
      const float* c = Pc + (r + R) * W + X0;
      float* orow = Po + (r + R) * W + X0;
      const float* krow = K + r * KW;
#pragma unroll 4
      for (int x = 2 * lane; x < nx; x += 64) {
        float2 qz[2 * R + 1];
#pragma unroll
        for (int j = -R; j <= R; ++j) qz[j + R] = *reinterpret_cast<const float2*>(c + j * W + x);
        float2 w[2 * H + 1];  // columns x-2H .. x+1+2H, as pairs
#pragma unroll
        for (int mm = -H; mm <= H; ++mm)
          w[mm + H] = (mm == 0) ? qz[R] : *reinterpret_cast<const float2*>(c + x + 2 * mm);
        const float2 pc = qz[R];
        const float2 p2 = f2_add(pc, pc);  // 2 p, exactly
        float2 lap = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 1; j <= R; ++j) {
          lap = f2_fma(cz[j], f2_sub(f2_add(qz[R + j], qz[R - j]), p2), lap);
          float2 xs;  // (x+j) + (x-j) for both columns
          if (j % 2 == 0) {
            xs = f2_add(w[H + j / 2], w[H - j / 2]);
          } else {  // odd offsets straddle the pairs: two scalar adds into one pair
            xs = make_float2(w[H + (j - 1) / 2].y + w[H - (j + 1) / 2].y, w[H + (j + 1) / 2].x + w[H - (j - 1) / 2].x);
          }
          lap = f2_fma(cx[j], f2_sub(xs, p2), lap);
        }
        const bool vb = x + 1 < nx;
        const int dxa = layer_distance(x, nx, f.nbl[4], f.nbl[5]);
        const int dxb = vb ? layer_distance(x + 1, nx, f.nbl[4], f.nbl[5]) : 0;
        const int d2a = dz * dz + dxa * dxa, d2b = dz * dz + dxb * dxb;
        float2 ca = make_float2(1.f, 1.f), e = make_float2(0.f, 0.f);
        if (d2a != 0) {
          const float2 dd = __ldg(&run.damp[d2a]);
          ca.x = dd.x;
          e.x = dd.y;
        }
        if (d2b != 0) {
          const float2 dd = __ldg(&run.damp[d2b]);
          ca.y = dd.x;
          e.y = dd.y;
        }
        const float2 po = *reinterpret_cast<const float2*>(orow + x);
        const float2 kp = *reinterpret_cast<const float2*>(krow + x);
        float2 pnew = f2_mul(ca, f2_add(pc, f2_fma(kp, lap, f2_fma(e, po, f2_sub(pc, po)))));
        if (zdir || (x == 0 && dir_x0) || (x == nx - 1 && dir_x1)) pnew.x = 0.f;
        if (zdir || (x + 1 == nx - 1 && dir_x1)) pnew.y = 0.f;
        if (vb)
          *reinterpret_cast<float2*>(orow + x) = pnew;
        else
          orow[x] = pnew.x;
      }
    }
    __syncthreads();
    // 3. this step's source increments on the band's nodes
    if (tap_off >= 0) atomicAdd(&Po[tap_off], tap_coef * sig_n);
    // 4. p[n+1] complete in every band
    cluster.sync();
    cur ^= 1;
  }
  if (run.n_steps > 0) sample(cur, run.n_steps - 1);
  // the last two levels back to the padded layout: p[n_steps] into
  // u[n_steps & 1], p[n_steps - 1] into the other (node values only)
  float* dst_cur = run.u[run.n_steps & 1];
  float* dst_old = run.u[(run.n_steps + 1) & 1];
  for (int r = warp; r < nb; r += NW) {
    const int64_t g = int64_t(z0 + r) * sz;
    for (int x = lane; x < nx; x += 32) {
      dst_cur[g + x] = level(cur)[(r + R) * W + X0 + x];
      dst_old[g + x] = level(cur ^ 1)[(r + R) * W + X0 + x];
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

}  // namespace sw
