// C ABI of the solver (declared in include/simwave_b300.h).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/simwave_b300.h"
#include "aux_kernels.cuh"
#include "host_setup.h"
#include "layout.h"
#include "cluster2d.cuh"
#include "stencil_plain.cuh"
#include "stencil_tma.cuh"
#include "tb2d.cuh"

using namespace sw;

namespace {

thread_local std::string g_last_error;

sw_status fail(sw_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define SW_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
  } while (0)

#define SW_TRY(expr)              \
  do {                            \
    sw_status s_ = (expr);        \
    if (s_ != SW_OK) return s_;   \
  } while (0)

// Can kernels on the current device use p directly?  Device memory of the
// current device, or managed memory.  Host memory and device memory of
// another GPU are not: callers stage those through a buffer of their own
// with cudaMemcpyDefault copies (which reach either).
bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Is p plain device memory (not managed, not host) of the current device?
bool is_current_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Is p device or managed memory of another device than the current one?
bool is_other_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.device != dev;
}

int grid_blocks(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 148 * 32) b = 148 * 32;
  return int(b < 1 ? 1 : b);
}

}  // namespace

struct sw_grid {
  int ndim = 0;
  int64_t n[3] = {1, 1, 1};  // nz, ny, nx
  double h[3] = {1, 1, 1};
  int order = 0, R = 0;
  int nbl[6] = {0, 0, 0, 0, 0, 0};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  double alpha = 0.0;
  int degree = 0;
  double dt_user = 0.0, dt = 0.0;
  bool dt_ready = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  Layout lay;

  float* u[2] = {nullptr, nullptr};
  // two more levels for the two-step 2D kernel (SW_STENCIL_TB2), allocated on
  // first use, and its tensor maps over the four levels (as p[n] and as
  // p[n-1]) and kappa
  float* u2[2] = {nullptr, nullptr};
  bool tb2_ready = false;
  CUtensorMap tb2_n[4], tb2_m[4], tb2_k;
  float* kappa = nullptr;
  float* lnrho = nullptr;
  float2* damp = nullptr;
  int64_t damp_len = 0;
  int* dflag = nullptr;        // device error flag
  unsigned* dscratch = nullptr;  // reduction results
  bool has_model = false, has_density = false;
  double c_max = 0.0;

  float* staging = nullptr;  // dense grid-sized buffer for host inputs/outputs
  float* staging2 = nullptr;
  float* seis_staging = nullptr;
  int64_t seis_staging_elems = 0;

  // acquisition
  bool has_acq = false;
  int n_src = 0, n_rec = 0, nt = 0, rw = 0, L = 0, lz = 1, ly = 1, lx = 1;
  int sig_stride = 0;
  int* src_first = nullptr;
  float* src_w = nullptr;
  float* wavelet = nullptr;
  // per time step: does some source have a nonzero sample?  (The injection
  // and source-imaging launches of steps where every sample is exactly zero,
  // the tail of a Ricker wavelet in FP32, add nothing and are skipped.)
  std::vector<uint8_t> sig_live;
  bool live(int n) const { return n >= 0 && size_t(n) < sig_live.size() && sig_live[size_t(n)]; }
  int64_t* tap_off = nullptr;  // source tap table of the pipelined path (n_src * taps)
  float* tap_coef = nullptr;
  float* tap_pre = nullptr;  // pre-injection coefficients (PreInject), same order
  int64_t src_d2_max = 0;    // largest squared layer distance of a source window node
  int* rec_first = nullptr;
  float* rec_w = nullptr;
  int4* rec_span = nullptr;  // per receiver: rows with non-zero weight along z and y
  int rec_rows_max = 0;       // the largest such row count

  // TMA tensor maps of the 3D pipelined stencil: p[n] with halo box and
  // interior box for each of the two wavefield buffers, kappa interior box
  int variant = SW_STENCIL_AUTO;
  int ckpt_budget = 0;  // sw_gradient: 0 uniform checkpoints, else at most this many stored states (binomial)
  bool tma_ready = false;
  bool starve = false;                               // failure-path test: no tensor copies
  unsigned long long wait_limit_ns = 2000000000ull;  // bound of every mbarrier wait
  int sm_count = 0;
  CUtensorMap map_halo[2], map_inner[2], map_warm[2], map_kappa;
  // variable density on the pipelined path: D_z, D_y, D_x ln(rho) fields and their maps
  float* glr[3] = {nullptr, nullptr, nullptr};
  CUtensorMap map_g[3];
  // 64 x 32 tiles of the variable-density forward at radius 8: maps of both
  // levels, kappa and the ln rho gradient fields
  bool tall_ready = false;
  CUtensorMap tall_halo[2], tall_inner[2], tall_warm[2], tall_kappa, tall_g[3];
  bool grad_ready = false;

  // distributed forcing (sw_set_forcing): dense fields and signatures
  int n_force = 0, force_len = 0;
  float* force_F = nullptr;
  float* force_T = nullptr;
  // initial levels p[0], p[-1] (sw_set_initial_state), dense, or NULL for 0
  float* init_p0 = nullptr;
  float* init_pm1 = nullptr;
  // wavefield snapshots written by sw_forward (sw_set_saving)
  int saving_stride = 0;
  float* snapshots = nullptr;
  int64_t snapshot_frames = 0;
  // profiling
  int profiling = 0;  // time every profiling-th stencil launch (0: none)
  // the time loop of sw_forward as a CUDA graph: captured on the second call
  // with an unchanged configuration, replayed while it stays unchanged
  uint64_t config_gen = 0;  // bumped by every call that changes what sw_forward launches
  struct ForwardKey {
    int n_steps = -1;
    const float* seis = nullptr;
    int profiling = 0;
    bool tma = false;
    uint64_t gen = 0;
    bool operator==(const ForwardKey& o) const {
      return n_steps == o.n_steps && seis == o.seis && profiling == o.profiling && tma == o.tma && gen == o.gen;
    }
  };
  ForwardKey last_key, graph_key;
  bool last_key_valid = false;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_launches = 0;
  cudaStream_t cap_stream = nullptr;  // private stream used only for capturing
  std::vector<cudaEvent_t> events;
  double stencil_ms = 0.0;
  int64_t stencil_launches = 0, kernel_launches = 0;
  int64_t device_bytes = 0;

  FaceInfo faces() const {
    FaceInfo f;
    f.sz = lay.sz;
    f.sy = lay.sy;
    f.nz = int(n[0]);
    f.ny = int(n[1]);
    f.nx = int(n[2]);
    for (int i = 0; i < 6; ++i) {
      f.nbl[i] = nbl[i];
      f.bc[i] = bc[i];
    }
    return f;
  }
  int64_t nodes() const { return n[0] * n[1] * n[2]; }
  float* at0(float* base) const { return base + lay.origin; }
};

namespace {

sw_status dev_alloc(sw_grid* g, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(SW_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  g->device_bytes += int64_t(bytes);
  return SW_OK;
}

void dev_free(sw_grid* g, void* p, size_t bytes) {
  if (p) {
    cudaFree(p);
    g->device_bytes -= int64_t(bytes);
  }
}

// Copies a grid-shaped input to the device if it lives on the host; returns the
// device pointer to read from.
sw_status device_input(sw_grid* g, const float* src, float** staging, const float** out) {
  if (is_device_pointer(src)) {
    *out = src;
    return SW_OK;
  }
  const size_t bytes = size_t(g->nodes()) * sizeof(float);
  if (!*staging) SW_TRY(dev_alloc(g, (void**)staging, bytes));
  SW_CUDA(cudaMemcpyAsync(*staging, src, bytes, cudaMemcpyDefault, g->stream));  // host or another GPU
  *out = *staging;
  return SW_OK;
}

// ---- stencil dispatch --------------------------------------------------------

StencilArgs stencil_args(const sw_grid* g) {
  StencilArgs a;
  memset(&a, 0, sizeof(a));
  a.sz = g->lay.sz;
  a.sy = g->lay.sy;
  a.nz = int(g->n[0]);
  a.ny = int(g->n[1]);
  a.nx = int(g->n[2]);
  for (int i = 0; i < 6; ++i) {
    a.nbl[i] = g->nbl[i];
    a.bc[i] = g->bc[i];
  }
  double v[kMaxR + 1], w[kMaxR + 1];
  fd_second_weights(g->order, v);
  fd_first_weights(g->order, w);
  const double hz = g->h[0], hy = g->h[1], hx = g->h[2];
  for (int j = 1; j <= g->R; ++j) {
    a.cz[j] = float(v[j] / (hz * hz));
    a.cy[j] = float(v[j] / (hy * hy));
    a.cx[j] = float(v[j] / (hx * hx));
    a.gz[j] = float(w[j] / (2.0 * hz));
    a.gy[j] = float(w[j] / (2.0 * hy));
    a.gx[j] = float(w[j] / (2.0 * hx));
  }
  a.damp = g->damp;
  a.kappa = g->at0(g->kappa);
  a.lnrho = g->has_density ? g->at0(g->lnrho) : nullptr;
  return a;
}

template <int R, int NDIM, bool VD>
void launch_stencil_t(StencilArgs a, cudaStream_t st) {
  if constexpr (NDIM == 3) {
    constexpr int TX = 32, TY = 16;
    constexpr int PPT = (VD || R > 5) ? 2 : 4;
    const int tiles_x = (a.nx + TX - 1) / TX, tiles_y = (a.ny + TY - 1) / TY;
    const int target = 148 * 4;
    int chunks = (target + tiles_x * tiles_y - 1) / (tiles_x * tiles_y);
    int zc = (a.nz + chunks - 1) / chunks;
    if (zc < 4 * R) zc = 4 * R;
    a.zchunk = zc;
    dim3 grid(tiles_x, tiles_y, (a.nz + zc - 1) / zc);
    stencil_plain_kernel<R, 3, VD, TX, TY, PPT><<<grid, TX * (TY / PPT), 0, st>>>(a);
  } else {
    const dim3 grid((a.nx + 127) / 128, std::min(a.nz, 65535));  // one thread per node
    launch_dependent(stencil_2d_kernel<R, VD>, grid, dim3(128), 0, st, a);  // waits for the previous step
  }
}

template <int R>
void launch_stencil_r(int ndim, bool vd, const StencilArgs& a, cudaStream_t st) {
  if (ndim == 3) {
    if (vd)
      launch_stencil_t<R, 3, true>(a, st);
    else
      launch_stencil_t<R, 3, false>(a, st);
  } else {
    if (vd)
      launch_stencil_t<R, 2, true>(a, st);
    else
      launch_stencil_t<R, 2, false>(a, st);
  }
}

void launch_stencil(int R, int ndim, bool vd, const StencilArgs& a, cudaStream_t st) {
  switch (R) {
    case 1: launch_stencil_r<1>(ndim, vd, a, st); break;
    case 2: launch_stencil_r<2>(ndim, vd, a, st); break;
    case 3: launch_stencil_r<3>(ndim, vd, a, st); break;
    case 4: launch_stencil_r<4>(ndim, vd, a, st); break;
    case 5: launch_stencil_r<5>(ndim, vd, a, st); break;
    case 6: launch_stencil_r<6>(ndim, vd, a, st); break;
    case 7: launch_stencil_r<7>(ndim, vd, a, st); break;
    case 8: launch_stencil_r<8>(ndim, vd, a, st); break;
    case 9: launch_stencil_r<9>(ndim, vd, a, st); break;
    case 10: launch_stencil_r<10>(ndim, vd, a, st); break;
    default: break;
  }
}

// ---- TMA pipelined 3D stencil ------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Tile shape of the pipelined kernel per stencil radius (must match the
// instantiations in launch_stencil_tma_maps; the 64 x 32 tiles of the
// variable-density forward have maps of their own).
void tma_tile(int R, int* tx, int* ty) {
  *tx = 64;
  *ty = 16;
  (void)R;
}

sw_status make_map(const sw_grid* g, float* base, uint32_t box_x, uint32_t box_y, CUtensorMap* map,
                   uint32_t box_z = 1) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(SW_ECUDA, "cuTensorMapEncodeTiled is not available");
  const Layout& L = g->lay;
  cuuint64_t dims[3] = {cuuint64_t(L.pitch), cuuint64_t(L.py), cuuint64_t(L.pz)};
  cuuint64_t strides[2] = {cuuint64_t(L.sy) * 4, cuuint64_t(L.sz) * 4};
  cuuint32_t box[3] = {box_x, box_y, box_z};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
  return SW_OK;
}

sw_status build_tma_maps(sw_grid* g) {
  int tx, ty;
  tma_tile(g->R, &tx, &ty);
  const uint32_t xh = uint32_t((g->R + 3) / 4 * 4);
  for (int i = 0; i < 2; ++i) {
    SW_TRY(make_map(g, g->u[i], uint32_t(tx) + 2 * xh, uint32_t(ty + 2 * g->R), &g->map_halo[i]));
    SW_TRY(make_map(g, g->u[i], uint32_t(tx), uint32_t(ty), &g->map_inner[i]));
    SW_TRY(make_map(g, g->u[i], uint32_t(tx), uint32_t(ty), &g->map_warm[i], kTmaWarmPlanes));
  }
  SW_TRY(make_map(g, g->kappa, uint32_t(tx), uint32_t(ty), &g->map_kappa));
  g->tma_ready = true;
  return SW_OK;
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // default bound of an mbarrier wait (2 s)

// Tensor maps of one stencil launch: p[n] with halo and interior, p[n-1]
// interior, p[n] warm-up boxes (kTmaWarmPlanes interior planes).
struct StepMaps {
  const CUtensorMap* halo;
  const CUtensorMap* inner;
  const CUtensorMap* old;
  const CUtensorMap* warm;
  bool tall = false;
  const CUtensorMap* kap = nullptr;  // replaces kappa's map (the imaging pass: gk)  // 64 x 32 tiles (variable density, radius 8; the tall_* maps)
};

template <int R, int TY, int PPT, int NB, int MINB, bool ISO, bool VD, bool IMG = false>
void launch_tma_iso(const sw_grid* g, const StencilArgs& a, const StepMaps& m, cudaStream_t st) {
  using C = TmaConfig<R, TY, PPT, NB, VD>;
  auto kern = stencil_tma_kernel<R, TY, PPT, NB, MINB, ISO, VD, IMG>;
  static int blocks_per_sm = 0;  // per instantiation; the library drives one device type
  if (!blocks_per_sm) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, C::NT, C::SMEM);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  TmaWork wk;
  wk.tiles_x = (a.nx + C::TX - 1) / C::TX;
  const int tiles_y = (a.ny + TY - 1) / TY;
  wk.nz = a.nz;
  wk.total = wk.tiles_x * tiles_y * a.nz;  // < 2^31: checked in use_tma
  wk.starve = g->starve ? 1 : 0;
  long long grid = (long long)g->sm_count * blocks_per_sm;
  if (grid > wk.total) grid = wk.total;
  const CUtensorMap* gm = VD ? (m.tall ? g->tall_g : g->map_g) : nullptr;  // unused maps: kappa's
  const CUtensorMap& km = m.kap ? *m.kap : (m.tall ? g->tall_kappa : g->map_kappa);
  launch_dependent(kern, dim3(unsigned(grid)), dim3(C::NT), C::SMEM, st, *m.halo, *m.inner, *m.warm, *m.old, km,
                   VD ? gm[0] : km, VD ? gm[1] : km, VD ? gm[2] : km, a, wk, g->dflag, g->wait_limit_ns);
}

template <int R, int TY, int PPT, int NB, int MINB, bool VD, bool IMG = false>
void launch_tma_t(const sw_grid* g, const StencilArgs& a, const StepMaps& m, cudaStream_t st) {
  if (g->h[0] == g->h[1] && g->h[1] == g->h[2])
    launch_tma_iso<R, TY, PPT, NB, MINB, true, VD, IMG>(g, a, m, st);
  else
    launch_tma_iso<R, TY, PPT, NB, MINB, false, VD, IMG>(g, a, m, st);
}

// The imaging pass of the gradient (constant density) on the pipelined
// kernel: m.halo/inner/warm over the forward state p, m.old over psi, m.kap
// over gk; a.pout = gk.  The tile shapes of the constant-density forward.
void launch_image_tma(const sw_grid* g, const StencilArgs& a, const StepMaps& m, cudaStream_t st) {
  switch (g->R) {
    case 1: launch_tma_t<1, 16, 4, 3, 3, false, true>(g, a, m, st); break;
    case 2: launch_tma_t<2, 16, 4, 3, 3, false, true>(g, a, m, st); break;
    case 3: launch_tma_t<3, 16, 4, 3, 3, false, true>(g, a, m, st); break;
    case 4: launch_tma_t<4, 16, 4, 3, 3, false, true>(g, a, m, st); break;
    case 5: launch_tma_t<5, 16, 2, 4, 2, false, true>(g, a, m, st); break;
    case 6: launch_tma_t<6, 16, 2, 4, 2, false, true>(g, a, m, st); break;
    case 7: launch_tma_t<7, 16, 2, 4, 1, false, true>(g, a, m, st); break;
    case 8: launch_tma_t<8, 16, 2, 4, 1, false, true>(g, a, m, st); break;
    case 9: launch_tma_t<9, 16, 2, 4, 1, false, true>(g, a, m, st); break;
    case 10: launch_tma_t<10, 16, 2, 4, 1, false, true>(g, a, m, st); break;
    default: break;
  }
}

// Tile height / rows per warp / ring depth / minimum CTAs per SM for each
// radius (tile width 64), constant and variable density.  tma_tile() gives
// the tile shape of every launch here except the 64 x 32 tiles (m.tall),
// whose maps sw_set_model builds separately.  Radii up to 4: four rows per
// thread in 4-warp CTAs, three per SM, three bundles in flight each
// (fastest on the order-8 bench workload: 70.8 against 80.2 us for two rows
// per thread in 8-warp CTAs; three rows in four CTAs per SM, six rows on
// 64 x 24 and eight rows on 64 x 32 tiles were slower too); larger radii
// keep two rows per thread (four would spill).  Variable density: four rows
// per thread in 4-warp CTAs with three bundles (730 against 863 us per
// launch at order 16 on 512 x 512 x 384 for two rows in 8-warp CTAs) up to
// radius 8, two rows in 8-warp CTAs above; the radius-8 forward uses 64 x 32
// tiles in one 8-warp CTA per SM.
void launch_stencil_tma_maps(const sw_grid* g, const StencilArgs& a, const StepMaps& m, cudaStream_t st,
                             bool vd) {
  if (vd && m.tall && g->R == 8) {
    // one CTA of 8 warps per SM on 64 x 32 tiles: the same 8 warps per SM as
    // two CTAs on 64 x 16 tiles, 1.5 instead of 2 centre-box rows per output
    // row, and half the tile boundaries whose halo rows come back from DRAM
    // (3d_vd_512x512x384: 128.9 -> 141.0 Gpts/s)
    launch_tma_t<8, 32, 4, 3, 1, true>(g, a, m, st);
    return;
  }
  if (vd) {
    switch (g->R) {
      case 1: launch_tma_t<1, 16, 4, 3, 1, true>(g, a, m, st); break;
      case 2: launch_tma_t<2, 16, 4, 3, 1, true>(g, a, m, st); break;
      case 3: launch_tma_t<3, 16, 4, 3, 1, true>(g, a, m, st); break;
      case 4: launch_tma_t<4, 16, 4, 3, 1, true>(g, a, m, st); break;
      case 5: launch_tma_t<5, 16, 4, 3, 1, true>(g, a, m, st); break;
      case 6: launch_tma_t<6, 16, 4, 3, 1, true>(g, a, m, st); break;
      case 7: launch_tma_t<7, 16, 4, 3, 1, true>(g, a, m, st); break;
      case 8: launch_tma_t<8, 16, 4, 3, 1, true>(g, a, m, st); break;
      case 9: launch_tma_t<9, 16, 2, 5, 1, true>(g, a, m, st); break;
      case 10: launch_tma_t<10, 16, 2, 5, 1, true>(g, a, m, st); break;
      default: break;
    }
    return;
  }
  switch (g->R) {
    case 1: launch_tma_t<1, 16, 4, 3, 3, false>(g, a, m, st); break;
    case 2: launch_tma_t<2, 16, 4, 3, 3, false>(g, a, m, st); break;
    case 3: launch_tma_t<3, 16, 4, 3, 3, false>(g, a, m, st); break;
    case 4: launch_tma_t<4, 16, 4, 3, 3, false>(g, a, m, st); break;
    case 5: launch_tma_t<5, 16, 2, 4, 2, false>(g, a, m, st); break;
    case 6: launch_tma_t<6, 16, 2, 4, 2, false>(g, a, m, st); break;
    case 7: launch_tma_t<7, 16, 2, 4, 1, false>(g, a, m, st); break;
    case 8: launch_tma_t<8, 16, 2, 4, 1, false>(g, a, m, st); break;
    case 9: launch_tma_t<9, 16, 2, 4, 1, false>(g, a, m, st); break;
    case 10: launch_tma_t<10, 16, 2, 4, 1, false>(g, a, m, st); break;
    default: break;
  }
}

// The time loop's step: p[n] in u[buf], p[n-1] and p[n+1] in u[buf ^ 1].
void launch_stencil_tma(const sw_grid* g, const StencilArgs& a, int buf, cudaStream_t st) {
  if (g->has_density && g->tall_ready) {  // variable density, radius 8: 64 x 32 tiles
    StepMaps m{&g->tall_halo[buf], &g->tall_inner[buf], &g->tall_inner[buf ^ 1], &g->tall_warm[buf]};
    m.tall = true;
    launch_stencil_tma_maps(g, a, m, st, true);
    return;
  }
  const StepMaps m{&g->map_halo[buf], &g->map_inner[buf], &g->map_inner[buf ^ 1], &g->map_warm[buf]};
  launch_stencil_tma_maps(g, a, m, st, g->has_density);
}

void launch_image(int R, int ndim, dim3 grid, const float* p, const float* psi, float* gk, const FaceInfo& f,
                  const LapCoef& lc, cudaStream_t st) {
#define SW_IMAGE(RR)                                                                            \
  case RR:                                                                                       \
    if (ndim == 3)                                                                               \
      launch_dependent(image_kernel<RR, 3>, grid, dim3(128), 0, st, p, psi, gk, f, lc);                              \
    else                                                                                         \
      launch_dependent(image_kernel<RR, 2>, grid, dim3(128), 0, st, p, psi, gk, f, lc);                              \
    break;
  switch (R) {
    SW_IMAGE(1) SW_IMAGE(2) SW_IMAGE(3) SW_IMAGE(4) SW_IMAGE(5)
    SW_IMAGE(6) SW_IMAGE(7) SW_IMAGE(8) SW_IMAGE(9) SW_IMAGE(10)
    default: break;
  }
#undef SW_IMAGE
}

void launch_image_vd(int R, int ndim, dim3 grid, const float* p, const float* psi, float* const* gg, float* gk,
                     float* const* ag, const FaceInfo& f, const LapCoef& lc, const VdWeights& w, cudaStream_t st) {
#define SW_IMAGE_VD(RR)                                                                                            \
  case RR:                                                                                                          \
    if (ndim == 3)                                                                                                  \
      launch_dependent(image_vd_kernel<RR, 3>, grid, dim3(128), 0, st, p, psi, gg[0], gg[1], gg[2], gk, ag[0], ag[1], ag[2], f,        \
                                                   lc, w);                                                          \
    else                                                                                                            \
      launch_dependent(image_vd_kernel<RR, 2>, grid, dim3(128), 0, st, p, psi, gg[0], gg[1], gg[2], gk, ag[0], ag[1], ag[2], f,        \
                                                   lc, w);                                                          \
    break;
  switch (R) {
    SW_IMAGE_VD(1) SW_IMAGE_VD(2) SW_IMAGE_VD(3) SW_IMAGE_VD(4) SW_IMAGE_VD(5)
    SW_IMAGE_VD(6) SW_IMAGE_VD(7) SW_IMAGE_VD(8) SW_IMAGE_VD(9) SW_IMAGE_VD(10)
    default: break;
  }
#undef SW_IMAGE_VD
}

bool use_tma(const sw_grid* g) {
  if (g->variant == SW_STENCIL_PLAIN) return false;
  // the pipelined kernel keeps in-plane offsets in 32 bits
  // and assumes every node is within R of at most one face per axis
  // and counts its (64 x 16 tile, plane) work items in 32 bits
  const int64_t m = 2 * int64_t(g->R) + 1;
  // (and the face-condition kernel numbers the lines of both sides of a face in 32 bits)
  const int64_t* n = g->lay.n;
  const int64_t items = (n[2] + 63) / 64 * ((n[1] + 15) / 16) * n[0];
  const int64_t lines = 2 * std::max(n[0] * n[1] * int64_t(g->R), std::max(n[0] * n[2], n[1] * n[2]));
  return g->ndim == 3 && (!g->has_density || g->grad_ready) && g->tma_ready && g->lay.sz < (int64_t(1) << 31) && n[0] > m &&
         n[1] > m && n[2] > m && items < (int64_t(1) << 31) && lines < (int64_t(1) << 31);
}

// ---- two-step 2D kernel (temporal blocking) ---------------------------------

// The two-step kernel runs 2D constant-density grids without distributed
// forcing or snapshot frames (those need every level): when asked for, and by
// default from 4M nodes on, where the fields no longer stay in L2 (measured
// against the per-step kernels: 1024^2 61.3 vs 84.8 Gpts/s, 2048^2 125.5 vs
// 111.5, 4096^2 164.5 vs 118.6).
constexpr int64_t kTb2AutoNodes = int64_t(1) << 22;
bool use_tb2(const sw_grid* g) {
  const bool asked = g->variant == SW_STENCIL_TB2 ||
                     (g->variant == SW_STENCIL_AUTO && g->n[0] * g->n[2] >= kTb2AutoNodes);
  return asked && g->ndim == 2 && !g->has_density && g->n_force == 0 && !g->snapshots &&
         g->n[0] > 2 * int64_t(g->R) + 1 && g->n[2] > 2 * int64_t(g->R) + 1;
}

using Tb2Fn = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const Tb2Args, int*,
                      unsigned long long);

// The kernel of a radius with its shared memory set up, and its resident
// CTAs per SM (once per radius).
template <int R>
Tb2Fn tb2_fn(int* per_sm) {
  static int blocks = 0;
  if (!blocks) {
    cudaFuncSetAttribute(tb2_2d_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Tb2Cfg<R>::BYTES));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, tb2_2d_kernel<R>, kTb2Threads, Tb2Cfg<R>::BYTES);
    if (blocks < 1) blocks = 1;
  }
  *per_sm = blocks;
  return tb2_2d_kernel<R>;
}

void launch_tb2(const sw_grid* g, const CUtensorMap& mn, const CUtensorMap& mm, const Tb2Args& t, cudaStream_t st) {
#define SW_TB2(RR)                                                                                              \
  case RR: {                                                                                                    \
    int per_sm = 1;                                                                                             \
    Tb2Fn fn = tb2_fn<RR>(&per_sm);                                                                             \
    const unsigned grid = unsigned(std::min<int64_t>(t.tiles, int64_t(g->sm_count) * per_sm));                 \
    launch_dependent(fn, dim3(grid), dim3(kTb2Threads), Tb2Cfg<RR>::BYTES, st, mn, mm, g->tb2_k, t, g->dflag,  \
                     g->wait_limit_ns);                                                                         \
    break;                                                                                                      \
  }
  switch (g->R) {
    SW_TB2(1) SW_TB2(2) SW_TB2(3) SW_TB2(4) SW_TB2(5) SW_TB2(6) SW_TB2(7) SW_TB2(8) SW_TB2(9) SW_TB2(10)
    default: break;
  }
#undef SW_TB2
}

// Tensor maps of the two-step kernel over the four level buffers and kappa.
sw_status build_tb2_maps(sw_grid* g) {
  int w0, h0, w1, h1;
  tb2_boxes(g->R, &w0, &h0, &w1, &h1);
  float* lv[4] = {g->u[0], g->u[1], g->u2[0], g->u2[1]};
  for (int i = 0; i < 4; ++i) {
    SW_TRY(make_map(g, lv[i], uint32_t(w0), 1, &g->tb2_n[i], uint32_t(h0)));
    SW_TRY(make_map(g, lv[i], uint32_t(w1), 1, &g->tb2_m[i], uint32_t(h1)));
  }
  SW_TRY(make_map(g, g->kappa, uint32_t(w1), 1, &g->tb2_k, uint32_t(h1)));
  g->tb2_ready = true;
  return SW_OK;
}

// Level buffers of a two-step run after `n_steps` steps: the run reads
// (u0, u1), writes (u2a, u2b), reads those, writes (u0, u1), ...; an odd
// last step runs in place over the older of the two current levels.
// Returns the index (0, 1: u, 2, 3: u2) of the buffer holding p[n_steps].
int tb2_last_level(int n_steps) {
  const int pairs = n_steps / 2;
  const int in_n = pairs == 0 ? 0 : (pairs % 2 ? 3 : 1), in_m = pairs == 0 ? 1 : (pairs % 2 ? 2 : 0);
  return n_steps % 2 ? in_m : in_n;
}

// ---- cluster-resident 2D forward run -----------------------------------------

using ClusterFn = void (*)(const ClusterRun);

ClusterFn cluster_kernel(int R) {
  switch (R) {
    case 1: return stencil_2d_cluster_kernel<1>;
    case 2: return stencil_2d_cluster_kernel<2>;
    case 3: return stencil_2d_cluster_kernel<3>;
    case 4: return stencil_2d_cluster_kernel<4>;
    case 5: return stencil_2d_cluster_kernel<5>;
    case 6: return stencil_2d_cluster_kernel<6>;
    case 7: return stencil_2d_cluster_kernel<7>;
    case 8: return stencil_2d_cluster_kernel<8>;
    case 9: return stencil_2d_cluster_kernel<9>;
    case 10: return stencil_2d_cluster_kernel<10>;
    default: return nullptr;
  }
}

// Launch shape of the cluster-resident run: CTAs in the cluster, rows per
// band, shared row length and bytes per CTA.
struct ClusterShape {
  int C = 0, B = 0, W = 0;
  size_t smem = 0;
};

// Can the whole run of this grid live in one cluster's shared memory?  2D,
// constant density, no distributed forcing and no snapshot frames (those
// run per step); the largest cluster (16, 8, 4 or 2 CTAs) whose bands fit
// the per-CTA shared memory and that the device can place.  Every band
// holds at least one row.
bool use_cluster(const sw_grid* g, ClusterShape* out) {
  if (g->ndim != 2 || g->has_density || g->n_force > 0 || g->snapshots || g->variant == SW_STENCIL_PLAIN ||
      g->variant == SW_STENCIL_TB2)
    return false;
  if (int64_t(g->n_src) * g->lz * g->lx > kClusterThreads) return false;  // one source tap per thread
  const int R = g->R;
  const int64_t nz = g->n[0], nx = g->n[2];
  if (nz <= 2 * R + 1 || nx <= 2 * R + 1 || nx > (int64_t(1) << 20)) return false;
  ClusterFn fn = cluster_kernel(R);
  if (!fn) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int W = cluster_row_len(int(nx), R);
  for (int C = kClusterMaxCtas; C >= 2; C /= 2) {
    const int B = int((nz + C - 1) / C);
    const int Ce = int((nz + B - 1) / B);  // every band non-empty
    const size_t smem = size_t(cluster_smem_floats(B, int(nx), R)) * sizeof(float);
    if (smem > size_t(optin)) continue;
    if (cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(Ce));
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(Ce);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, (const void*)fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (clusters < 1) continue;
    out->C = Ce;
    out->B = B;
    out->W = W;
    out->smem = smem;
    return true;
  }
  return false;
}

PointSet point_set(const sw_grid* g, bool src) {
  PointSet p;
  p.first = src ? g->src_first : g->rec_first;
  p.w = src ? g->src_w : g->rec_w;
  p.count = src ? g->n_src : g->n_rec;
  p.L = g->L;
  p.lz = g->lz;
  p.ly = g->ly;
  p.lx = g->lx;
  p.span = src ? nullptr : g->rec_span;
  return p;
}

void free_acquisition(sw_grid* g) {
  const size_t ntaps = size_t(g->n_src) * g->lz * g->ly * g->lx;
  dev_free(g, g->tap_off, ntaps * sizeof(int64_t));
  dev_free(g, g->tap_coef, ntaps * sizeof(float));
  dev_free(g, g->tap_pre, ntaps * sizeof(float));
  g->tap_off = nullptr;
  g->tap_coef = nullptr;
  g->tap_pre = nullptr;
  dev_free(g, g->src_first, size_t(g->n_src) * 3 * sizeof(int));
  dev_free(g, g->src_w, size_t(g->n_src) * 3 * g->L * sizeof(float));
  dev_free(g, g->rec_first, size_t(g->n_rec) * 3 * sizeof(int));
  dev_free(g, g->rec_w, size_t(g->n_rec) * 3 * g->L * sizeof(float));
  dev_free(g, g->rec_span, size_t(g->n_rec) * sizeof(int4));
  g->rec_span = nullptr;
  g->rec_rows_max = 0;
  dev_free(g, g->wavelet, size_t(g->n_src > 0 ? g->n_src : 1) * g->nt * sizeof(float));
  g->src_first = g->rec_first = nullptr;
  g->src_w = g->rec_w = g->wavelet = nullptr;
  g->has_acq = false;
  g->sig_live.clear();
}

// Window weights of a set of points: per point and axis the first node and the
// 2 r_w Kaiser-sinc weights (a single unit weight along the absent 2D y axis).
sw_status build_windows(const sw_grid* g, int count, const double* pos, bool fold_cell,
                        std::vector<int>& first, std::vector<float>& w) {
  const int rw = g->rw, L = g->L;
  first.assign(size_t(count) * 3, 0);
  w.assign(size_t(count) * 3 * L, 0.f);
  double cell = 1.0;
  for (int a = 0; a < g->ndim; ++a) cell *= (g->ndim == 3 ? g->h[a] : (a == 0 ? g->h[0] : g->h[2]));
  for (int i = 0; i < count; ++i) {
    for (int a = 0; a < g->ndim; ++a) {
      const int axis = (g->ndim == 3) ? a : (a == 0 ? 0 : 2);
      const double coord = pos[size_t(i) * g->ndim + a];
      if (!std::isfinite(coord)) return fail(SW_EINVAL, "position %d is not finite", i);
      const double s = double(g->nbl[2 * axis]) + coord / g->h[axis];
      int64_t f0;
      double ww[2 * kMaxR], wf[2 * kMaxR];
      kaiser_sinc_weights(s, rw, &f0, ww);
      // A window that sticks out of the grid only with exactly-zero weights (an
      // on-grid coordinate near a face) is moved inside; nonzero weights keep
      // their nodes.
      const int64_t nax = g->n[axis];
      if (2 * rw > nax) return fail(SW_EINVAL, "window longer than axis %d", axis);
      const int64_t nf = std::min(std::max<int64_t>(f0, 0), nax - 2 * rw);
      for (int j = 0; j < 2 * rw; ++j) wf[j] = 0.0;
      for (int j = 0; j < 2 * rw; ++j) {
        const int64_t node = f0 + j;
        if (node >= nf && node < nf + 2 * rw)
          wf[node - nf] = ww[j];
        else if (ww[j] != 0.0)
          return fail(SW_EINVAL, "window of point %d leaves the grid along axis %d", i, axis);
      }
      first[size_t(i) * 3 + axis] = int(nf);
      for (int j = 0; j < 2 * rw; ++j) {
        double v = wf[j];
        if (fold_cell && axis == 2) v /= cell;
        w[(size_t(i) * 3 + axis) * L + j] = float(v);
      }
    }
    if (g->ndim == 2) {
      first[size_t(i) * 3 + 1] = 0;
      w[(size_t(i) * 3 + 1) * L] = 1.f;
    }
  }
  return SW_OK;
}

sw_status check_device_flag(sw_grid* g) {
  int flag = 0;
  SW_CUDA(cudaMemcpyAsync(&flag, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  SW_CUDA(cudaStreamSynchronize(g->stream));
  if (flag != 0) {
    SW_CUDA(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
    return fail(SW_ETIMEOUT, "device error flag 0x%x (bit 0: a bounded wait gave up; bit 1: a tensor-copy "
                             "buffer failed its alignment check)", flag);
  }
  return SW_OK;
}

}  // namespace

extern "C" {

const char* sw_last_error(void) { return g_last_error.c_str(); }

sw_status sw_create_grid(sw_grid** out, int ndim, const int64_t* shape, const double* spacing,
                         int space_order, const int* nbl, const int* bc, double damp_alpha,
                         int damp_degree, double dt, void* cuda_stream) {
  g_last_error.clear();
  if (!out || !shape || !spacing || !nbl || !bc) return fail(SW_EINVAL, "NULL argument");
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return fail(SW_EINVAL, "ndim must be 2 or 3 (got %d)", ndim);
  if (space_order < 2 || space_order > 2 * kMaxR || space_order % 2)
    return fail(SW_EINVAL, "space_order must be even in [2, 20] (got %d)", space_order);
  if (!(damp_alpha >= 0.0) || !std::isfinite(damp_alpha) || damp_degree < 0 || damp_degree > 16)
    return fail(SW_EINVAL, "damping parameters out of range");
  if (!std::isfinite(dt)) return fail(SW_EINVAL, "dt is not finite");
  const int R = space_order / 2;
  sw_grid* g = new sw_grid();
  g->ndim = ndim;
  g->order = space_order;
  g->R = R;
  for (int a = 0; a < ndim; ++a) {
    const int axis = (ndim == 3) ? a : (a == 0 ? 0 : 2);
    if (shape[a] < R + 1 || shape[a] > (int64_t(1) << 24)) {
      delete g;
      return fail(SW_EINVAL, "shape[%d] = %lld out of range (needs r+1 .. 2^24)", a, (long long)shape[a]);
    }
    if (!(spacing[a] > 0.0) || !std::isfinite(spacing[a])) {
      delete g;
      return fail(SW_EINVAL, "spacing[%d] must be positive", a);
    }
    g->n[axis] = shape[a];
    g->h[axis] = spacing[a];
    for (int s = 0; s < 2; ++s) {
      const int nb = nbl[2 * a + s], b = bc[2 * a + s];
      if (nb < 0 || nb >= shape[a]) {
        delete g;
        return fail(SW_EINVAL, "nbl[%d] out of range", 2 * a + s);
      }
      if (b != SW_BC_NONE && b != SW_BC_DIRICHLET && b != SW_BC_NEUMANN) {
        delete g;
        return fail(SW_EINVAL, "bc[%d] invalid", 2 * a + s);
      }
      g->nbl[2 * axis + s] = nb;
      g->bc[2 * axis + s] = b;
    }
    if (nbl[2 * a] + nbl[2 * a + 1] >= shape[a]) {
      delete g;
      return fail(SW_EINVAL, "absorbing layers cover the whole axis %d", a);
    }
  }
  const int64_t total_nodes = g->n[0] * g->n[1] * g->n[2];
  if (total_nodes > (int64_t(1) << 34)) {
    delete g;
    return fail(SW_EINVAL, "grid too large");
  }
  g->alpha = damp_alpha;
  g->degree = damp_degree;
  g->dt_user = dt;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&g->device);
  g->lay.init(ndim, R, g->n);

  sw_status st = SW_OK;
  const size_t fbytes = size_t(g->lay.total) * sizeof(float);
  for (int i = 0; i < 2 && st == SW_OK; ++i) st = dev_alloc(g, (void**)&g->u[i], fbytes);
  if (st == SW_OK) st = dev_alloc(g, (void**)&g->kappa, fbytes);
  if (st == SW_OK) st = dev_alloc(g, (void**)&g->dflag, 64);
  if (st == SW_OK) st = dev_alloc(g, (void**)&g->dscratch, 64);
  if (st == SW_OK) {
    int64_t maxd2 = 0;
    for (int a = 0; a < 3; ++a) {
      const int64_t m = std::max(g->nbl[2 * a], g->nbl[2 * a + 1]);
      maxd2 += m * m;
    }
    g->damp_len = maxd2 + 1;
    st = dev_alloc(g, (void**)&g->damp, size_t(g->damp_len) * sizeof(float2));
  }
  if (st == SW_OK) {
    cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    if (ndim == 3) st = build_tma_maps(g);
  }
  if (st == SW_OK) {
    cudaError_t e = cudaMemsetAsync(g->kappa, 0, fbytes, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->dflag, 0, 64, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) st = fail(SW_ECUDA, "initialisation failed: %s", cudaGetErrorString(e));
  }
  if (st != SW_OK) {
    std::string msg = g_last_error;
    sw_destroy_grid(g);
    g_last_error = msg;
    return st;
  }
  *out = g;
  return SW_OK;
}

sw_status sw_set_model(sw_grid* g, const float* velocity, const float* density) {
  g_last_error.clear();
  if (!g || !velocity) return fail(SW_EINVAL, "NULL argument");
  ++g->config_gen;
  const FaceInfo f = g->faces();
  const int64_t nn = g->nodes();
  const float* vdev = nullptr;
  SW_TRY(device_input(g, velocity, &g->staging, &vdev));
  // velocity range
  unsigned init[2] = {0u, 0x7f800000u};
  SW_CUDA(cudaMemcpyAsync(g->dscratch, init, sizeof(init), cudaMemcpyHostToDevice, g->stream));
  SW_CUDA(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
  field_range_kernel<<<grid_blocks(nn, 256), 256, 0, g->stream>>>(vdev, nn, g->dscratch, g->dscratch + 1,
                                                                  g->dflag);
  SW_CUDA(cudaGetLastError());
  unsigned res[2];
  int bad = 0;
  SW_CUDA(cudaMemcpyAsync(res, g->dscratch, sizeof(res), cudaMemcpyDeviceToHost, g->stream));
  SW_CUDA(cudaMemcpyAsync(&bad, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  SW_CUDA(cudaStreamSynchronize(g->stream));
  if (bad) {
    SW_CUDA(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
    return fail(SW_EINVAL, "velocity must be finite and positive everywhere");
  }
  float vmax;
  memcpy(&vmax, &res[0], sizeof(float));
  const double hh[3] = {g->h[0], g->ndim == 3 ? g->h[1] : g->h[2], g->h[2]};
  const double dtc = critical_dt(g->ndim, g->order, hh, double(vmax));
  double dt = g->dt_user;
  if (dt <= 0.0) {
    dt = dtc;
  } else if (dt > dtc) {
    return fail(SW_ECFL, "dt = %.6g s exceeds the stability bound %.6g s (c_max = %.6g m/s)", dt, dtc,
                double(vmax));
  }
  g->dt = dt;
  g->dt_ready = true;
  g->c_max = vmax;

  kappa_kernel<<<grid_blocks(nn, 256), 256, 0, g->stream>>>(vdev, g->at0(g->kappa), f, dt);
  SW_CUDA(cudaGetLastError());

  // damping coefficients by squared distance
  std::vector<float2> table(size_t(g->damp_len));
  for (int64_t d2 = 0; d2 < g->damp_len; ++d2) {
    double a, e;
    damping_coefficients(g->alpha, g->degree, dt, d2, &a, &e);
    table[size_t(d2)] = make_float2(float(a), float(e));
  }
  SW_CUDA(cudaMemcpyAsync(g->damp, table.data(), table.size() * sizeof(float2), cudaMemcpyHostToDevice,
                          g->stream));

  if (density) {
    const float* rdev = nullptr;
    SW_TRY(device_input(g, density, &g->staging2, &rdev));
    SW_CUDA(cudaMemcpyAsync(g->dscratch, init, sizeof(init), cudaMemcpyHostToDevice, g->stream));
    field_range_kernel<<<grid_blocks(nn, 256), 256, 0, g->stream>>>(rdev, nn, g->dscratch, g->dscratch + 1,
                                                                    g->dflag);
    SW_CUDA(cudaGetLastError());
    SW_CUDA(cudaMemcpyAsync(&bad, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    SW_CUDA(cudaStreamSynchronize(g->stream));
    if (bad) {
      SW_CUDA(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
      return fail(SW_EINVAL, "density must be finite and positive everywhere");
    }
    const size_t fbytes = size_t(g->lay.total) * sizeof(float);
    if (!g->lnrho) {
      SW_TRY(dev_alloc(g, (void**)&g->lnrho, fbytes));
      SW_CUDA(cudaMemsetAsync(g->lnrho, 0, fbytes, g->stream));
    }
    lnrho_kernel<<<grid_blocks(nn, 256), 256, 0, g->stream>>>(rdev, g->at0(g->lnrho), f);
    SW_CUDA(cudaGetLastError());
    for (int axis = 0; axis < 3; ++axis) {
      if (g->ndim == 2 && axis == 1) continue;
      mirror_even_kernel<<<grid_blocks(nn, 256), 256, 0, g->stream>>>(g->at0(g->lnrho), f, axis, g->R);
      SW_CUDA(cudaGetLastError());
    }
    if (g->ndim == 3 && g->tma_ready) {
      // ln(rho) gradient fields for the pipelined kernel (Eq. 10 weights, FP64 sums)
      for (int i = 0; i < 3; ++i)
        if (!g->glr[i]) {
          SW_TRY(dev_alloc(g, (void**)&g->glr[i], fbytes));
          SW_CUDA(cudaMemsetAsync(g->glr[i], 0, fbytes, g->stream));  // ghosts and padding stay zero
        }
      GradWeights gw;
      double wj[kMaxR + 1];
      fd_first_weights(g->order, wj);
      for (int j = 0; j <= kMaxR; ++j) {
        const bool in = j >= 1 && j <= g->R;
        gw.z[j] = in ? wj[j] / (2.0 * g->h[0]) : 0.0;
        gw.y[j] = in ? wj[j] / (2.0 * g->h[1]) : 0.0;
        gw.x[j] = in ? wj[j] / (2.0 * g->h[2]) : 0.0;
      }
      lnrho_gradient_kernel<<<grid_blocks(nn, 256), 256, 0, g->stream>>>(
          g->at0(g->lnrho), g->at0(g->glr[0]), g->at0(g->glr[1]), g->at0(g->glr[2]), f, gw, g->R);
      SW_CUDA(cudaGetLastError());
      int tx, ty;
      tma_tile(g->R, &tx, &ty);
      for (int i = 0; i < 3; ++i) SW_TRY(make_map(g, g->glr[i], uint32_t(tx), uint32_t(ty), &g->map_g[i]));
      if (g->R == 8) {  // the 64 x 32 tiles of the forward
        const uint32_t xh = 8, tt = 32;
        for (int i = 0; i < 2; ++i) {
          SW_TRY(make_map(g, g->u[i], uint32_t(tx) + 2 * xh, tt + 2 * 8, &g->tall_halo[i]));
          SW_TRY(make_map(g, g->u[i], uint32_t(tx), tt, &g->tall_inner[i]));
          SW_TRY(make_map(g, g->u[i], uint32_t(tx), tt, &g->tall_warm[i], kTmaWarmPlanes));
        }
        SW_TRY(make_map(g, g->kappa, uint32_t(tx), tt, &g->tall_kappa));
        for (int i = 0; i < 3; ++i) SW_TRY(make_map(g, g->glr[i], uint32_t(tx), tt, &g->tall_g[i]));
        g->tall_ready = true;
      }
      g->grad_ready = true;
    }
    g->has_density = true;
  } else {
    g->has_density = false;
  }
  SW_CUDA(cudaStreamSynchronize(g->stream));
  g->has_model = true;
  return SW_OK;
}

sw_status sw_set_acquisition(sw_grid* g, int n_src, const double* src_pos, int n_rec, const double* rec_pos,
                             int nt, const float* wavelet, int wavelet_per_source, int window_radius) {
  g_last_error.clear();
  if (!g) return fail(SW_EINVAL, "NULL grid");
  ++g->config_gen;
  if (n_src < 0 || n_rec < 0 || nt < 0) return fail(SW_EINVAL, "negative count");
  if ((n_src > 0 && (!src_pos || !wavelet || nt == 0)) || (n_rec > 0 && !rec_pos))
    return fail(SW_EINVAL, "NULL positions or wavelet");
  if (window_radius < 1 || window_radius > kMaxR) return fail(SW_EINVAL, "window_radius must be in [1, 10]");
  free_acquisition(g);
  g->rw = window_radius;
  g->L = 2 * window_radius;
  g->lz = g->L;
  g->ly = (g->ndim == 3) ? g->L : 1;
  g->lx = g->L;
  std::vector<int> sf, rf;
  std::vector<float> swt, rwt;
  SW_TRY(build_windows(g, n_src, src_pos, true, sf, swt));
  SW_TRY(build_windows(g, n_rec, rec_pos, false, rf, rwt));
  g->n_src = n_src;
  g->n_rec = n_rec;
  g->nt = nt;
  g->src_d2_max = 0;  // the window nodes deepest in the absorbing layers (per axis, a window end)
  for (int i = 0; i < n_src; ++i) {
    int64_t d2 = 0;
    for (int a = 0; a < 3; ++a) {
      if (g->ndim == 2 && a == 1) continue;
      const int lo = g->nbl[2 * a], hi = g->nbl[2 * a + 1];
      const int64_t n0 = sf[size_t(i) * 3 + a], n1 = n0 + 2 * window_radius - 1;
      const int64_t d = std::max<int64_t>({lo - n0, n1 - (g->n[a] - 1 - hi), 0});
      d2 += d * d;
    }
    g->src_d2_max = std::max(g->src_d2_max, d2);
  }
  g->sig_stride = wavelet_per_source ? nt : 0;
  if (n_src > 0) {
    SW_TRY(dev_alloc(g, (void**)&g->src_first, sf.size() * sizeof(int)));
    SW_TRY(dev_alloc(g, (void**)&g->src_w, swt.size() * sizeof(float)));
    SW_CUDA(cudaMemcpyAsync(g->src_first, sf.data(), sf.size() * sizeof(int), cudaMemcpyHostToDevice, g->stream));
    SW_CUDA(cudaMemcpyAsync(g->src_w, swt.data(), swt.size() * sizeof(float), cudaMemcpyHostToDevice, g->stream));
    const size_t wl = size_t(wavelet_per_source ? n_src : 1) * nt;
    SW_TRY(dev_alloc(g, (void**)&g->wavelet, size_t(n_src) * nt * sizeof(float)));
    SW_CUDA(cudaMemcpyAsync(g->wavelet, wavelet, wl * sizeof(float), cudaMemcpyDefault, g->stream));
    std::vector<float> host_w(wl);
    SW_CUDA(cudaMemcpyAsync(host_w.data(), g->wavelet, wl * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    SW_CUDA(cudaStreamSynchronize(g->stream));
    g->sig_live.assign(size_t(nt), 0);
    for (size_t i = 0; i < wl; ++i)
      if (host_w[i] != 0.f) g->sig_live[i % size_t(nt)] = 1;
  }
  if (n_rec > 0) {
    SW_TRY(dev_alloc(g, (void**)&g->rec_first, rf.size() * sizeof(int)));
    SW_TRY(dev_alloc(g, (void**)&g->rec_w, rwt.size() * sizeof(float)));
    SW_CUDA(cudaMemcpyAsync(g->rec_first, rf.data(), rf.size() * sizeof(int), cudaMemcpyHostToDevice, g->stream));
    SW_CUDA(cudaMemcpyAsync(g->rec_w, rwt.data(), rwt.size() * sizeof(float), cudaMemcpyHostToDevice, g->stream));
    // rows of each window with a non-zero weight along z and y (the sampler reads only those)
    std::vector<int4> span(static_cast<size_t>(n_rec));
    for (int i = 0; i < n_rec; ++i) {
      int lo[2], cnt[2];
      const int len[2] = {g->lz, g->ly};
      for (int k = 0; k < 2; ++k) {
        const float* wk = rwt.data() + (size_t(i) * 3 + k) * g->L;
        int a = 0, b = len[k];
        while (a < b - 1 && wk[a] == 0.f) ++a;
        while (b - 1 > a && wk[b - 1] == 0.f) --b;
        lo[k] = a;
        cnt[k] = b - a;
      }
      span[size_t(i)] = make_int4(lo[0], cnt[0], lo[1], cnt[1]);
      g->rec_rows_max = std::max(g->rec_rows_max, cnt[0] * cnt[1]);
    }
    SW_TRY(dev_alloc(g, (void**)&g->rec_span, span.size() * sizeof(int4)));
    SW_CUDA(cudaMemcpyAsync(g->rec_span, span.data(), span.size() * sizeof(int4), cudaMemcpyHostToDevice, g->stream));
  }
  SW_CUDA(cudaStreamSynchronize(g->stream));
  g->has_acq = true;
  return SW_OK;
}

sw_status sw_forward(sw_grid* g, int n_steps, float* seismogram, float* final_field) {
  g_last_error.clear();
  if (!g) return fail(SW_EINVAL, "NULL grid");
  if (!g->has_model) return fail(SW_ESTATE, "sw_forward before sw_set_model");
  if (!g->has_acq) return fail(SW_ESTATE, "sw_forward before sw_set_acquisition");
  if (n_steps < 0) return fail(SW_EINVAL, "n_steps < 0");
  if (g->n_src > 0 && n_steps > g->nt) return fail(SW_EINVAL, "n_steps (%d) exceeds the wavelet length (%d)", n_steps, g->nt);
  if (g->n_rec > 0 && n_steps > 0 && !seismogram) return fail(SW_EINVAL, "seismogram is NULL");
  if (g->n_force > 0 && n_steps > g->force_len)
    return fail(SW_EINVAL, "n_steps (%d) exceeds the forcing signatures (%d)", n_steps, g->force_len);

  const FaceInfo f = g->faces();
  const size_t fbytes = size_t(g->lay.total) * sizeof(float);
  SW_CUDA(cudaMemsetAsync(g->u[0], 0, fbytes, g->stream));
  SW_CUDA(cudaMemsetAsync(g->u[1], 0, fbytes, g->stream));
  if (g->init_p0)
    insert_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, g->stream>>>(g->init_p0, g->at0(g->u[0]), f, g->ndim, g->R);
  if (g->init_pm1)
    insert_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, g->stream>>>(g->init_pm1, g->at0(g->u[1]), f, g->ndim,
                                                                       g->R);
  SW_CUDA(cudaGetLastError());

  float* seis_dev = nullptr;
  const bool seis_host = seismogram && !is_device_pointer(seismogram);
  const int64_t seis_elems = int64_t(n_steps) * g->n_rec;
  if (g->n_rec > 0 && n_steps > 0) {
    if (seis_host) {
      if (g->seis_staging_elems < seis_elems) {
        dev_free(g, g->seis_staging, size_t(g->seis_staging_elems) * sizeof(float));
        g->seis_staging = nullptr;
        g->seis_staging_elems = 0;
        SW_TRY(dev_alloc(g, (void**)&g->seis_staging, size_t(seis_elems) * sizeof(float)));
        g->seis_staging_elems = seis_elems;
      }
      seis_dev = g->seis_staging;
    } else {
      seis_dev = seismogram;
    }
  }

  StencilArgs a = stencil_args(g);
  const PointSet src = point_set(g, true), rec = point_set(g, false);
  // small 2D grids: the whole run in one launch of one cluster (timed as one launch)
  ClusterShape cshape;
  const bool cluster = n_steps > 0 && use_cluster(g, &cshape);
  // two steps per launch (SW_STENCIL_TB2): n_steps / 2 launches, then an odd last step per step
  const bool tb2 = n_steps >= 2 && use_tb2(g);
  const int pairs = tb2 ? n_steps / 2 : 0;
  const int timed = !g->profiling ? 0
                    : (cluster ? 1
                               : (tb2 ? (pairs + g->profiling - 1) / g->profiling
                                      : (n_steps + g->profiling - 1) / g->profiling));  // launches timed
  if (tb2 && !g->u2[0]) {
    for (int i = 0; i < 2; ++i) {
      SW_TRY(dev_alloc(g, (void**)&g->u2[i], fbytes));
      SW_CUDA(cudaMemsetAsync(g->u2[i], 0, fbytes, g->stream));
    }
  }
  if (tb2 && !g->tb2_ready) {
    if (!g->sm_count) cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    SW_TRY(build_tb2_maps(g));
  }
  float* const lv[4] = {g->u[0], g->u[1], g->u2[0], g->u2[1]};  // level buffers of a two-step run
  if (timed && g->events.size() < size_t(2 * timed)) {
    size_t old = g->events.size();
    g->events.resize(size_t(2 * timed));
    for (size_t i = old; i < g->events.size(); ++i) SW_CUDA(cudaEventCreate(&g->events[i]));
  }
  int64_t launches = 0;
  const int src_threads = g->n_src * g->lz * g->ly * g->lx;
  const bool tma = use_tma(g);
  // pipelined path: each step's sources enter through the level the step
  // reads as p[n-1] (PreInject), added in the previous step's face launch,
  // instead of a launch of their own after the stencil
  double src_a, src_e;  // eta dt at the source window node deepest in the layers
  damping_coefficients(g->alpha, g->degree, g->dt, g->src_d2_max, &src_a, &src_e);
  const bool pre_inject = tma && src_threads > 0 && src_e < 0.5;
  // everything the time loop launches, in stream order
  auto enqueue = [&](cudaStream_t st, bool capturing, int64_t* nl) -> sw_status {
  // timing events become real event nodes of a captured graph
  const unsigned evflags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  int64_t launches = 0;
  if (tma && src_threads > 0) {  // tap table of the sources (model and dt are fixed for the run)
    if (!g->tap_off) {
      SW_TRY(dev_alloc(g, (void**)&g->tap_off, size_t(src_threads) * sizeof(int64_t)));
      SW_TRY(dev_alloc(g, (void**)&g->tap_coef, size_t(src_threads) * sizeof(float)));
      SW_TRY(dev_alloc(g, (void**)&g->tap_pre, size_t(src_threads) * sizeof(float)));
    }
    source_taps_kernel<<<(src_threads + 127) / 128, 128, 0, st>>>(a.kappa, g->damp, src, f, g->tap_off,
                                                                         g->tap_coef, g->tap_pre);
    SW_CUDA(cudaGetLastError());
    ++launches;
    if (pre_inject && n_steps > 0 && g->live(0)) {  // step 0's sources, into p[-1]
      inject_taps_kernel<<<(src_threads + 127) / 128, 128, 0, st>>>(
          g->at0(g->u[1]), g->tap_off, g->tap_pre, g->lz * g->ly * g->lx, g->n_src, g->wavelet, g->sig_stride, 0);
      SW_CUDA(cudaGetLastError());
      ++launches;
    }
  }
  int in_n = 0, in_m = 1;  // buffers (of lv) of p[step] and p[step - 1]
  int first_step = 0;
  if (tb2) {
    Tb2Args t;
    t.damp = g->damp;
    t.sz = g->lay.sz;
    t.nz = int(g->n[0]);
    t.nx = int(g->n[2]);
    const int fmap[4] = {0, 1, 4, 5};  // z low, z high, x low, x high
    for (int i = 0; i < 4; ++i) {
      t.nbl[i] = g->nbl[fmap[i]];
      t.bc[i] = g->bc[fmap[i]];
    }
    for (int j = 0; j <= kMaxR; ++j) {
      t.cz[j] = a.cz[j];
      t.cx[j] = a.cx[j];
    }
    t.src = src;
    t.sig = g->wavelet;
    t.sig_stride = g->sig_stride;
    t.tiles_x = int((g->n[2] + kTb2TX - 1) / kTb2TX);
    t.tiles = int(t.tiles_x * ((g->n[0] + kTb2TZ - 1) / kTb2TZ));
    for (int pr = 0; pr < pairs; ++pr) {
      const int step = 2 * pr;
      const int o1 = in_n < 2 ? 2 : 0, o2 = o1 + 1;  // the other two buffers: p[step + 1], p[step + 2]
      t.out1 = g->at0(lv[o1]);
      t.out2 = g->at0(lv[o2]);
      t.step = step;
      t.src.count = g->live(step) ? src.count : 0;  // step n's taps, in the kernel
      const bool time_it = g->profiling && pr % g->profiling == 0;
      const int ev = time_it ? 2 * (pr / g->profiling) : 0;
      if (time_it) SW_CUDA(cudaEventRecordWithFlags(g->events[ev], st, evflags));
      launch_tb2(g, g->tb2_n[in_n], g->tb2_m[in_m], t, st);
      if (time_it) SW_CUDA(cudaEventRecordWithFlags(g->events[ev + 1], st, evflags));
      // p[step + 1]: ghosts and its receivers
      launch_face_conditions(t.out1, f, g->R, rec, seis_dev, step, st);
      // p[step + 2]: step + 1's sources, then ghosts and its receivers
      if (src_threads > 0 && g->live(step + 1)) {
        launch_dependent(inject_sources_kernel, dim3((src_threads + 127) / 128), dim3(128), 0, st, t.out2,
                         (const float*)a.kappa, (const float2*)g->damp, src, (const float*)g->wavelet, g->sig_stride,
                         step + 1, f, g->ndim, g->R);
        ++launches;
      }
      launch_face_conditions(t.out2, f, g->R, rec, seis_dev, step + 1, st);
      launches += 3;
      in_n = o2;
      in_m = o1;
    }
    first_step = 2 * pairs;
  }
  for (int step = first_step; step < n_steps; ++step) {
    float* pn = tb2 ? lv[in_n] : g->u[step & 1];
    float* pnm1 = tb2 ? lv[in_m] : g->u[(step + 1) & 1];
    a.pn = g->at0(pn);
    a.pnm1 = g->at0(pnm1);
    a.pout = g->at0(pnm1);
    const bool time_it = !tb2 && g->profiling && step % g->profiling == 0;  // with tb2: its launches only
    const int ev = time_it ? 2 * (step / g->profiling) : 0;
    if (time_it) SW_CUDA(cudaEventRecordWithFlags(g->events[ev], st, evflags));
    if (tma)
      launch_stencil_tma(g, a, step & 1, st);
    else
      launch_stencil(g->R, g->ndim, g->has_density, a, st);
    if (time_it) SW_CUDA(cudaEventRecordWithFlags(g->events[ev + 1], st, evflags));
    ++launches;
    if (pre_inject) {
      // added to p[n-1] before the step (by the previous face launch, or before the loop)
    } else if (src_threads > 0 && tma && g->live(step)) {  // before the face conditions, which mirror its increments
      launch_dependent(inject_taps_kernel, dim3((src_threads + 127) / 128), dim3(128), 0, st, a.pout,
                       (const int64_t*)g->tap_off, (const float*)g->tap_coef, g->lz * g->ly * g->lx, g->n_src,
                       (const float*)g->wavelet, g->sig_stride, step);
      ++launches;
    } else if (src_threads > 0 && g->ndim == 2 && g->live(step)) {
      launch_dependent(inject_sources_kernel, dim3((src_threads + 127) / 128), dim3(128), 0, st, a.pout,
                       (const float*)a.kappa, (const float2*)g->damp, src, (const float*)g->wavelet, g->sig_stride,
                       step, f, g->ndim, g->R);
      ++launches;
    } else if (src_threads > 0 && g->live(step)) {
      inject_sources_kernel<<<(src_threads + 127) / 128, 128, 0, st>>>(
          a.pout, a.kappa, g->damp, src, g->wavelet, g->sig_stride, step, f, g->ndim, g->R);
      ++launches;
    }
    if (g->n_force > 0) {
      forcing_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(a.pout, a.kappa, g->damp, g->force_F, g->force_T,
                                                                   g->n_force, g->force_len, step, f, g->ndim, g->R,
                                                                   tma ? 0 : 1);
      ++launches;
    }
    if (tma) {
      // the pipelined kernel writes node values only: the face conditions
      // follow, with the receiver samples in the same launch
      PreInject pi{};
      if (pre_inject && step + 1 < n_steps && g->live(step + 1))
        pi = PreInject{g->at0(pn), g->tap_off, g->tap_pre, g->wavelet, g->lz * g->ly * g->lx, g->n_src, g->sig_stride,
                       step + 1};
      launch_face_conditions(a.pout, f, g->R, rec, seis_dev, step, st, pi);
      ++launches;
    } else if (g->n_rec > 0 && g->ndim == 2) {
      launch_dependent(sample_receivers_grouped_kernel, dim3((grouped_receiver_warps(rec) + 3) / 4), dim3(128), 0,
                       st, (const float*)a.pout, rec, f, seis_dev, step);
      ++launches;
    } else if (g->n_rec > 0) {
      sample_receivers_kernel<<<(g->n_rec + 3) / 4, 128, 0, st>>>(a.pout, rec, f, seis_dev, step);
      ++launches;
    }
    if (g->snapshots && (step + 1) % g->saving_stride == 0) {  // frame k holds p after (k+1) * stride steps
      const int64_t frame = (step + 1) / g->saving_stride - 1;
      if (frame < g->snapshot_frames) {
        extract_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(a.pout, g->snapshots + frame * g->nodes(), f);
        ++launches;
      }
    }
  }
  SW_CUDA(cudaGetLastError());
  *nl = launches;
  return SW_OK;
  };
  const sw_grid::ForwardKey key{n_steps, seis_dev, g->profiling, tma, g->config_gen};
  if (cluster) {
    ClusterRun run;
    run.u[0] = g->at0(g->u[0]);
    run.u[1] = g->at0(g->u[1]);
    run.kappa = a.kappa;
    run.damp = g->damp;
    run.f = f;
    run.B = cshape.B;
    run.W = cshape.W;
    for (int j = 0; j <= kMaxR; ++j) {
      run.cz[j] = a.cz[j];
      run.cx[j] = a.cx[j];
    }
    run.src = src;
    run.rec = rec;
    run.sig = g->wavelet;
    run.sig_stride = g->sig_stride;
    run.seis = g->n_rec > 0 ? seis_dev : nullptr;
    run.n_steps = n_steps;
    {  // receivers in registers: one pass of the cluster's warps, at most kClusterRecRows rows per window
      const int per_warp = g->lx <= 8 ? 4 : (g->lx <= 16 ? 2 : 1);
      const int rows = g->rec_span ? g->rec_rows_max : g->lz;
      run.rec_fast = g->n_rec <= cshape.C * (kClusterThreads / 32) * per_warp && rows <= kClusterRecRows ? 1 : 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(cshape.C));
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = cshape.smem;
    cfg.stream = g->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(cshape.C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (timed) SW_CUDA(cudaEventRecord(g->events[0], g->stream));
    SW_CUDA(cudaLaunchKernelEx(&cfg, cluster_kernel(g->R), run));
    if (timed) SW_CUDA(cudaEventRecord(g->events[1], g->stream));
    launches = 1;
  } else if (n_steps > 0 && g->graph && g->graph_key == key) {
    SW_CUDA(cudaGraphLaunch(g->graph, g->stream));
    launches = g->graph_launches;
  } else if (n_steps > 0 && g->last_key_valid && g->last_key == key) {
    // second call with this configuration: capture the time loop once
    if (g->graph) {
      cudaGraphExecDestroy(g->graph);
      g->graph = nullptr;
    }
    // captured on a private stream (the grid's stream may be the legacy
    // default stream, which cannot be captured), launched on the grid's
    if (!g->cap_stream) SW_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    SW_CUDA(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    const sw_status st = enqueue(g->cap_stream, true, &launches);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
    if (st != SW_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return st != SW_OK ? st : fail(SW_ECUDA, "capturing the time loop failed: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&g->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      g->graph = nullptr;
      return fail(SW_ECUDA, "instantiating the time loop failed: %s", cudaGetErrorString(ei));
    }
    g->graph_key = key;
    g->graph_launches = launches;
    SW_CUDA(cudaGraphLaunch(g->graph, g->stream));
  } else if (n_steps > 0) {
    SW_TRY(enqueue(g->stream, false, &launches));
  }
  g->last_key = key;
  g->last_key_valid = true;
  if (final_field) {
    float* last = g->at0(tb2 ? lv[tb2_last_level(n_steps)] : g->u[n_steps & 1]);
    const bool fh = !is_device_pointer(final_field);
    float* dst = final_field;
    if (fh) {
      if (!g->staging) SW_TRY(dev_alloc(g, (void**)&g->staging, size_t(g->nodes()) * sizeof(float)));
      dst = g->staging;
    }
    extract_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, g->stream>>>(last, dst, f);
    SW_CUDA(cudaGetLastError());
    ++launches;
    if (fh)
      SW_CUDA(cudaMemcpyAsync(final_field, dst, size_t(g->nodes()) * sizeof(float), cudaMemcpyDefault,
                              g->stream));
  }
  if (seis_host && seis_elems > 0)
    SW_CUDA(cudaMemcpyAsync(seismogram, seis_dev, size_t(seis_elems) * sizeof(float), cudaMemcpyDefault,
                            g->stream));
  SW_TRY(check_device_flag(g));
  g->kernel_launches = launches;
  g->stencil_launches = cluster && timed ? n_steps : timed;  // the cluster run's time counts per time step
  g->stencil_ms = 0.0;
  for (int i = 0; i < timed; ++i) {
    float ms = 0.f;
    SW_CUDA(cudaEventElapsedTime(&ms, g->events[2 * i], g->events[2 * i + 1]));
    g->stencil_ms += ms;
  }
  return SW_OK;
}

// The misfit gradient of sw_gradient (n_shots = 1, shot_src_pos = NULL: the
// acquisition's own sources) and of sw_gradient_shots (shot s runs with the
// sources at shot_src_pos + s * n_src * ndim and the observed data at
// observed + s * n_steps * n_rec).  Misfit and gradient accumulators,
// checkpoints and segment buffers are shared by all shots; the acquisition's
// own source windows are put back afterwards.
static sw_status gradient_impl(sw_grid* g, int n_shots, const double* shot_src_pos, int n_steps, const float* observed,
                        double* misfit, float* grad_vel, float* grad_rho, int checkpoint_every,
                        int checkpoint_format) {
  if (!g || !observed || !misfit || !grad_vel) return fail(SW_EINVAL, "NULL argument");
  if (!g->has_model) return fail(SW_ESTATE, "sw_gradient before sw_set_model");
  if (!g->has_acq) return fail(SW_ESTATE, "sw_gradient before sw_set_acquisition");
  if (grad_rho && !g->has_density) return fail(SW_EINVAL, "a density gradient needs a density model");
  if (g->n_force > 0 || g->init_p0 || g->init_pm1)
    return fail(SW_ESTATE, "the gradient assumes zero initial levels and no distributed forcing");
  if (g->n_rec <= 0) return fail(SW_EINVAL, "the gradient needs receivers");
  if (n_steps < 1) return fail(SW_EINVAL, "n_steps < 1");
  if (g->n_src > 0 && n_steps > g->nt) return fail(SW_EINVAL, "n_steps (%d) exceeds the wavelet length (%d)", n_steps, g->nt);
  if (n_shots < 1) return fail(SW_EINVAL, "n_shots < 1");
  if (shot_src_pos && g->n_src < 1) return fail(SW_EINVAL, "shots need an acquisition with sources");
  // every shot's source windows, built (and checked) before any device work
  std::vector<std::vector<int>> shot_first;
  std::vector<std::vector<float>> shot_w;
  if (shot_src_pos) {
    shot_first.resize(size_t(n_shots));
    shot_w.resize(size_t(n_shots));
    for (int sh = 0; sh < n_shots; ++sh)
      SW_TRY(build_windows(g, g->n_src, shot_src_pos + size_t(sh) * g->n_src * g->ndim, true,
                           shot_first[size_t(sh)], shot_w[size_t(sh)]));
  }
  if (checkpoint_every < 0) return fail(SW_EINVAL, "checkpoint_every < 0");
  if (checkpoint_format != SW_CKPT_FP32 && checkpoint_format != SW_CKPT_BF16 && checkpoint_format != SW_CKPT_FP16 &&
      checkpoint_format != SW_CKPT_I16)
    return fail(SW_EINVAL, "unknown checkpoint format %d", checkpoint_format);
  if (g->n[0] > 65535 || g->n[1] > 65535) return fail(SW_EINVAL, "axis longer than 65535 nodes");
  for (int ax = 0; ax < 3; ++ax)  // the face passes need every node within R of one face only
    if ((g->ndim == 3 || ax != 1) && g->n[ax] <= 2 * int64_t(g->R) + 1)
      return fail(SW_EINVAL, "the gradient needs more than 2R+1 nodes along every axis");
  const int N = n_steps;
  // binomial (revolve) schedule: at most `budget` stored states and two
  // working levels; else uniform segments of K steps
  const int budget = g->ckpt_budget;
  const bool revolve = budget > 0;
  if (revolve && checkpoint_format != SW_CKPT_FP32)
    return fail(SW_EINVAL, "the binomial schedule keeps FP32 states");
  const FaceInfo f = g->faces();
  const size_t fbytes = size_t(g->lay.total) * sizeof(float);
  const bool vd = g->has_density;
  // with density: dJ/dG_a accumulators, and G_a = D_a ln rho unless the
  // pipelined kernel's copies exist
  const bool own_g = vd && !g->glr[0];
  const int nvd = vd ? 3 + (own_g ? 3 : 0) : 0;
  int K = checkpoint_every;
  if (K == 0) {  // every forward level kept when they fit in 80% of the free device memory, else K ~ sqrt(2N)
    size_t free_b = 0, total_b = 0;
    SW_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double need = double(N + 1 + 3 + nvd) * double(fbytes);
    K = need <= 0.8 * double(free_b) ? N : std::max(1, int(std::lround(std::sqrt(2.0 * N))));
  }
  K = revolve ? 1 : std::min(K, N);
  const int nseg = revolve ? budget : (N + K - 1) / K;
  // one segment of every step: the forward pass itself writes p[0 .. N-1]
  // into the segment buffers, so the adjoint sweep recomputes nothing and
  // nothing is rounded to a checkpoint format
  const bool keep_all = !revolve && nseg == 1;
  const bool tma = use_tma(g);
  cudaStream_t st = g->stream;

  // device memory of this call: checkpoint pairs (padded FP32 fields, or
  // 16-bit node arrays with their scales), segment states (one block), psi,
  // dJ/dkappa
  const bool packed = checkpoint_format != SW_CKPT_FP32 && !keep_all;
  const int nck = packed || keep_all ? 0 : 2 * nseg;
  const int nfields = nck + (K + 1) + 2 + 1 + nvd;
  const size_t pbytes = size_t(g->nodes()) * 2;  // one packed checkpoint
  void* packs = nullptr;
  unsigned* scales = nullptr;
  const bool i16 = checkpoint_format == SW_CKPT_I16;
  const int64_t nrows = g->n[0] * g->n[1];
  float* row_scales = nullptr;  // SW_CKPT_I16: one scale per (z, y) row of every stored level
  std::vector<float*> F(size_t(nfields), nullptr);
  float *syn = nullptr, *obs = nullptr, *res = nullptr;
  double* macc = nullptr;
  const size_t sbytes = size_t(N) * g->n_rec * sizeof(float);
  const size_t seg_stride = (fbytes + 255) / 256 * 256;  // segment states: one allocation of K + 1 fields
  float* seg_block = nullptr;
  auto release = [&]() {
    cudaStreamSynchronize(st);
    for (size_t i = 0; i < F.size(); ++i) {
      if (i < size_t(nck) || i > size_t(nck + K)) dev_free(g, F[i], fbytes);
      F[i] = nullptr;
    }
    dev_free(g, seg_block, seg_stride * size_t(K + 1));
    dev_free(g, syn, sbytes);
    dev_free(g, obs, sbytes);
    dev_free(g, res, sbytes);
    dev_free(g, macc, sizeof(double));
    dev_free(g, packs, packed ? pbytes * 2 * nseg : 0);
    dev_free(g, scales, packed ? sizeof(unsigned) * 2 * nseg : 0);
    dev_free(g, row_scales, i16 ? sizeof(float) * size_t(nrows) * 2 * nseg : 0);
  };
  struct Guard {
    std::function<void()> fn;
    ~Guard() { fn(); }
  } guard{release};
  SW_TRY(dev_alloc(g, (void**)&seg_block, seg_stride * size_t(K + 1)));
  SW_CUDA(cudaMemsetAsync(seg_block, 0, seg_stride * size_t(K + 1), st));
  for (size_t i = 0; i < F.size(); ++i) {
    if (i >= size_t(nck) && i <= size_t(nck + K)) {
      F[i] = reinterpret_cast<float*>(reinterpret_cast<char*>(seg_block) + seg_stride * (i - size_t(nck)));
      continue;
    }
    SW_TRY(dev_alloc(g, (void**)&F[i], fbytes));
    SW_CUDA(cudaMemsetAsync(F[i], 0, fbytes, st));
  }
  SW_TRY(dev_alloc(g, (void**)&syn, sbytes));
  SW_TRY(dev_alloc(g, (void**)&obs, sbytes));
  SW_TRY(dev_alloc(g, (void**)&res, sbytes));
  SW_TRY(dev_alloc(g, (void**)&macc, sizeof(double)));
  if (packed) {
    SW_TRY(dev_alloc(g, &packs, pbytes * 2 * nseg));
    SW_TRY(dev_alloc(g, (void**)&scales, sizeof(unsigned) * 2 * nseg));
    SW_CUDA(cudaMemsetAsync(scales, 0, sizeof(unsigned) * 2 * nseg, st));
    if (i16) SW_TRY(dev_alloc(g, (void**)&row_scales, sizeof(float) * size_t(nrows) * 2 * nseg));
  }
  SW_CUDA(cudaMemsetAsync(macc, 0, sizeof(double), st));
  auto ck = [&](int sgm, int i) { return F[size_t(2 * sgm + i)]; };  // FP32: i = 0: p[k0-1], 1: p[k0]
  auto B = [&](int j) { return F[size_t(nck + j)]; };                 // p[k0 + j - 1]
  auto PSI = [&](int i) { return F[size_t(nck + K + 1 + i)]; };
  float* GK = F[size_t(nck + K + 3)];
  float* AG[3] = {nullptr, nullptr, nullptr};  // dJ/dG_a
  float* GG[3] = {nullptr, nullptr, nullptr};  // G_a
  VdWeights vw;
  memset(&vw, 0, sizeof(vw));
  if (vd) {
    for (int i = 0; i < 3; ++i) {
      AG[i] = g->at0(F[size_t(nck + K + 4 + i)]);
      GG[i] = own_g ? g->at0(F[size_t(nck + K + 7 + i)]) : g->at0(g->glr[i]);
    }
    double wj[kMaxR + 1];
    fd_first_weights(g->order, wj);
    GradWeights gw;
    for (int j = 0; j <= kMaxR; ++j) {
      const bool in = j >= 1 && j <= g->R;
      gw.z[j] = in ? wj[j] / (2.0 * g->h[0]) : 0.0;
      gw.y[j] = in ? wj[j] / (2.0 * g->h[1]) : 0.0;
      gw.x[j] = in ? wj[j] / (2.0 * g->h[2]) : 0.0;
      vw.w[0][j] = float(gw.z[j]);
      vw.w[1][j] = float(gw.y[j]);
      vw.w[2][j] = float(gw.x[j]);
    }
    if (own_g) {
      lnrho_gradient_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(g->at0(g->lnrho), GG[0], GG[1], GG[2], f,
                                                                          gw, g->R);
      SW_CUDA(cudaGetLastError());
    }
  }
  std::vector<CUtensorMap> halo(static_cast<size_t>(nfields)), inner(static_cast<size_t>(nfields)),
      warm(static_cast<size_t>(nfields));
  if (tma) {
    int tx, ty;
    tma_tile(g->R, &tx, &ty);
    const uint32_t xh = uint32_t((g->R + 3) / 4 * 4);
    for (int i = nck; i < nck + K + 4; ++i) {  // segment states, psi and gk
      SW_TRY(make_map(g, F[size_t(i)], uint32_t(tx) + 2 * xh, uint32_t(ty + 2 * g->R), &halo[size_t(i)]));
      SW_TRY(make_map(g, F[size_t(i)], uint32_t(tx), uint32_t(ty), &inner[size_t(i)]));
      SW_TRY(make_map(g, F[size_t(i)], uint32_t(tx), uint32_t(ty), &warm[size_t(i)], kTmaWarmPlanes));
    }
  }
  auto idx = [&](float* p) { return size_t(std::find(F.begin(), F.end(), p) - F.begin()); };

  StencilArgs a = stencil_args(g);
  const PointSet src = point_set(g, true), rec = point_set(g, false);
  PointSet none = rec;
  none.count = 0;
  const int src_threads = g->n_src * g->lz * g->ly * g->lx;
  LapCoef lc;
  for (int j = 0; j <= kMaxR; ++j) {
    lc.c[0][j] = a.cz[j];
    lc.c[1][j] = a.cy[j];
    lc.c[2][j] = a.cx[j];
  }
  int64_t nk = 0;  // kernels launched by this call
  int pending_src = -1;  // the adjoint step whose source imaging is still to come
  // one step p[n] (pn), p[n-1] (pm) -> p[n+1] (po), with sources at step n
  auto step = [&](float* pn, float* pm, float* po, const StepMaps* m, int n, const float* sig, int sig_stride,
                  const PointSet& pts, const PointSet& recs, float* seis) -> sw_status {
    const int taps = g->live(n) ? pts.count * pts.lz * pts.ly * pts.lx : 0;  // no launch for a silent step
    nk += 2 + (taps > 0);
    a.pn = g->at0(pn);
    a.pnm1 = g->at0(pm);
    a.pout = g->at0(po);
    if (m)
      launch_stencil_tma_maps(g, a, *m, st, vd);
    else
      launch_stencil(g->R, g->ndim, vd, a, st);
    if (taps > 0)
      launch_dependent(inject_sources_kernel, dim3((taps + 127) / 128), dim3(128), 0, st, a.pout, a.kappa, g->damp, pts, sig, sig_stride, n,
                                                                f, g->ndim, g->R);
    launch_face_conditions(a.pout, f, g->R, recs, seis, n, st);
    SW_CUDA(cudaGetLastError());
    return SW_OK;
  };

  // the acquisition's own source windows, put back after the shots
  std::vector<int> own_first;
  std::vector<float> own_w;
  const size_t nfirst = size_t(g->n_src) * 3, nw = size_t(g->n_src) * 3 * g->L;
  if (shot_src_pos) {
    own_first.resize(nfirst);
    own_w.resize(nw);
    SW_CUDA(cudaMemcpyAsync(own_first.data(), g->src_first, nfirst * sizeof(int), cudaMemcpyDeviceToHost, st));
    SW_CUDA(cudaMemcpyAsync(own_w.data(), g->src_w, nw * sizeof(float), cudaMemcpyDeviceToHost, st));
    SW_CUDA(cudaStreamSynchronize(st));
  }
  struct RestoreSources {
    sw_grid* g;
    const std::vector<int>* f;
    const std::vector<float>* w;
    bool on;
    ~RestoreSources() {
      if (!on) return;
      cudaMemcpyAsync(g->src_first, f->data(), f->size() * sizeof(int), cudaMemcpyHostToDevice, g->stream);
      cudaMemcpyAsync(g->src_w, w->data(), w->size() * sizeof(float), cudaMemcpyHostToDevice, g->stream);
      cudaStreamSynchronize(g->stream);
    }
  } restore{g, &own_first, &own_w, shot_src_pos != nullptr};

  for (int shot = 0; shot < n_shots; ++shot) {
  if (shot_src_pos) {  // this shot's sources (the copies are ordered before the shot's kernels)
    SW_CUDA(cudaMemcpyAsync(g->src_first, shot_first[size_t(shot)].data(), nfirst * sizeof(int),
                            cudaMemcpyHostToDevice, st));
    SW_CUDA(cudaMemcpyAsync(g->src_w, shot_w[size_t(shot)].data(), nw * sizeof(float), cudaMemcpyHostToDevice, st));
  }
  SW_CUDA(cudaMemcpyAsync(obs, observed + size_t(shot) * N * g->n_rec, sbytes, cudaMemcpyDefault, st));
  if (shot > 0) {  // the adjoint levels and the 16-bit scales start from zero for every shot
    SW_CUDA(cudaMemsetAsync(PSI(0), 0, fbytes, st));
    SW_CUDA(cudaMemsetAsync(PSI(1), 0, fbytes, st));
    if (packed) SW_CUDA(cudaMemsetAsync(scales, 0, sizeof(unsigned) * 2 * nseg, st));
  }
  pending_src = -1;
  if (keep_all) {
    // forward into the segment buffers: p[n] in B(n + 1), p[N] (for the
    // receivers only) in B(0), which held p[-1]
    SW_CUDA(cudaMemsetAsync(B(0), 0, fbytes, st));
    SW_CUDA(cudaMemsetAsync(B(1), 0, fbytes, st));
    for (int n = 0; n < N; ++n) {
      float* po = n + 2 <= K ? B(n + 2) : B(0);
      const StepMaps m{&halo[idx(B(n + 1))], &inner[idx(B(n + 1))], &inner[idx(B(n))], &warm[idx(B(n + 1))]};
      SW_TRY(step(B(n + 1), B(n), po, tma ? &m : nullptr, n, g->wavelet, g->sig_stride, src, rec, syn));
    }
    // the grid's levels hold p[N - 1] and p[N], as after sw_forward
    SW_CUDA(cudaMemcpyAsync(g->u[(N - 1) & 1], B(N), fbytes, cudaMemcpyDeviceToDevice, st));
    SW_CUDA(cudaMemcpyAsync(g->u[N & 1], B(0), fbytes, cudaMemcpyDeviceToDevice, st));
  }
  // forward, keeping (p[k0-1], p[k0]) at every segment start
  if (!keep_all) {
    SW_CUDA(cudaMemsetAsync(g->u[0], 0, fbytes, st));
    SW_CUDA(cudaMemsetAsync(g->u[1], 0, fbytes, st));
  }
  for (int n = 0; n < (keep_all ? 0 : N); ++n) {
    float* pn = g->u[n & 1];
    float* pm = g->u[(n + 1) & 1];
    if (!revolve && n % K == 0) {
      if (packed) {
        // slot 1: p[n]; slot 0: p[n] - p[n-1], small next to p, kept with its
        // own scale so that the time difference a recomputed segment starts
        // from is as accurate as the level itself
        for (int i = 0; i < 2; ++i) {
          const int slot = 2 * (n / K) + i;
          const float* a_f = g->at0(pn);
          const float* b_f = i == 0 ? g->at0(pm) : nullptr;
          unsigned* sc = scales + slot;
          char* dst = static_cast<char*>(packs) + pbytes * slot;
          if (i16) {
            launch_dependent(pack_rows_i16_kernel, dim3(unsigned(std::min<int64_t>((nrows + 7) / 8, 4736))), dim3(256), 0, st, 
                a_f, b_f, f, row_scales + size_t(nrows) * slot, reinterpret_cast<int16_t*>(dst));
            continue;
          }
          absmax_kernel<<<row_grid(f), 256, 0, st>>>(a_f, b_f, f, sc);
          if (checkpoint_format == SW_CKPT_BF16)
            pack_snapshot_kernel<__nv_bfloat16><<<row_grid(f), 256, 0, st>>>(
                a_f, b_f, f, sc, reinterpret_cast<__nv_bfloat16*>(dst));
          else
            pack_snapshot_kernel<__half><<<row_grid(f), 256, 0, st>>>(a_f, b_f, f, sc,
                                                                     reinterpret_cast<__half*>(dst));
        }
        SW_CUDA(cudaGetLastError());
      } else {
        SW_CUDA(cudaMemcpyAsync(ck(n / K, 0), pm, fbytes, cudaMemcpyDeviceToDevice, st));
        SW_CUDA(cudaMemcpyAsync(ck(n / K, 1), pn, fbytes, cudaMemcpyDeviceToDevice, st));
      }
    }
    const StepMaps m{&g->map_halo[n & 1], &g->map_inner[n & 1], &g->map_inner[(n + 1) & 1], &g->map_warm[n & 1]};
    SW_TRY(step(pn, pm, pm, tma ? &m : nullptr, n, g->wavelet, g->sig_stride, src, rec, syn));
  }
  residual_kernel<<<256, 256, 0, st>>>(syn, obs, res, macc, N, g->n_rec);
  SW_CUDA(cudaGetLastError());

  // backward: per segment, recompute p[k0 .. k1-1], then the adjoint steps k1 .. k0+1
  // one adjoint step: psi[k] from psi[k+1], psi[k+2], then its imaging
  // terms with the forward state p[k-1] (pk1, ghosts set)
  auto adjoint_step = [&](int k, float* pk1) -> sw_status {
    nk += 4 + (vd ? 1 : 0);
    float* p1 = PSI((k + 1) & 1);  // psi[k+1]
    float* p2 = PSI(k & 1);        // psi[k+2], overwritten by psi[k]
    const StepMaps m{&halo[idx(p1)], &inner[idx(p1)], &inner[idx(p2)], &warm[idx(p1)]};
    a.pn = g->at0(p1);
    a.pnm1 = g->at0(p2);
    a.pout = g->at0(p2);
    // L^T psi: the constant-density stencil, then its Neumann-face correction
    if (tma)
      launch_stencil_tma_maps(g, a, m, st, false);
    else
      launch_stencil(g->R, g->ndim, false, a, st);
    if (vd)  // - sum_a D_a^T (G_a psi)
      launch_dependent(vd_adjoint_kernel, dim3(grid_blocks(g->nodes(), 256)), dim3(256), 0, st, g->at0(p1), GG[0], GG[1], GG[2], a.kappa,
                                                                      g->damp, g->at0(p2), f, vw, g->R, g->ndim);
    // its Neumann-face correction and the residuals into psi through the
    // receiver windows (rows with non-zero weight only), in one launch
    // blocks of the Neumann correction per axis: both faces' lines, none for an axis without a Neumann face
    auto neumann_blocks = [&](int ax, int64_t face) {
      return g->bc[2 * ax] == SW_BC_NEUMANN || g->bc[2 * ax + 1] == SW_BC_NEUMANN ? int((2 * face + 255) / 256) : 0;
    };
    const int3 nb = make_int3(neumann_blocks(0, g->n[1] * g->n[2]), neumann_blocks(1, g->n[0] * g->n[2]),
                              neumann_blocks(2, g->n[0] * g->n[1]));
    const int rthreads = rec.count * g->rec_rows_max * rec.lx;
    // step k+1's source imaging: psi[k+1] is p1, which this step only reads
    SourceImaging si{};
    if (src_threads > 0 && pending_src == k + 1 && g->live(k))
      si = SourceImaging{g->at0(p1), g->at0(GK), src, g->wavelet, g->sig_stride, k, (src_threads + 255) / 256};
    launch_dependent(adjoint_additions_kernel, dim3(unsigned(si.blocks + nb.x + nb.y + nb.z + (rthreads + 255) / 256)), dim3(256), 0, st, 
        g->at0(p1), g->at0(p2), a.kappa, g->damp, f, lc, g->R, nb, rec, g->rec_rows_max, res, N, k - 1, g->ndim,
        si);
    launch_face_conditions(g->at0(p2), f, g->R, none, nullptr, 0, st);
    const dim3 ig(unsigned((g->n[2] + 127) / 128), unsigned(g->n[1]), unsigned(g->n[0]));
    if (vd) {
      launch_image_vd(g->R, g->ndim, ig, g->at0(pk1), g->at0(p2), GG, g->at0(GK), AG, f, lc, vw, st);
    } else if (tma) {  // gk += psi[k] L p[k-1] on the pipelined kernel
      StepMaps im{&halo[idx(pk1)], &inner[idx(pk1)], &inner[idx(p2)], &warm[idx(pk1)]};
      im.kap = &inner[idx(GK)];
      StencilArgs ai = a;
      ai.pout = g->at0(GK);
      launch_image_tma(g, ai, im, st);
    } else {
      launch_image(g->R, g->ndim, ig, g->at0(pk1), g->at0(p2), g->at0(GK), f, lc, st);
    }
    pending_src = k;  // its source imaging goes with the next step's additions, or follows the sweep
    SW_CUDA(cudaGetLastError());
    return SW_OK;
  };

  if (revolve) {
    // Binomial checkpointing (the recursive form of Griewank's revolve):
    // reverse steps (l, r] from the stored state (p[l-1], p[l]) in slot sl
    // (-1: the zero state at level 0) with `fr` free slots.  With n = r - l
    // steps and t the least repetition count with C(fr + t, fr) >= n, the
    // state at m = r - min(C(fr - 1 + t, fr - 1), n - 1) is stored; (m, r]
    // is reversed with one slot fewer, then (l, m] with the same slots.
    // Without a free slot every step recomputes from l.  The two working
    // levels are B(0) and B(1); each forward step overwrites the older.
    auto binom = [](int s_, int t_) {
      double b = 1.0;
      for (int i = 1; i <= s_; ++i) b = b * double(t_ + i) / double(i);
      return b;
    };
    int cur = 1;  // B(cur) holds the newest working level
    auto load = [&](int sl) -> sw_status {
      if (sl < 0) {
        SW_CUDA(cudaMemsetAsync(B(0), 0, fbytes, st));
        SW_CUDA(cudaMemsetAsync(B(1), 0, fbytes, st));
      } else {
        SW_CUDA(cudaMemcpyAsync(B(0), ck(sl, 0), fbytes, cudaMemcpyDeviceToDevice, st));
        SW_CUDA(cudaMemcpyAsync(B(1), ck(sl, 1), fbytes, cudaMemcpyDeviceToDevice, st));
      }
      cur = 1;
      return SW_OK;
    };
    auto advance = [&](int from, int to) -> sw_status {  // working levels from `from` to `to`
      for (int n = from; n < to; ++n) {
        float* pn = B(cur);
        float* pm = B(cur ^ 1);
        const StepMaps m{&halo[idx(pn)], &inner[idx(pn)], &inner[idx(pm)], &warm[idx(pn)]};
        SW_TRY(step(pn, pm, pm, tma ? &m : nullptr, n, g->wavelet, g->sig_stride, src, none, nullptr));
        cur ^= 1;
      }
      return SW_OK;
    };
    std::function<sw_status(int, int, int, int)> reverse = [&](int l, int r, int sl, int fr) -> sw_status {
      const int n = r - l;
      if (n <= 0) return SW_OK;
      if (n == 1) {
        SW_TRY(load(sl));
        return adjoint_step(r, B(cur));
      }
      if (fr == 0) {
        for (int k = r; k > l; --k) {
          SW_TRY(load(sl));
          SW_TRY(advance(l, k - 1));
          SW_TRY(adjoint_step(k, B(cur)));
        }
        return SW_OK;
      }
      int t = 0;
      while (binom(fr, t) < double(n)) ++t;
      const int right = int(std::min(binom(fr - 1, t), double(n - 1)));
      const int m = r - std::max(right, 1);
      const int slot = budget - fr;  // slots are taken in stack order
      SW_TRY(load(sl));
      SW_TRY(advance(l, m));
      SW_CUDA(cudaMemcpyAsync(ck(slot, 0), B(cur ^ 1), fbytes, cudaMemcpyDeviceToDevice, st));
      SW_CUDA(cudaMemcpyAsync(ck(slot, 1), B(cur), fbytes, cudaMemcpyDeviceToDevice, st));
      SW_TRY(reverse(m, r, slot, fr - 1));
      return reverse(l, m, sl, fr);
    };
    SW_TRY(reverse(0, N, -1, budget));
  } else {  // uniform: per segment, recompute p[k0 .. k1-1], then the adjoint steps k1 .. k0+1
    for (int sgm = nseg - 1; sgm >= 0; --sgm) {
      const int k0 = sgm * K, k1 = std::min(N, k0 + K);
      if (keep_all) {  // B(1 .. N) hold p[0 .. N-1] from the forward pass
      } else if (packed) {
        for (int i = 1; i >= 0; --i) {  // p[k0] first, then p[k0-1] = p[k0] - (p[k0] - p[k0-1])
          const int slot = 2 * sgm + i;
          const char* src_p = static_cast<const char*>(packs) + pbytes * slot;
          const float* base = i == 0 ? g->at0(B(1)) : nullptr;
          if (i16)
            launch_dependent(unpack_rows_i16_kernel, dim3(unsigned(std::min<int64_t>((nrows + 7) / 8, 4736))), dim3(256), 0, st, 
                reinterpret_cast<const int16_t*>(src_p),
                                                                row_scales + size_t(nrows) * slot, f, base,
                                                                g->at0(B(i)));
          else if (checkpoint_format == SW_CKPT_BF16)
            unpack_snapshot_kernel<__nv_bfloat16><<<row_grid(f), 256, 0, st>>>(
                reinterpret_cast<const __nv_bfloat16*>(src_p), scales + slot, f, base, g->at0(B(i)));
          else
            unpack_snapshot_kernel<__half><<<row_grid(f), 256, 0, st>>>(
                reinterpret_cast<const __half*>(src_p), scales + slot, f, base, g->at0(B(i)));
        }
        // ghosts of the restored p[k0]; p[k0-1] is read at its nodes only (as
        // the first recomputed step's p[n-1]), and its Dirichlet face nodes
        // come back as exact zeros (0 - 0 from zero codes), so it needs none
        launch_face_conditions(g->at0(B(1)), f, g->R, none, nullptr, 0, st);
        SW_CUDA(cudaGetLastError());
      } else {
        SW_CUDA(cudaMemcpyAsync(B(0), ck(sgm, 0), fbytes, cudaMemcpyDeviceToDevice, st));
        SW_CUDA(cudaMemcpyAsync(B(1), ck(sgm, 1), fbytes, cudaMemcpyDeviceToDevice, st));
      }
      for (int n = k0; n <= (keep_all ? k0 - 1 : k1 - 2); ++n) {
        const int j = n - k0 + 1;
        const StepMaps m{&halo[idx(B(j))], &inner[idx(B(j))], &inner[idx(B(j - 1))], &warm[idx(B(j))]};
        SW_TRY(step(B(j), B(j - 1), B(j + 1), tma ? &m : nullptr, n, g->wavelet, g->sig_stride, src, none, nullptr));
      }
      for (int k = k1; k >= k0 + 1; --k) SW_TRY(adjoint_step(k, B(k - k0)));
    }
  }

  if (src_threads > 0 && pending_src > 0 && g->live(pending_src - 1)) {  // the last adjoint step's source imaging
    image_sources_kernel<<<(src_threads + 127) / 128, 128, 0, st>>>(g->at0(PSI(pending_src & 1)), g->at0(GK), src,
                                                                    g->wavelet, g->sig_stride, pending_src - 1, f);
    SW_CUDA(cudaGetLastError());
    ++nk;
  }
  }  // shots
  // dJ/dc, densely per node
  float* out = grad_vel;
  const bool host_out = !is_device_pointer(grad_vel);
  if (host_out) {
    if (!g->staging) SW_TRY(dev_alloc(g, (void**)&g->staging, size_t(g->nodes()) * sizeof(float)));
    out = g->staging;
  }
  gradient_velocity_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(g->at0(GK), a.kappa, out, f, float(g->dt));
  SW_CUDA(cudaGetLastError());
  if (host_out)
    SW_CUDA(cudaMemcpyAsync(grad_vel, out, size_t(g->nodes()) * sizeof(float), cudaMemcpyDefault, st));
  if (grad_rho) {  // dJ/drho
    float* ro = grad_rho;
    const bool host_r = !is_device_pointer(grad_rho);
    if (host_r) {
      if (!g->staging2) SW_TRY(dev_alloc(g, (void**)&g->staging2, size_t(g->nodes()) * sizeof(float)));
      ro = g->staging2;
    }
    gradient_density_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(AG[0], AG[1], AG[2], g->at0(g->lnrho), ro,
                                                                           f, vw, g->R, g->ndim);
    SW_CUDA(cudaGetLastError());
    if (host_r)
      SW_CUDA(cudaMemcpyAsync(grad_rho, ro, size_t(g->nodes()) * sizeof(float), cudaMemcpyDefault, st));
  }
  SW_CUDA(cudaMemcpyAsync(misfit, macc, sizeof(double), cudaMemcpyDeviceToHost, st));
  SW_TRY(check_device_flag(g));
  // + residual and velocity gradient, density gradient, ln rho gradients,
  // and per 16-bit checkpoint segment absmax + pack and unpack + the face pass of the restored level
  g->kernel_launches = nk + 1 + n_shots + (grad_rho ? 1 : 0) + (own_g ? 1 : 0) +
                       (packed ? (i16 ? 5 : 7) * int64_t(nseg) * n_shots : 0);
  g->stencil_launches = 0;
  g->stencil_ms = 0.0;
  return SW_OK;
}

sw_status sw_gradient(sw_grid* g, int n_steps, const float* observed, double* misfit, float* grad_vel,
                      float* grad_rho, int checkpoint_every, int checkpoint_format) {
  g_last_error.clear();
  return gradient_impl(g, 1, nullptr, n_steps, observed, misfit, grad_vel, grad_rho, checkpoint_every,
                       checkpoint_format);
}

sw_status sw_gradient_shots(sw_grid* g, int n_shots, const double* shot_src_pos, int n_steps, const float* observed,
                            double* misfit, float* grad_vel, float* grad_rho, int checkpoint_every,
                            int checkpoint_format) {
  g_last_error.clear();
  if (!shot_src_pos) return fail(SW_EINVAL, "NULL shot positions");
  if (g) ++g->config_gen;  // the source windows change during the call (and are put back)
  return gradient_impl(g, n_shots, shot_src_pos, n_steps, observed, misfit, grad_vel, grad_rho, checkpoint_every,
                       checkpoint_format);
}

sw_status sw_get_dt(const sw_grid* g, double* dt) {
  if (!g || !dt) return fail(SW_EINVAL, "NULL argument");
  if (!g->dt_ready) {
    if (g->dt_user > 0.0) {
      *dt = g->dt_user;
      return SW_OK;
    }
    return fail(SW_ESTATE, "automatic dt is resolved by sw_set_model");
  }
  *dt = g->dt;
  return SW_OK;
}

sw_status sw_ricker(double f_peak, double t0, double dt, int nt, float* out) {
  if (!out || nt < 0 || !(f_peak > 0.0) || !(dt > 0.0)) return fail(SW_EINVAL, "bad Ricker arguments");
  ricker(f_peak, t0, dt, nt, out);
  return SW_OK;
}

sw_status sw_set_stencil_variant(sw_grid* g, int variant) {
  if (!g) return fail(SW_EINVAL, "NULL grid");
  if (variant != SW_STENCIL_AUTO && variant != SW_STENCIL_PLAIN && variant != SW_STENCIL_TMA &&
      variant != SW_STENCIL_CLUSTER && variant != SW_STENCIL_TB2)
    return fail(SW_EINVAL, "unknown stencil variant %d", variant);
  if (variant == SW_STENCIL_TMA && g->ndim != 3) return fail(SW_EINVAL, "the pipelined stencil is 3D only");
  if (variant == SW_STENCIL_CLUSTER && g->ndim != 2) return fail(SW_EINVAL, "the cluster-resident run is 2D only");
  if (variant == SW_STENCIL_TB2 && g->ndim != 2) return fail(SW_EINVAL, "the two-step kernel is 2D only");
  g->variant = variant;
  ++g->config_gen;
  return SW_OK;
}

sw_status sw_set_pipeline_test(sw_grid* g, int starve, unsigned long long wait_limit_ns) {
  if (!g) return fail(SW_EINVAL, "NULL grid");
  g->starve = starve != 0;
  g->wait_limit_ns = wait_limit_ns ? wait_limit_ns : kWaitLimitNs;
  ++g->config_gen;
  return SW_OK;
}

sw_status sw_get_stencil_variant(const sw_grid* g, int* variant) {
  if (!g || !variant) return fail(SW_EINVAL, "NULL argument");
  ClusterShape cs;
  *variant = use_tma(g) ? SW_STENCIL_TMA
                        : (use_tb2(g) ? SW_STENCIL_TB2 : (use_cluster(g, &cs) ? SW_STENCIL_CLUSTER : SW_STENCIL_PLAIN));
  return SW_OK;
}

sw_status sw_set_forcing(sw_grid* g, int n_force, const float* fields, const float* signatures, int n_sig) {
  g_last_error.clear();
  if (!g) return fail(SW_EINVAL, "NULL grid");
  if (n_force < 0) return fail(SW_EINVAL, "n_force < 0");
  if (n_force > 0 && (!fields || !signatures || n_sig < 1))
    return fail(SW_EINVAL, "forcing needs fields, signatures and n_sig >= 1");
  ++g->config_gen;
  const int64_t nn = g->nodes();
  dev_free(g, g->force_F, size_t(g->n_force) * nn * sizeof(float));
  dev_free(g, g->force_T, size_t(g->n_force) * g->force_len * sizeof(float));
  g->force_F = g->force_T = nullptr;
  g->n_force = g->force_len = 0;
  if (n_force == 0) return SW_OK;
  float *F = nullptr, *T = nullptr;
  SW_TRY(dev_alloc(g, (void**)&F, size_t(n_force) * nn * sizeof(float)));
  const sw_status st = dev_alloc(g, (void**)&T, size_t(n_force) * n_sig * sizeof(float));
  if (st != SW_OK) {
    dev_free(g, F, size_t(n_force) * nn * sizeof(float));
    return st;
  }
  g->force_F = F;
  g->force_T = T;
  g->n_force = n_force;
  g->force_len = n_sig;
  SW_CUDA(cudaMemcpyAsync(F, fields, size_t(n_force) * nn * sizeof(float), cudaMemcpyDefault, g->stream));
  SW_CUDA(cudaMemcpyAsync(T, signatures, size_t(n_force) * n_sig * sizeof(float), cudaMemcpyDefault, g->stream));
  SW_CUDA(cudaStreamSynchronize(g->stream));
  return SW_OK;
}

sw_status sw_set_initial_state(sw_grid* g, const float* p0, const float* pm1) {
  g_last_error.clear();
  if (!g) return fail(SW_EINVAL, "NULL grid");
  const size_t bytes = size_t(g->nodes()) * sizeof(float);
  const float* src[2] = {p0, pm1};
  float** dst[2] = {&g->init_p0, &g->init_pm1};
  for (int i = 0; i < 2; ++i) {
    if (!src[i]) {
      dev_free(g, *dst[i], bytes);
      *dst[i] = nullptr;
      continue;
    }
    if (!*dst[i]) SW_TRY(dev_alloc(g, (void**)dst[i], bytes));
    SW_CUDA(cudaMemcpyAsync(*dst[i], src[i], bytes, cudaMemcpyDefault, g->stream));
  }
  SW_CUDA(cudaStreamSynchronize(g->stream));
  return SW_OK;
}

sw_status sw_set_checkpoint_budget(sw_grid* g, int max_states) {
  g_last_error.clear();
  if (!g) return fail(SW_EINVAL, "NULL grid");
  if (max_states < 0) return fail(SW_EINVAL, "negative checkpoint budget");
  g->ckpt_budget = max_states;
  return SW_OK;
}

sw_status sw_set_saving(sw_grid* g, int saving_stride, float* snapshots, int64_t max_frames) {
  g_last_error.clear();
  if (!g) return fail(SW_EINVAL, "NULL grid");
  if (saving_stride < 0 || max_frames < 0) return fail(SW_EINVAL, "negative saving stride or frame count");
  if (saving_stride > 0 && (!snapshots || max_frames == 0))
    return fail(SW_EINVAL, "a saving stride needs a snapshot buffer and a frame count");
  if (snapshots && !is_device_pointer(snapshots)) return fail(SW_EINVAL, "the snapshot buffer must be device memory");
  g->saving_stride = saving_stride;
  g->snapshots = saving_stride > 0 ? snapshots : nullptr;
  g->snapshot_frames = saving_stride > 0 ? max_frames : 0;
  ++g->config_gen;
  return SW_OK;
}

sw_status sw_set_profiling(sw_grid* g, int every) {
  if (!g) return fail(SW_EINVAL, "NULL grid");
  if (every < 0) return fail(SW_EINVAL, "negative profiling stride");
  g->profiling = every;
  ++g->config_gen;
  return SW_OK;
}

sw_status sw_get_profile(const sw_grid* g, double* stencil_ms, int64_t* stencil_launches,
                         int64_t* kernel_launches) {
  if (!g) return fail(SW_EINVAL, "NULL grid");
  if (stencil_ms) *stencil_ms = g->stencil_ms;
  if (stencil_launches) *stencil_launches = g->stencil_launches;
  if (kernel_launches) *kernel_launches = g->kernel_launches;
  return SW_OK;
}

sw_status sw_get_device_bytes(const sw_grid* g, int64_t* bytes) {
  if (!g || !bytes) return fail(SW_EINVAL, "NULL argument");
  *bytes = g->device_bytes;
  return SW_OK;
}

void sw_destroy_grid(sw_grid* g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  if (g->graph) cudaGraphExecDestroy(g->graph);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  free_acquisition(g);
  const size_t fbytes = size_t(g->lay.total) * sizeof(float);
  dev_free(g, g->u[0], fbytes);
  dev_free(g, g->u[1], fbytes);
  dev_free(g, g->u2[0], fbytes);
  dev_free(g, g->u2[1], fbytes);
  dev_free(g, g->kappa, fbytes);
  dev_free(g, g->lnrho, fbytes);
  for (int i = 0; i < 3; ++i) dev_free(g, g->glr[i], fbytes);
  dev_free(g, g->damp, size_t(g->damp_len) * sizeof(float2));
  dev_free(g, g->force_F, size_t(g->n_force) * g->nodes() * sizeof(float));
  dev_free(g, g->force_T, size_t(g->n_force) * g->force_len * sizeof(float));
  dev_free(g, g->init_p0, size_t(g->nodes()) * sizeof(float));
  dev_free(g, g->init_pm1, size_t(g->nodes()) * sizeof(float));
  dev_free(g, g->dflag, 64);
  dev_free(g, g->dscratch, 64);
  dev_free(g, g->staging, size_t(g->nodes()) * sizeof(float));
  dev_free(g, g->staging2, size_t(g->nodes()) * sizeof(float));
  dev_free(g, g->seis_staging, size_t(g->seis_staging_elems) * sizeof(float));
  for (cudaEvent_t e : g->events) cudaEventDestroy(e);
  delete g;
}

}  // extern "C"

// ---- allocation-free forward ------------------------------------------------
//
// sw_forward_noalloc runs the forward simulation of the handle-based calls for
// callers that cannot allocate device memory.  It always takes the plain
// per-step path (stencil_plain kernels, then separate source-injection and
// receiver-sampling launches per step), not the pipelined 3D kernel or the
// cluster-resident 2D run that sw_forward picks, so its results agree with
// sw_forward within the FP32 parity tolerance, not bit for bit, and its
// throughput is lower.  Everything the simulation needs besides the caller's
// inputs and outputs lives in one file-scope device array of
// SW_NOALLOC_SCRATCH_BYTES.

static __device__ __align__(256) float noalloc_scratch[SW_NOALLOC_SCRATCH_BYTES / sizeof(float)];

namespace {

// Device address of the scratch array on the current device.  Host code only
// sees a host-side stand-in under the array's name, so the address is looked
// up on every call with the caller's device current (no allocation; nothing
// is cached, so a torn-down and re-created context never sees a stale
// address).  The first lookup on a device may load the library's device code.
sw_status noalloc_scratch_address(float** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return fail(SW_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
  }
  *out = static_cast<float*>(p);
  return SW_OK;
}

// Bump carving of the scratch array in 256-byte units (host arithmetic only).
// A request larger than what is left marks the plan as over capacity instead
// of adding to `used`, so the running sum can never wrap.
struct ScratchCarver {
  float* base;
  size_t used;
  size_t cap;
  bool over = false;
  float* take(size_t floats) {
    if (over || floats > cap - used) {
      over = true;
      return nullptr;
    }
    const size_t n = (floats + 63) / 64 * 64;
    float* p = base ? base + used : nullptr;
    used = n > cap - used ? cap : used + n;
    return p;
  }
};

// One point's per-axis first node and weights (same windows and fitting as
// build_windows), written into fixed-size caller arrays.
sw_status noalloc_point_window(const sw_grid* g, const double* pos, bool fold_cell, int i, int* first3,
                               float* w3) {
  const int rw = g->rw, L = g->L;
  double cell = 1.0;
  for (int a = 0; a < g->ndim; ++a) cell *= (g->ndim == 3 ? g->h[a] : (a == 0 ? g->h[0] : g->h[2]));
  for (int k = 0; k < 3 * L; ++k) w3[k] = 0.f;
  first3[0] = first3[1] = first3[2] = 0;
  for (int a = 0; a < g->ndim; ++a) {
    const int axis = (g->ndim == 3) ? a : (a == 0 ? 0 : 2);
    const double coord = pos[size_t(i) * g->ndim + a];
    if (!std::isfinite(coord)) return fail(SW_EINVAL, "position %d is not finite", i);
    const double s = double(g->nbl[2 * axis]) + coord / g->h[axis];
    int64_t f0;
    double ww[2 * kMaxR], wf[2 * kMaxR];
    kaiser_sinc_weights(s, rw, &f0, ww);
    const int64_t nax = g->n[axis];
    if (2 * rw > nax) return fail(SW_EINVAL, "window longer than axis %d", axis);
    const int64_t nf = std::min(std::max<int64_t>(f0, 0), nax - 2 * rw);
    for (int j = 0; j < 2 * rw; ++j) wf[j] = 0.0;
    for (int j = 0; j < 2 * rw; ++j) {
      const int64_t node = f0 + j;
      if (node >= nf && node < nf + 2 * rw)
        wf[node - nf] = ww[j];
      else if (ww[j] != 0.0)
        return fail(SW_EINVAL, "window of point %d leaves the grid along axis %d", i, axis);
    }
    first3[axis] = int(nf);
    for (int j = 0; j < 2 * rw; ++j) {
      double v = wf[j];
      if (fold_cell && axis == 2) v /= cell;
      w3[axis * L + j] = float(v);
    }
  }
  if (g->ndim == 2) w3[1 * L] = 1.f;
  return SW_OK;
}

// Uploads the windows of `count` points in fixed-size chunks from the stack
// (pageable-source copies return once the source may be reused).
sw_status noalloc_upload_windows(const sw_grid* g, int count, const double* pos, bool fold_cell, int* dfirst,
                                 float* dw) {
  constexpr int kChunk = 32;
  int first[kChunk * 3];
  float w[kChunk * 3 * 2 * kMaxR];
  const int L = g->L;
  for (int i0 = 0; i0 < count; i0 += kChunk) {
    const int nc = std::min(kChunk, count - i0);
    for (int k = 0; k < nc; ++k)
      SW_TRY(noalloc_point_window(g, pos, fold_cell, i0 + k, first + 3 * k, w + 3 * L * k));
    SW_CUDA(cudaMemcpyAsync(dfirst + 3 * i0, first, size_t(nc) * 3 * sizeof(int), cudaMemcpyHostToDevice,
                            g->stream));
    SW_CUDA(cudaMemcpyAsync(dw + size_t(3) * L * i0, w, size_t(nc) * 3 * L * sizeof(float),
                            cudaMemcpyHostToDevice, g->stream));
  }
  return SW_OK;
}

}  // namespace

extern "C" sw_status sw_forward_noalloc(int ndim, const int64_t* shape, const double* spacing, int space_order,
                                        const int* nbl, const int* bc, double damp_alpha, int damp_degree,
                                        double dt, const float* velocity, const float* density, int n_src,
                                        const double* src_pos, int n_rec, const double* rec_pos, int nt,
                                        const float* wavelet, int wavelet_per_source, int window_radius,
                                        int n_steps, float* seismogram, float* final_field, void* cuda_stream) {
  g_last_error.clear();
  // -- arguments (same rules as sw_create_grid / sw_set_model / sw_set_acquisition / sw_forward)
  if (!shape || !spacing || !nbl || !bc || !velocity) return fail(SW_EINVAL, "NULL argument");
  if (ndim != 2 && ndim != 3) return fail(SW_EINVAL, "ndim must be 2 or 3 (got %d)", ndim);
  if (space_order < 2 || space_order > 2 * kMaxR || space_order % 2)
    return fail(SW_EINVAL, "space_order must be even in [2, 20] (got %d)", space_order);
  if (!(damp_alpha >= 0.0) || !std::isfinite(damp_alpha) || damp_degree < 0 || damp_degree > 16)
    return fail(SW_EINVAL, "damping parameters out of range");
  if (!std::isfinite(dt)) return fail(SW_EINVAL, "dt is not finite");
  if (n_src < 0 || n_rec < 0 || nt < 0 || n_steps < 0) return fail(SW_EINVAL, "negative count");
  if ((n_src > 0 && (!src_pos || !wavelet || nt == 0)) || (n_rec > 0 && !rec_pos))
    return fail(SW_EINVAL, "NULL positions or wavelet");
  if (window_radius < 1 || window_radius > kMaxR) return fail(SW_EINVAL, "window_radius must be in [1, 10]");
  if (n_src > 0 && n_steps > nt) return fail(SW_EINVAL, "n_steps (%d) exceeds the wavelet length (%d)", n_steps, nt);
  if (n_rec > 0 && n_steps > 0 && !seismogram) return fail(SW_EINVAL, "seismogram is NULL");

  sw_grid g;  // description only: every device pointer below points into the scratch array
  g.ndim = ndim;
  g.order = space_order;
  g.R = space_order / 2;
  for (int a = 0; a < ndim; ++a) {
    const int axis = (ndim == 3) ? a : (a == 0 ? 0 : 2);
    if (shape[a] < g.R + 1 || shape[a] > (int64_t(1) << 24))
      return fail(SW_EINVAL, "shape[%d] = %lld out of range", a, (long long)shape[a]);
    if (!(spacing[a] > 0.0) || !std::isfinite(spacing[a])) return fail(SW_EINVAL, "spacing[%d] must be positive", a);
    g.n[axis] = shape[a];
    g.h[axis] = spacing[a];
    for (int s = 0; s < 2; ++s) {
      const int nb = nbl[2 * a + s], b = bc[2 * a + s];
      if (nb < 0 || nb >= shape[a]) return fail(SW_EINVAL, "nbl[%d] out of range", 2 * a + s);
      if (b != SW_BC_NONE && b != SW_BC_DIRICHLET && b != SW_BC_NEUMANN)
        return fail(SW_EINVAL, "bc[%d] invalid", 2 * a + s);
      g.nbl[2 * axis + s] = nb;
      g.bc[2 * axis + s] = b;
    }
    if (nbl[2 * a] + nbl[2 * a + 1] >= shape[a]) return fail(SW_EINVAL, "absorbing layers cover the whole axis %d", a);
  }
  if (g.n[0] * g.n[1] * g.n[2] > (int64_t(1) << 34)) return fail(SW_EINVAL, "grid too large");
  g.alpha = damp_alpha;
  g.degree = damp_degree;
  g.dt_user = dt;
  g.stream = static_cast<cudaStream_t>(cuda_stream);
  g.lay.init(ndim, g.R, g.n);
  g.rw = window_radius;
  g.L = 2 * window_radius;
  g.lz = g.L;
  g.ly = (ndim == 3) ? g.L : 1;
  g.lx = g.L;
  g.n_src = n_src;
  g.n_rec = n_rec;
  g.nt = nt;
  g.sig_stride = wavelet_per_source ? nt : 0;
  g.has_density = density != nullptr;
  int64_t maxd2 = 0;
  for (int a = 0; a < 3; ++a) {
    const int64_t m = std::max(g.nbl[2 * a], g.nbl[2 * a + 1]);
    maxd2 += m * m;
  }
  g.damp_len = maxd2 + 1;

  // -- scratch plan; reject problems that do not fit before touching the device
  const size_t field = size_t(g.lay.total);
  const size_t wav_floats = size_t(n_src > 0 ? (wavelet_per_source ? n_src : 1) : 0) * size_t(nt);
  const size_t cap = SW_NOALLOC_SCRATCH_BYTES / sizeof(float);
  ScratchCarver plan{nullptr, 0, cap};
  plan.take(field);
  plan.take(field);
  plan.take(field);
  if (g.has_density) plan.take(field);
  plan.take(size_t(g.damp_len) * 2);
  plan.take(64);
  plan.take(size_t(n_src) * 3);
  plan.take(size_t(n_src) * 3 * g.L);
  plan.take(wav_floats);
  plan.take(size_t(n_rec) * 3);
  plan.take(size_t(n_rec) * 3 * g.L);
  if (plan.over) {
    const double need = 4.0 * (double(field) * (g.has_density ? 4.0 : 3.0) + double(wav_floats) +
                               double(g.damp_len) * 2.0 + double(n_src + n_rec) * 3.0 * (1.0 + g.L));
    return fail(SW_EINVAL, "problem needs about %.4g bytes of scratch; sw_forward_noalloc is limited to %zu bytes",
                need, size_t(SW_NOALLOC_SCRATCH_BYTES));
  }

  // grid-shaped inputs and outputs must already be device memory of the current
  // device (host staging would allocate; another device's memory is not reachable)
  if (!is_current_device_pointer(velocity) || (density && !is_current_device_pointer(density)) ||
      (seismogram && !is_current_device_pointer(seismogram)) ||
      (final_field && !is_current_device_pointer(final_field)))
    return fail(SW_EINVAL,
                "sw_forward_noalloc needs velocity, density and the outputs in device memory of the current device");
  if (n_src > 0 && is_other_device_pointer(wavelet))
    return fail(SW_EINVAL, "the wavelet is memory of another device");

  float* base = nullptr;
  SW_TRY(noalloc_scratch_address(&base));
  ScratchCarver sc{base, 0, cap};
  g.u[0] = sc.take(field);
  g.u[1] = sc.take(field);
  g.kappa = sc.take(field);
  g.lnrho = g.has_density ? sc.take(field) : nullptr;
  g.damp = reinterpret_cast<float2*>(sc.take(size_t(g.damp_len) * 2));
  g.dflag = reinterpret_cast<int*>(sc.take(64));
  g.dscratch = reinterpret_cast<unsigned*>(g.dflag + 16);
  g.src_first = reinterpret_cast<int*>(sc.take(size_t(n_src) * 3));
  g.src_w = sc.take(size_t(n_src) * 3 * g.L);
  g.wavelet = sc.take(wav_floats);
  g.rec_first = reinterpret_cast<int*>(sc.take(size_t(n_rec) * 3));
  g.rec_w = sc.take(size_t(n_rec) * 3 * g.L);

  // -- the array keeps the previous call's contents: clear what must start at zero
  const size_t fbytes = field * sizeof(float);
  SW_CUDA(cudaMemsetAsync(g.u[0], 0, fbytes, g.stream));
  SW_CUDA(cudaMemsetAsync(g.u[1], 0, fbytes, g.stream));
  SW_CUDA(cudaMemsetAsync(g.kappa, 0, fbytes, g.stream));
  if (g.lnrho) SW_CUDA(cudaMemsetAsync(g.lnrho, 0, fbytes, g.stream));
  SW_CUDA(cudaMemsetAsync(g.dflag, 0, 64 * sizeof(float), g.stream));

  // -- model: velocity range, dt (Eq. 8), kappa, damping table, ln(rho)
  const FaceInfo f = g.faces();
  const int64_t nn = g.nodes();
  const unsigned init[2] = {0u, 0x7f800000u};
  SW_CUDA(cudaMemcpyAsync(g.dscratch, init, sizeof(init), cudaMemcpyHostToDevice, g.stream));
  field_range_kernel<<<grid_blocks(nn, 256), 256, 0, g.stream>>>(velocity, nn, g.dscratch, g.dscratch + 1, g.dflag);
  if (density)
    field_range_kernel<<<grid_blocks(nn, 256), 256, 0, g.stream>>>(density, nn, g.dscratch + 2, g.dscratch + 3,
                                                                   g.dflag);
  SW_CUDA(cudaGetLastError());
  unsigned res[2];
  int bad = 0;
  SW_CUDA(cudaMemcpyAsync(res, g.dscratch, sizeof(res), cudaMemcpyDeviceToHost, g.stream));
  SW_CUDA(cudaMemcpyAsync(&bad, g.dflag, sizeof(int), cudaMemcpyDeviceToHost, g.stream));
  SW_CUDA(cudaStreamSynchronize(g.stream));
  if (bad) return fail(SW_EINVAL, "velocity and density must be finite and positive everywhere");
  float vmax;
  memcpy(&vmax, &res[0], sizeof(float));
  const double hh[3] = {g.h[0], ndim == 3 ? g.h[1] : g.h[2], g.h[2]};
  const double dtc = critical_dt(ndim, g.order, hh, double(vmax));
  if (dt <= 0.0)
    dt = dtc;
  else if (dt > dtc)
    return fail(SW_ECFL, "dt = %.6g s exceeds the stability bound %.6g s (c_max = %.6g m/s)", dt, dtc, double(vmax));
  g.dt = dt;
  kappa_kernel<<<grid_blocks(nn, 256), 256, 0, g.stream>>>(velocity, g.at0(g.kappa), f, dt);
  SW_CUDA(cudaGetLastError());
  {
    constexpr int kChunk = 512;
    float2 table[kChunk];
    for (int64_t d0 = 0; d0 < g.damp_len; d0 += kChunk) {
      const int nc = int(std::min<int64_t>(kChunk, g.damp_len - d0));
      for (int k = 0; k < nc; ++k) {
        double da, de;
        damping_coefficients(g.alpha, g.degree, dt, d0 + k, &da, &de);
        table[k] = make_float2(float(da), float(de));
      }
      SW_CUDA(cudaMemcpyAsync(g.damp + d0, table, size_t(nc) * sizeof(float2), cudaMemcpyHostToDevice, g.stream));
    }
  }
  if (density) {
    lnrho_kernel<<<grid_blocks(nn, 256), 256, 0, g.stream>>>(density, g.at0(g.lnrho), f);
    SW_CUDA(cudaGetLastError());
    for (int axis = 0; axis < 3; ++axis) {
      if (ndim == 2 && axis == 1) continue;
      mirror_even_kernel<<<grid_blocks(nn, 256), 256, 0, g.stream>>>(g.at0(g.lnrho), f, axis, g.R);
      SW_CUDA(cudaGetLastError());
    }
  }

  // -- acquisition
  if (n_src > 0) {
    SW_TRY(noalloc_upload_windows(&g, n_src, src_pos, true, g.src_first, g.src_w));
    SW_CUDA(cudaMemcpyAsync(g.wavelet, wavelet, wav_floats * sizeof(float), cudaMemcpyDefault, g.stream));
  }
  if (n_rec > 0) SW_TRY(noalloc_upload_windows(&g, n_rec, rec_pos, false, g.rec_first, g.rec_w));

  // -- time loop (as sw_forward)
  StencilArgs a = stencil_args(&g);
  const PointSet src = point_set(&g, true), rec = point_set(&g, false);
  const int src_threads = n_src * g.lz * g.ly * g.lx;
  for (int step = 0; step < n_steps; ++step) {
    a.pn = g.at0(g.u[step & 1]);
    a.pnm1 = g.at0(g.u[(step + 1) & 1]);
    a.pout = g.at0(g.u[(step + 1) & 1]);
    launch_stencil(g.R, ndim, g.has_density, a, g.stream);
    if (src_threads > 0)
      inject_sources_kernel<<<(src_threads + 127) / 128, 128, 0, g.stream>>>(a.pout, a.kappa, g.damp, src, g.wavelet,
                                                                            g.sig_stride, step, f, ndim, g.R);
    if (n_rec > 0)
      sample_receivers_kernel<<<(n_rec + 3) / 4, 128, 0, g.stream>>>(a.pout, rec, f, seismogram, step);
  }
  SW_CUDA(cudaGetLastError());
  if (final_field) {
    extract_kernel<<<grid_blocks(nn, 256), 256, 0, g.stream>>>(g.at0(g.u[n_steps & 1]), final_field, f);
    SW_CUDA(cudaGetLastError());
  }
  SW_CUDA(cudaMemcpyAsync(&bad, g.dflag, sizeof(int), cudaMemcpyDeviceToHost, g.stream));
  SW_CUDA(cudaStreamSynchronize(g.stream));
  if (bad) return fail(SW_ETIMEOUT, "a kernel raised the device error flag (0x%x)", bad);
  return SW_OK;
}

// ---- batched shots -----------------------------------------------------------

#include "batch.cuh"

struct sw_batch {
  std::vector<sw_grid*> grids;
  std::vector<uint64_t> gens;    // config_gen of every grid when the batch was made
  std::vector<int> slot_grid;    // shot-table slot -> grid index
  std::vector<int> grid_group;   // grid index -> group
  std::vector<BatchShot> shots;  // host copy of the shot table
  // one work list per tile height the tuner tries (kBatchZBs); `cfg` is the one in use
  BatchGroup* d_groups[3] = {nullptr, nullptr, nullptr};
  int total_items[3] = {0, 0, 0}, blocks[3] = {0, 0, 0}, smem[3] = {0, 0, 0};
  float tuned_us[3] = {0.f, 0.f, 0.f};  // one stencil launch per tile height, timed at creation
  int cfg = 1;
  BatchShot* d_shots = nullptr;
  int n_groups = 0, R = 0;
  int max_src_taps = 0, max_rec = 0, max_rec_warps = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = -1, last_steps = -1;
  int profiling = 0;
  std::vector<cudaEvent_t> events;
  double stencil_ms = 0.0;
  int64_t stencil_launches = 0, kernel_launches = 0;
  int64_t nodes_per_step = 0;
  // batches of 3D grids: one pipelined stencil launch and one face launch per
  // step for all grids (descriptors per level parity in device memory)
  bool is3d = false, iso = false;
  int units = 0, face_blocks = 0;
  TmaGridDesc* d_tdesc[2] = {nullptr, nullptr};
  std::vector<FaceBatchDesc> fdesc;
  FaceBatchDesc* d_fdesc = nullptr;
  std::vector<unsigned char*> d_live;  // per grid: per step, some source sample is non-zero
};

namespace {

using BatchFn = void (*)(const BatchGroup*, int, const BatchShot*, int, int, int*, unsigned long long);

template <int ZB>
void batch_variant(int R, BatchFn* fn, int* smem) {
#define SW_BATCH_R(RR)                                 \
  case RR:                                             \
    *fn = batch_stencil_2d_kernel<RR, ZB>;             \
    *smem = BatchSmem<RR, ZB>::BYTES;                  \
    break;
  switch (R) {
    SW_BATCH_R(1) SW_BATCH_R(2) SW_BATCH_R(3) SW_BATCH_R(4) SW_BATCH_R(5)
    SW_BATCH_R(6) SW_BATCH_R(7) SW_BATCH_R(8) SW_BATCH_R(9) SW_BATCH_R(10)
    default: *fn = nullptr; *smem = 0; break;
  }
#undef SW_BATCH_R
}

// The batched stencil for radius R and tile height kBatchZBs[cfg].
void batch_kernel(int R, int cfg, BatchFn* fn, int* smem) {
  if (cfg == 0) batch_variant<kBatchZBs[0]>(R, fn, smem);
  else if (cfg == 1) batch_variant<kBatchZBs[1]>(R, fn, smem);
  else batch_variant<kBatchZBs[2]>(R, fn, smem);
}

bool same_geometry(const sw_grid* a, const sw_grid* b) {
  if (a->ndim != b->ndim || a->R != b->R || a->dt != b->dt || a->alpha != b->alpha || a->degree != b->degree)
    return false;
  for (int i = 0; i < 3; ++i)
    if (a->n[i] != b->n[i] || a->h[i] != b->h[i]) return false;
  for (int i = 0; i < 6; ++i)
    if (a->nbl[i] != b->nbl[i] || a->bc[i] != b->bc[i]) return false;
  return true;
}

__global__ void differ_kernel(const unsigned* a, const unsigned* b, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (a[i] != b[i]) {
      *flag = 1;
      return;
    }
}

// Do two grids of the same geometry hold bit-identical kappa fields?
sw_status same_model(sw_grid* a, sw_grid* b, cudaStream_t st, bool* same) {
  SW_CUDA(cudaMemsetAsync(a->dflag, 0, sizeof(int), st));
  differ_kernel<<<grid_blocks(a->lay.total, 256), 256, 0, st>>>(
      reinterpret_cast<const unsigned*>(a->kappa), reinterpret_cast<const unsigned*>(b->kappa), a->lay.total, a->dflag);
  SW_CUDA(cudaGetLastError());
  int flag = 0;
  SW_CUDA(cudaMemcpyAsync(&flag, a->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  SW_CUDA(cudaStreamSynchronize(st));
  SW_CUDA(cudaMemsetAsync(a->dflag, 0, sizeof(int), st));
  *same = flag == 0;
  return SW_OK;
}

sw_status tune_batch(sw_batch* b) {
  cudaStream_t st = b->stream;
  for (sw_grid* g : b->grids) {
    const size_t fbytes = size_t(g->lay.total) * sizeof(float);
    SW_CUDA(cudaMemsetAsync(g->u[0], 0, fbytes, st));
    SW_CUDA(cudaMemsetAsync(g->u[1], 0, fbytes, st));
  }
  cudaEvent_t ev[2];
  SW_CUDA(cudaEventCreate(&ev[0]));
  SW_CUDA(cudaEventCreate(&ev[1]));
  float best = 0.f;
  sw_status status = SW_OK;
  for (int c = 0; c < 3 && status == SW_OK; ++c) {
    BatchFn fn = nullptr;
    int smem = 0;
    batch_kernel(b->R, c, &fn, &smem);
    const BatchGroup* dg = b->d_groups[c];
    const BatchShot* ds = b->d_shots;
    int ng = b->n_groups, nt = b->total_items[c];
    int* flag = b->grids[0]->dflag;
    unsigned long long limit = b->grids[0]->wait_limit_ns;
    constexpr int kWarm = 1, kTimed = 4;
    for (int i = 0; i < kWarm + kTimed && status == SW_OK; ++i) {
      int parity = i & 1;
      void* args[] = {&dg, &ng, &ds, &nt, &parity, &flag, &limit};
      if (i == kWarm && cudaEventRecord(ev[0], st) != cudaSuccess) status = fail(SW_ECUDA, "tuner event");
      const cudaError_t e = cudaLaunchKernel((const void*)fn, dim3(unsigned(b->blocks[c])), dim3(kBatchThreads), args,
                                             size_t(smem), st);
      if (e != cudaSuccess) status = fail(SW_ECUDA, "tuner launch: %s", cudaGetErrorString(e));
    }
    float ms = 0.f;
    if (status == SW_OK && (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess))
      status = fail(SW_ECUDA, "tuner timing");
    b->tuned_us[c] = 1000.f * ms / float(kTimed);
    if (status == SW_OK && (c == 0 || b->tuned_us[c] < best)) {
      best = b->tuned_us[c];
      b->cfg = c;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (status != SW_OK) return status;
  return check_device_flag(b->grids[0]);
}


// ---- batches of 3D grids ------------------------------------------------

template <int R, int TY, int PPT, int NB, int MINB, bool ISO>
void launch_tma_batch_iso(const sw_batch* b, int parity, cudaStream_t st) {
  using C = TmaConfig<R, TY, PPT, NB, false>;
  auto kern = stencil_tma_kernel<R, TY, PPT, NB, MINB, ISO, false, false, true>;
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, C::NT, C::SMEM);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const sw_grid* g0 = b->grids[0];
  TmaWork wk;
  wk.tiles_x = 1;
  wk.nz = 1;
  wk.total = b->units;
  wk.starve = g0->starve ? 1 : 0;
  wk.grids = b->d_tdesc[parity];
  wk.n_grids = int(b->grids.size());
  long long grid = (long long)g0->sm_count * blocks_per_sm;
  if (grid > wk.total) grid = wk.total;
  // the kernel's own maps and arguments are not read in a batch (each grid's
  // come from its descriptor); grid 0's stand in
  const StencilArgs a0 = stencil_args(g0);
  launch_dependent(kern, dim3(unsigned(grid)), dim3(C::NT), C::SMEM, st, g0->map_halo[0], g0->map_inner[0],
                   g0->map_warm[0], g0->map_inner[1], g0->map_kappa, g0->map_kappa, g0->map_kappa, g0->map_kappa, a0,
                   wk, g0->dflag, g0->wait_limit_ns);
}

template <int R, int TY, int PPT, int NB, int MINB>
void launch_tma_batch_t(const sw_batch* b, int parity, cudaStream_t st) {
  if (b->iso)
    launch_tma_batch_iso<R, TY, PPT, NB, MINB, true>(b, parity, st);
  else
    launch_tma_batch_iso<R, TY, PPT, NB, MINB, false>(b, parity, st);
}

// One step's stencil for every grid of a 3D batch (the tile shapes of the
// single-grid constant-density kernel).
void launch_stencil_tma_batch(const sw_batch* b, int parity, cudaStream_t st) {
  switch (b->R) {
    case 1: launch_tma_batch_t<1, 16, 4, 3, 3>(b, parity, st); break;
    case 2: launch_tma_batch_t<2, 16, 4, 3, 3>(b, parity, st); break;
    case 3: launch_tma_batch_t<3, 16, 4, 3, 3>(b, parity, st); break;
    case 4: launch_tma_batch_t<4, 16, 4, 3, 3>(b, parity, st); break;
    case 5: launch_tma_batch_t<5, 16, 2, 4, 2>(b, parity, st); break;
    case 6: launch_tma_batch_t<6, 16, 2, 4, 2>(b, parity, st); break;
    case 7: launch_tma_batch_t<7, 16, 2, 4, 1>(b, parity, st); break;
    case 8: launch_tma_batch_t<8, 16, 2, 4, 1>(b, parity, st); break;
    case 9: launch_tma_batch_t<9, 16, 2, 4, 1>(b, parity, st); break;
    case 10: launch_tma_batch_t<10, 16, 2, 4, 1>(b, parity, st); break;
    default: break;
  }
}

void launch_face_batch(const sw_batch* b, int step, int n_steps, cudaStream_t st) {
  const int n = int(b->grids.size());
  // a persistent grid walks every grid's face blocks (many small faces: no block launched per 256 positions)
  const int total = b->face_blocks;
  const dim3 grid(unsigned(std::min(total, b->grids[0]->sm_count * 8))), block(256);
  switch (b->R) {
    case 1: launch_dependent(face_batch_kernel<1>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 2: launch_dependent(face_batch_kernel<2>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 3: launch_dependent(face_batch_kernel<3>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 4: launch_dependent(face_batch_kernel<4>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 5: launch_dependent(face_batch_kernel<5>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 6: launch_dependent(face_batch_kernel<6>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 7: launch_dependent(face_batch_kernel<7>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 8: launch_dependent(face_batch_kernel<8>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 9: launch_dependent(face_batch_kernel<9>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    case 10: launch_dependent(face_batch_kernel<10>, grid, block, 0, st, (const FaceBatchDesc*)b->d_fdesc, n, total, step, n_steps); break;
    default: break;
  }
}


void free_batch_3d(sw_batch* b) {
  for (int c = 0; c < 2; ++c) cudaFree(b->d_tdesc[c]);
  cudaFree(b->d_fdesc);
  for (unsigned char* p : b->d_live) cudaFree(p);
  b->d_live.clear();
}

// A batch of 3D grids of constant density: one work list of (64 x 16 tile,
// plane) items over every grid for the pipelined stencil, one face launch
// of every grid's blocks.  The grids keep their own levels, tensor maps,
// model and acquisition; each grid's sources enter through p[n-1]
// (PreInject), so their windows must not lie where eta dt reaches 1/2.
sw_status create_batch_3d(sw_batch** out, sw_grid* const* grids, int n) {
  const sw_grid* g0 = grids[0];
  auto iso_of = [](const sw_grid* g) { return g->h[0] == g->h[1] && g->h[1] == g->h[2]; };
  int64_t units = 0, face_blocks = 0;
  for (int i = 0; i < n; ++i) {
    const sw_grid* g = grids[i];
    if (!g) return fail(SW_EINVAL, "grid %d is NULL", i);
    if (!g->has_model || !g->has_acq) return fail(SW_ESTATE, "grid %d has no model or acquisition yet", i);
    if (g->ndim != 3) return fail(SW_EINVAL, "a batch holds grids of one dimension (grid %d)", i);
    if (g->has_density) return fail(SW_EINVAL, "batches hold constant-density grids only (grid %d)", i);
    if (g->R != g0->R) return fail(SW_EINVAL, "all grids of a batch need one space order (grid %d)", i);
    if (iso_of(g) != iso_of(g0))
      return fail(SW_EINVAL, "3D batches need equal spacings along the axes in every grid or in none (grid %d)", i);
    if (g->stream != g0->stream || g->device != g0->device)
      return fail(SW_EINVAL, "all grids of a batch need one device and stream (grid %d)", i);
    if (g->n_force > 0 || g->snapshots) return fail(SW_EINVAL, "grid %d has forcing or snapshots set", i);
    if (!use_tma(g)) return fail(SW_EINVAL, "grid %d cannot use the pipelined 3D kernel", i);
    for (int j = 0; j < i; ++j)
      if (grids[j] == g) return fail(SW_EINVAL, "grid %d appears twice", i);
    if (g->n_src > 0) {
      double sa, se;
      damping_coefficients(g->alpha, g->degree, g->dt, g->src_d2_max, &sa, &se);
      if (!(se < 0.5)) return fail(SW_EINVAL, "grid %d has source windows too deep in the absorbing layers", i);
    }
    const int64_t tiles = ((g->n[2] + 63) / 64) * ((g->n[1] + 15) / 16);
    units += tiles * g->n[0];
    const FaceGrid fg = face_grid(g->faces(), g->R, g->n_rec, g->n_src * g->lz * g->ly * g->lx, true);
    face_blocks += fg.total();
  }
  if (units >= (int64_t(1) << 31) || face_blocks >= (int64_t(1) << 31))
    return fail(SW_EINVAL, "the batch is too large for one work list");
  sw_batch* b = new sw_batch();
  b->is3d = true;
  b->iso = iso_of(g0);
  b->grids.assign(grids, grids + n);
  b->R = g0->R;
  b->stream = g0->stream;
  b->units = int(units);
  b->face_blocks = int(face_blocks);
  b->n_groups = n;
  std::vector<TmaGridDesc> td[2];
  b->fdesc.resize(size_t(n));
  int unit0 = 0, block0 = 0;
  for (int i = 0; i < n; ++i) {
    sw_grid* g = grids[i];
    b->gens.push_back(g->config_gen);
    b->nodes_per_step += g->nodes();
    const int tx = int((g->n[2] + 63) / 64), ty = int((g->n[1] + 15) / 16);
    for (int par = 0; par < 2; ++par) {
      TmaGridDesc D;
      memset(&D, 0, sizeof(D));
      D.c = g->map_halo[par];
      D.f = g->map_inner[par];
      D.w = g->map_warm[par];
      D.o = g->map_inner[par ^ 1];
      D.k = g->map_kappa;
      D.a = stencil_args(g);
      D.a.pn = g->at0(g->u[par]);
      D.a.pnm1 = g->at0(g->u[par ^ 1]);
      D.a.pout = g->at0(g->u[par ^ 1]);
      D.unit0 = unit0;
      D.tiles_x = tx;
      D.nz = int(g->n[0]);
      td[par].push_back(D);
    }
    unit0 += tx * ty * int(g->n[0]);
    const int taps = g->lz * g->ly * g->lx;
    if (g->n_src > 0 && !g->tap_off) {  // the source tap table (filled by every batch forward)
      const size_t nt = size_t(g->n_src) * taps;
      sw_status st = dev_alloc(g, (void**)&g->tap_off, nt * sizeof(int64_t));
      if (st == SW_OK) st = dev_alloc(g, (void**)&g->tap_coef, nt * sizeof(float));
      if (st == SW_OK) st = dev_alloc(g, (void**)&g->tap_pre, nt * sizeof(float));
      if (st != SW_OK) {
        free_batch_3d(b);
        delete b;
        return st;
      }
    }
    unsigned char* live = nullptr;
    if (g->n_src > 0) {
      if (cudaMalloc((void**)&live, g->sig_live.size()) != cudaSuccess) {
        cudaGetLastError();
        free_batch_3d(b);
        delete b;
        return fail(SW_ENOMEM, "cudaMalloc of the batch's step table failed");
      }
      b->d_live.push_back(live);
      cudaMemcpyAsync(live, g->sig_live.data(), g->sig_live.size(), cudaMemcpyHostToDevice, b->stream);
    }
    FaceBatchDesc& F = b->fdesc[size_t(i)];
    memset(&F, 0, sizeof(F));
    F.lv[0] = g->at0(g->u[0]);
    F.lv[1] = g->at0(g->u[1]);
    F.f = g->faces();
    F.rec = point_set(g, false);
    F.seis = nullptr;
    F.fg = face_grid(F.f, g->R, g->n_rec, g->n_src * taps, true);
    F.tap_off = g->tap_off;
    F.tap_pre = g->tap_pre;
    F.sig = g->wavelet;
    F.live = live;
    F.taps = taps;
    F.n_src = g->n_src;
    F.sig_stride = g->sig_stride;
    F.block0 = block0;
    block0 += F.fg.total();
  }
  bool ok = true;
  for (int par = 0; par < 2 && ok; ++par)
    ok = cudaMalloc((void**)&b->d_tdesc[par], size_t(n) * sizeof(TmaGridDesc)) == cudaSuccess &&
         cudaMemcpyAsync(b->d_tdesc[par], td[par].data(), size_t(n) * sizeof(TmaGridDesc), cudaMemcpyHostToDevice,
                         b->stream) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&b->d_fdesc, size_t(n) * sizeof(FaceBatchDesc)) == cudaSuccess &&
       cudaMemcpyAsync(b->d_fdesc, b->fdesc.data(), size_t(n) * sizeof(FaceBatchDesc), cudaMemcpyHostToDevice,
                       b->stream) == cudaSuccess &&
       cudaStreamSynchronize(b->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_batch_3d(b);
    delete b;
    return fail(SW_ENOMEM, "device memory for the batch's descriptors");
  }
  *out = b;
  return SW_OK;
}

sw_status batch_forward_3d(sw_batch* b, int n_steps, float* const* seismograms, float* const* final_fields) {
  const int n = int(b->grids.size());
  for (int i = 0; i < n; ++i) {
    const sw_grid* g = b->grids[size_t(i)];
    if (g->config_gen != b->gens[size_t(i)] || g->n_force > 0 || g->snapshots || !use_tma(g))
      return fail(SW_ESTATE, "grid %d changed after sw_create_batch", i);
    if (g->n_src > 0 && n_steps > g->nt)
      return fail(SW_EINVAL, "n_steps (%d) exceeds the wavelet length of grid %d (%d)", n_steps, i, g->nt);
    if (g->n_rec > 0 && n_steps > 0) {
      if (!seismograms || !seismograms[i]) return fail(SW_EINVAL, "seismogram of grid %d is NULL", i);
      if (!is_device_pointer(seismograms[i])) return fail(SW_EINVAL, "seismogram of grid %d is not device memory", i);
    }
  }
  cudaStream_t st = b->stream;
  bool changed = false;
  for (int i = 0; i < n; ++i) {
    float* sp = (b->grids[size_t(i)]->n_rec > 0 && n_steps > 0) ? seismograms[i] : nullptr;
    if (b->fdesc[size_t(i)].seis != sp) {
      b->fdesc[size_t(i)].seis = sp;
      changed = true;
    }
  }
  if (changed) {
    SW_CUDA(cudaMemcpyAsync(b->d_fdesc, b->fdesc.data(), b->fdesc.size() * sizeof(FaceBatchDesc),
                            cudaMemcpyHostToDevice, st));
    SW_CUDA(cudaStreamSynchronize(st));  // the host table may change again on the next call
  }
  int64_t launches = 0;
  for (sw_grid* g : b->grids) {  // levels from rest (or the initial state), source taps, step 0's sources
    const size_t fbytes = size_t(g->lay.total) * sizeof(float);
    SW_CUDA(cudaMemsetAsync(g->u[0], 0, fbytes, st));
    SW_CUDA(cudaMemsetAsync(g->u[1], 0, fbytes, st));
    const FaceInfo f = g->faces();
    if (g->init_p0) {
      insert_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(g->init_p0, g->at0(g->u[0]), f, 3, g->R);
      ++launches;
    }
    if (g->init_pm1) {
      insert_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(g->init_pm1, g->at0(g->u[1]), f, 3, g->R);
      ++launches;
    }
    const int src_threads = g->n_src * g->lz * g->ly * g->lx;
    if (src_threads > 0) {
      source_taps_kernel<<<(src_threads + 127) / 128, 128, 0, st>>>(g->at0(g->kappa), g->damp, point_set(g, true), f,
                                                                    g->tap_off, g->tap_coef, g->tap_pre);
      ++launches;
      if (n_steps > 0 && g->live(0)) {  // step 0's sources, into p[-1]
        inject_taps_kernel<<<(src_threads + 127) / 128, 128, 0, st>>>(
            g->at0(g->u[1]), g->tap_off, g->tap_pre, g->lz * g->ly * g->lx, g->n_src, g->wavelet, g->sig_stride, 0);
        ++launches;
      }
    }
  }
  SW_CUDA(cudaGetLastError());
  const int timed = b->profiling ? (n_steps + b->profiling - 1) / b->profiling : 0;
  if (timed && b->events.size() < size_t(2 * timed)) {
    const size_t old = b->events.size();
    b->events.resize(size_t(2 * timed));
    for (size_t i = old; i < b->events.size(); ++i) SW_CUDA(cudaEventCreate(&b->events[i]));
  }
  // per step: the stencil of every grid, then every grid's face conditions,
  // receiver samples and next step's sources
  auto enqueue = [&](cudaStream_t s, bool capturing) -> sw_status {
    const unsigned evflags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    for (int step = 0; step < n_steps; ++step) {
      const bool time_it = b->profiling && step % b->profiling == 0;
      const int ev = time_it ? 2 * (step / b->profiling) : 0;
      if (time_it) SW_CUDA(cudaEventRecordWithFlags(b->events[size_t(ev)], s, evflags));
      launch_stencil_tma_batch(b, step & 1, s);
      if (time_it) SW_CUDA(cudaEventRecordWithFlags(b->events[size_t(ev + 1)], s, evflags));
      launch_face_batch(b, step, n_steps, s);
    }
    SW_CUDA(cudaGetLastError());
    return SW_OK;
  };
  if (n_steps > 0 && b->graph && b->graph_steps == n_steps) {
    SW_CUDA(cudaGraphLaunch(b->graph, st));
  } else if (n_steps > 0 && b->last_steps == n_steps) {
    // second call with this length: capture the time loop once, replay it after
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      b->graph_steps = -1;
    }
    if (!b->cap_stream) SW_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    SW_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const sw_status s1 = enqueue(b->cap_stream, true);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (s1 != SW_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return s1 != SW_OK ? s1 : fail(SW_ECUDA, "capturing the batch time loop failed: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      b->graph = nullptr;
      return fail(SW_ECUDA, "instantiating the batch time loop failed: %s", cudaGetErrorString(ei));
    }
    b->graph_steps = n_steps;
    SW_CUDA(cudaGraphLaunch(b->graph, st));
  } else if (n_steps > 0) {
    SW_TRY(enqueue(st, false));
  }
  if (n_steps > 0) b->last_steps = n_steps;
  launches += 2 * int64_t(n_steps);
  for (int i = 0; final_fields && i < n; ++i) {
    if (!final_fields[i]) continue;
    sw_grid* g = b->grids[size_t(i)];
    float* dst = final_fields[i];
    const bool fh = !is_device_pointer(dst);
    if (fh) {
      if (!g->staging) SW_TRY(dev_alloc(g, (void**)&g->staging, size_t(g->nodes()) * sizeof(float)));
      dst = g->staging;
    }
    extract_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(g->at0(g->u[n_steps & 1]), dst, g->faces());
    SW_CUDA(cudaGetLastError());
    ++launches;
    if (fh)
      SW_CUDA(cudaMemcpyAsync(final_fields[i], dst, size_t(g->nodes()) * sizeof(float), cudaMemcpyDefault, st));
  }
  SW_TRY(check_device_flag(b->grids[0]));  // synchronises
  b->kernel_launches = launches;
  b->stencil_launches = timed;
  b->stencil_ms = 0.0;
  for (int i = 0; i < timed; ++i) {
    float ms = 0.f;
    SW_CUDA(cudaEventElapsedTime(&ms, b->events[size_t(2 * i)], b->events[size_t(2 * i + 1)]));
    b->stencil_ms += ms;
  }
  return SW_OK;
}
}  // namespace

extern "C" {

sw_status sw_create_batch(sw_batch** out, sw_grid* const* grids, int n_grids) {
  g_last_error.clear();
  if (!out || !grids || n_grids < 1) return fail(SW_EINVAL, "NULL argument or empty batch");
  *out = nullptr;
  const sw_grid* g0 = grids[0];
  if (g0 && g0->ndim == 3) return create_batch_3d(out, grids, n_grids);
  for (int i = 0; i < n_grids; ++i) {
    const sw_grid* g = grids[i];
    if (!g) return fail(SW_EINVAL, "grid %d is NULL", i);
    if (!g->has_model || !g->has_acq) return fail(SW_ESTATE, "grid %d has no model or acquisition yet", i);
    if (g->ndim != 2) return fail(SW_EINVAL, "batches hold 2D grids only (grid %d)", i);
    if (g->has_density) return fail(SW_EINVAL, "batches hold constant-density grids only (grid %d)", i);
    if (g->R != g0->R) return fail(SW_EINVAL, "all grids of a batch need one space order (grid %d)", i);
    if (g->stream != g0->stream || g->device != g0->device)
      return fail(SW_EINVAL, "all grids of a batch need one device and stream (grid %d)", i);
    if (g->n_force > 0 || g->snapshots) return fail(SW_EINVAL, "grid %d has forcing or snapshots set", i);
    if (g->lay.total >= (int64_t(1) << 31)) return fail(SW_EINVAL, "grid %d is too large for a batch", i);
    for (int j = 0; j < i; ++j)
      if (grids[j] == g) return fail(SW_EINVAL, "grid %d appears twice", i);
  }
  sw_batch* b = new sw_batch();
  b->grids.assign(grids, grids + n_grids);
  b->R = g0->R;
  b->stream = g0->stream;
  // groups: grids of the same geometry with bit-identical kappa
  std::vector<std::vector<int>> members;
  b->grid_group.assign(size_t(n_grids), -1);
  for (int i = 0; i < n_grids; ++i) {
    b->gens.push_back(grids[i]->config_gen);
    for (size_t k = 0; k < members.size() && b->grid_group[size_t(i)] < 0; ++k) {
      sw_grid* rep = grids[members[k][0]];
      if (!same_geometry(rep, grids[i])) continue;
      bool same = false;
      const sw_status st = same_model(rep, grids[i], b->stream, &same);
      if (st != SW_OK) {
        delete b;
        return st;
      }
      if (same) {
        members[k].push_back(i);
        b->grid_group[size_t(i)] = int(k);
      }
    }
    if (b->grid_group[size_t(i)] < 0) {
      b->grid_group[size_t(i)] = int(members.size());
      members.push_back({i});
    }
  }
  std::vector<BatchGroup> groups;
  double v[kMaxR + 1];
  fd_second_weights(g0->order, v);
  for (const auto& m : members) {
    const sw_grid* g = grids[m[0]];
    BatchGroup G;
    memset(&G, 0, sizeof(G));
    G.kappa = g->at0(g->kappa);
    G.damp = g->damp;
    G.sz = g->lay.sz;
    G.nz = int(g->n[0]);
    G.nx = int(g->n[2]);
    const int faces[4] = {0, 1, 4, 5};
    for (int k = 0; k < 4; ++k) {
      G.nbl[k] = g->nbl[faces[k]];
      G.bc[k] = g->bc[faces[k]];
    }
    for (int j = 1; j <= g->R; ++j) {
      G.cz[j] = float(v[j] / (g->h[0] * g->h[0]));
      G.cx[j] = float(v[j] / (g->h[2] * g->h[2]));
    }
    G.first = int(b->slot_grid.size());
    G.count = int(m.size());
    G.tiles_x = (G.nx + kBatchTX - 1) / kBatchTX;
    G.item_base = 0;  // per tile height, below
    for (int i : m) {
      sw_grid* s = grids[i];
      b->slot_grid.push_back(i);
      BatchShot S;
      memset(&S, 0, sizeof(S));
      S.u[0] = s->at0(s->u[0]);
      S.u[1] = s->at0(s->u[1]);
      S.src = point_set(s, true);
      S.rec = point_set(s, false);
      S.kappa = s->at0(s->kappa);
      S.damp = s->damp;
      S.f = s->faces();
      S.wavelet = s->wavelet;
      S.sig_stride = s->sig_stride;
      S.seis = nullptr;
      b->shots.push_back(S);
      b->max_src_taps = std::max(b->max_src_taps, s->n_src * s->lz * s->ly * s->lx);
      b->max_rec = std::max(b->max_rec, s->n_rec);
      b->max_rec_warps = std::max(b->max_rec_warps, grouped_receiver_warps(S.rec));
      b->nodes_per_step += s->nodes();
    }
    groups.push_back(G);
  }
  b->n_groups = int(groups.size());
  // one work list, occupancy and launch size per tile height
  cudaError_t e = cudaMalloc((void**)&b->d_shots, b->shots.size() * sizeof(BatchShot));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_shots, b->shots.data(), b->shots.size() * sizeof(BatchShot), cudaMemcpyHostToDevice,
                        b->stream);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
    int items = 0;
    for (BatchGroup& G : groups) {
      G.item_base = items;
      items += G.tiles_x * ((G.nz + kBatchZBs[c] - 1) / kBatchZBs[c]) * G.count;
    }
    b->total_items[c] = items;
    BatchFn fn = nullptr;
    batch_kernel(b->R, c, &fn, &b->smem[c]);
    int per_sm = 0;
    e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b->smem[c]);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, size_t(b->smem[c]));
    if (e == cudaSuccess) {
      b->blocks[c] = std::max(1, std::min(items, std::max(per_sm, 1) * std::max(g0->sm_count, 1)));
      e = cudaMalloc((void**)&b->d_groups[c], groups.size() * sizeof(BatchGroup));
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_groups[c], groups.data(), groups.size() * sizeof(BatchGroup), cudaMemcpyHostToDevice,
                          b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // the host table changes for the next height
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    sw_destroy_batch(b);
    return fail(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, "batch set-up failed: %s",
                cudaGetErrorString(e));
  }
  // tuner: time a few stencil launches with every tile height on this batch
  // (zeroed fields; every forward zeroes them again) and keep the fastest
  const sw_status ts = tune_batch(b);
  if (ts != SW_OK) {
    std::string msg = g_last_error;
    sw_destroy_batch(b);
    g_last_error = msg;
    return ts;
  }
  *out = b;
  return SW_OK;
}

sw_status sw_batch_info(const sw_batch* b, int* n_groups, int* n_items) {
  if (!b) return fail(SW_EINVAL, "NULL batch");
  if (n_groups) *n_groups = b->n_groups;
  if (n_items) *n_items = b->is3d ? b->units : b->total_items[b->cfg];
  return SW_OK;
}

sw_status sw_batch_get_tile(const sw_batch* b, int* tile_rows, float* tuned_us) {
  if (!b) return fail(SW_EINVAL, "NULL batch");
  if (tile_rows) *tile_rows = kBatchZBs[b->cfg];
  if (tuned_us)
    for (int c = 0; c < 3; ++c) tuned_us[c] = b->tuned_us[c];
  return SW_OK;
}

sw_status sw_batch_set_tile(sw_batch* b, int tile_rows) {
  if (!b) return fail(SW_EINVAL, "NULL batch");
  if (b->is3d) return fail(SW_EINVAL, "a 3D batch has the pipelined kernel's tiles");
  for (int c = 0; c < 3; ++c)
    if (kBatchZBs[c] == tile_rows) {
      if (c != b->cfg) {
        b->cfg = c;
        b->last_steps = -1;  // the captured loop holds the old kernel: capture anew
        if (b->graph) {
          cudaGraphExecDestroy(b->graph);
          b->graph = nullptr;
          b->graph_steps = -1;
        }
      }
      return SW_OK;
    }
  return fail(SW_EINVAL, "tile height %d is not one of 16, 32, 64", tile_rows);
}

sw_status sw_batch_set_profiling(sw_batch* b, int every) {
  if (!b) return fail(SW_EINVAL, "NULL batch");
  if (every < 0) return fail(SW_EINVAL, "negative profiling stride");
  b->profiling = every;
  b->last_steps = -1;  // the captured loop has no timing events: capture anew
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = -1;
  }
  return SW_OK;
}

sw_status sw_batch_get_profile(const sw_batch* b, double* stencil_ms, int64_t* stencil_launches,
                               int64_t* kernel_launches) {
  if (!b) return fail(SW_EINVAL, "NULL batch");
  if (stencil_ms) *stencil_ms = b->stencil_ms;
  if (stencil_launches) *stencil_launches = b->stencil_launches;
  if (kernel_launches) *kernel_launches = b->kernel_launches;
  return SW_OK;
}

sw_status sw_batch_forward(sw_batch* b, int n_steps, float* const* seismograms, float* const* final_fields) {
  g_last_error.clear();
  if (!b) return fail(SW_EINVAL, "NULL batch");
  if (n_steps < 0) return fail(SW_EINVAL, "n_steps < 0");
  if (b->is3d) return batch_forward_3d(b, n_steps, seismograms, final_fields);
  const int n = int(b->grids.size());
  for (int i = 0; i < n; ++i) {
    const sw_grid* g = b->grids[size_t(i)];
    if (g->config_gen != b->gens[size_t(i)] || g->n_force > 0 || g->snapshots)
      return fail(SW_ESTATE, "grid %d changed after sw_create_batch", i);
    if (g->n_src > 0 && n_steps > g->nt)
      return fail(SW_EINVAL, "n_steps (%d) exceeds the wavelet length of grid %d (%d)", n_steps, i, g->nt);
    if (g->n_rec > 0 && n_steps > 0) {
      if (!seismograms || !seismograms[i]) return fail(SW_EINVAL, "seismogram of grid %d is NULL", i);
      if (!is_device_pointer(seismograms[i])) return fail(SW_EINVAL, "seismogram of grid %d is not device memory", i);
    }
  }
  cudaStream_t st = b->stream;
  // the seismogram pointers of this call into the shot table
  bool changed = false;
  for (size_t k = 0; k < b->shots.size(); ++k) {
    const int i = b->slot_grid[k];
    float* s = (b->grids[size_t(i)]->n_rec > 0 && n_steps > 0) ? seismograms[i] : nullptr;
    if (b->shots[k].seis != s) {
      b->shots[k].seis = s;
      changed = true;
    }
  }
  if (changed) {
    SW_CUDA(cudaMemcpyAsync(b->d_shots, b->shots.data(), b->shots.size() * sizeof(BatchShot),
                            cudaMemcpyHostToDevice, st));
    SW_CUDA(cudaStreamSynchronize(st));  // the host table may change again on the next call
  }
  for (sw_grid* g : b->grids) {
    const size_t fbytes = size_t(g->lay.total) * sizeof(float);
    SW_CUDA(cudaMemsetAsync(g->u[0], 0, fbytes, st));
    SW_CUDA(cudaMemsetAsync(g->u[1], 0, fbytes, st));
    const FaceInfo f = g->faces();
    if (g->init_p0)
      insert_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(g->init_p0, g->at0(g->u[0]), f, 2, g->R);
    if (g->init_pm1)
      insert_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(g->init_pm1, g->at0(g->u[1]), f, 2, g->R);
  }
  SW_CUDA(cudaGetLastError());
  const int timed = b->profiling ? (n_steps + b->profiling - 1) / b->profiling : 0;
  if (timed && b->events.size() < size_t(2 * timed)) {
    const size_t old = b->events.size();
    b->events.resize(size_t(2 * timed));
    for (size_t i = old; i < b->events.size(); ++i) SW_CUDA(cudaEventCreate(&b->events[i]));
  }
  BatchFn fn = nullptr;
  int smem_c = 0;
  batch_kernel(b->R, b->cfg, &fn, &smem_c);
  const int n_shots = int(b->shots.size());
  int64_t launches = 0;
  auto enqueue = [&](cudaStream_t s, bool capturing) -> sw_status {
    const unsigned evflags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    launches = 0;
    for (int step = 0; step < n_steps; ++step) {
      int parity = step & 1;
      const bool time_it = b->profiling && step % b->profiling == 0;
      const int ev = time_it ? 2 * (step / b->profiling) : 0;
      if (time_it) SW_CUDA(cudaEventRecordWithFlags(b->events[size_t(ev)], s, evflags));
      const BatchGroup* dg = b->d_groups[b->cfg];
      const BatchShot* ds = b->d_shots;
      int ng = b->n_groups, nt = b->total_items[b->cfg];
      int* flag = b->grids[0]->dflag;
      unsigned long long limit = b->grids[0]->wait_limit_ns;
      void* args[] = {&dg, &ng, &ds, &nt, &parity, &flag, &limit};
      SW_CUDA(cudaLaunchKernel((const void*)fn, dim3(unsigned(b->blocks[b->cfg])), dim3(kBatchThreads), args,
                               size_t(smem_c), s));
      if (time_it) SW_CUDA(cudaEventRecordWithFlags(b->events[size_t(ev + 1)], s, evflags));
      ++launches;
      if (b->max_src_taps > 0) {
        batch_inject_kernel<<<dim3((b->max_src_taps + 127) / 128, n_shots), 128, 0, s>>>(b->d_shots, step, parity,
                                                                                         b->R);
        ++launches;
      }
      if (b->max_rec > 0 && n_steps > 0) {
        batch_receivers_kernel<<<dim3(unsigned((b->max_rec_warps + 3) / 4), n_shots), 128, 0, s>>>(b->d_shots, step,
                                                                                                   parity);
        ++launches;
      }
    }
    SW_CUDA(cudaGetLastError());
    return SW_OK;
  };
  if (n_steps > 0 && b->graph && b->graph_steps == n_steps) {
    SW_CUDA(cudaGraphLaunch(b->graph, st));
  } else if (n_steps > 0 && b->last_steps == n_steps) {
    // second call with this length: capture the time loop once, replay it after
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      b->graph_steps = -1;
    }
    // captured on a private stream, launched on the batch's stream after the zeroing above
    if (!b->cap_stream) SW_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    SW_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    const sw_status s1 = enqueue(b->cap_stream, true);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (s1 != SW_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return s1 != SW_OK ? s1 : fail(SW_ECUDA, "capturing the batch time loop failed: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      b->graph = nullptr;
      return fail(SW_ECUDA, "instantiating the batch time loop failed: %s", cudaGetErrorString(ei));
    }
    b->graph_steps = n_steps;
    SW_CUDA(cudaGraphLaunch(b->graph, st));
  } else if (n_steps > 0) {
    SW_TRY(enqueue(st, false));
  }
  if (n_steps > 0) b->last_steps = n_steps;
  if (n_steps > 0 && launches == 0) {  // a replayed graph: count what it holds
    launches = int64_t(n_steps) * (1 + (b->max_src_taps > 0) + (b->max_rec > 0));
  }
  for (int i = 0; final_fields && i < n; ++i) {
    if (!final_fields[i]) continue;
    sw_grid* g = b->grids[size_t(i)];
    float* dst = final_fields[i];
    const bool fh = !is_device_pointer(dst);
    if (fh) {
      if (!g->staging) SW_TRY(dev_alloc(g, (void**)&g->staging, size_t(g->nodes()) * sizeof(float)));
      dst = g->staging;
    }
    extract_kernel<<<grid_blocks(g->nodes(), 256), 256, 0, st>>>(g->at0(g->u[n_steps & 1]), dst, g->faces());
    SW_CUDA(cudaGetLastError());
    ++launches;
    if (fh)
      SW_CUDA(cudaMemcpyAsync(final_fields[i], dst, size_t(g->nodes()) * sizeof(float), cudaMemcpyDefault, st));
  }
  SW_TRY(check_device_flag(b->grids[0]));  // synchronises
  b->kernel_launches = launches;
  b->stencil_launches = timed;
  b->stencil_ms = 0.0;
  for (int i = 0; i < timed; ++i) {
    float ms = 0.f;
    SW_CUDA(cudaEventElapsedTime(&ms, b->events[size_t(2 * i)], b->events[size_t(2 * i + 1)]));
    b->stencil_ms += ms;
  }
  return SW_OK;
}

void sw_destroy_batch(sw_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (int c = 0; c < 3; ++c) cudaFree(b->d_groups[c]);
  cudaFree(b->d_shots);
  free_batch_3d(b);
  delete b;
}

}  // extern "C"
