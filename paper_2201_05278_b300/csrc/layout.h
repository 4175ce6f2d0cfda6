// Device data layout of the wavefields and model fields.
//
// Every grid-shaped device field is stored padded: r ghost planes before and
// after the nodes along z (and y in 3D), and along x a 32-float front pad so
// that interior rows start on a 128-byte boundary.  Pointers handed to kernels
// point at node (0, 0, 0); ghost nodes sit at negative or >= n indices.
//
//   index(z, y, x) = z * sz + y * sy + x,   sy = pitch, sz = py * pitch
//   pitch = kXOff + roundup(nx, kTileXMax) + kXOff
//   py    = roundup(ny, kTileYMax) + 2 r   (3D),  1 (2D)
//   pz    = nz + 2 r
//
// Rounding the extents up to whole tiles lets the tail tiles of the stencil
// read (and ignore) lanes past the last node without leaving the allocation.
#pragma once

#include <cstdint>

namespace sw {

constexpr int kXOff = 32;       // front pad along x (>= max radius, 128-byte aligned)
constexpr int kTileXMax = 128;  // widest x tile of any stencil kernel
constexpr int kTileYMax = 32;   // tallest y tile of any stencil kernel
constexpr int kMaxR = 10;

enum { kBcNone = 0, kBcDirichlet = 1, kBcNeumann = 2 };

struct Layout {
  int ndim;
  int r;
  int64_t n[3];  // nz, ny (1 in 2D), nx
  int64_t pitch, py, pz;
  int64_t sy, sz;
  int64_t origin;  // offset of node (0,0,0) from the allocation start
  int64_t total;   // elements per padded field

  void init(int ndim_, int r_, const int64_t* n3) {
    ndim = ndim_;
    r = r_;
    for (int a = 0; a < 3; ++a) n[a] = n3[a];
    pitch = kXOff + ((n[2] + kTileXMax - 1) / kTileXMax) * kTileXMax + kXOff;
    py = (ndim == 3) ? ((n[1] + kTileYMax - 1) / kTileYMax) * kTileYMax + 2 * r : 1;
    pz = n[0] + 2 * r;
    sy = pitch;
    sz = py * pitch;
    origin = int64_t(r) * sz + ((ndim == 3) ? int64_t(r) * sy : 0) + kXOff;
    total = pz * sz;
  }
};

}  // namespace sw
