"""Seeded synthetic workloads (inputs only).

This module generates the inputs that both the CUDA library and the CPU
oracle consume: grid shapes, spacings, boundary set-up, velocity/density
models, time step, source/receiver positions and the wavelet's parameters.
It holds none of the solver's arithmetic (no FD weights, stability bound,
damping profile or window weights) and imports neither the library nor the
oracle.

The paper's benchmark models (Marmousi2, Overthrust; Sec. 4-5) are not
available, so synthetic layered models of the same kind stand in for them:

  2d_homogeneous_256   256 x 256, h = 10 m, v = 1500 m/s, order 8, 1000 steps,
                       10 Hz Ricker at the grid centre, 20-cell layer on the
                       bottom/left/right faces, 64 receivers at 20 m depth
  3d_layered_256       256^3, h = 10 m, order 8, 8 flat layers 1500-4500 m/s
                       times (1 + 0.05 G), G Gaussian-smoothed white noise
                       (sigma 3 cells, seed 2201, unit std), 2000 steps, 15 Hz
                       Ricker 5 cells deep, 40-cell layer on five faces,
                       64 x 64 receivers 2 cells deep
  3d_vd_512x512x384    (384, 512, 512), h = 12.5 m, order 16, the layered
                       model plus two dipping interfaces (+500 m/s each),
                       Gardner density rho = 310 v^0.25, 3000 steps, 10 Hz,
                       50-cell layer, 128 x 128 receivers at the surface
  2d_layered_4096      4096 x 4096, h = 5 m, order 8, the layered model of
                       3d_layered_256 in 2D (8 layers, smoothed 5% noise),
                       1000 steps, 15 Hz Ricker 5 cells deep, 40-cell layer,
                       256 receivers 2 cells deep: a 2D grid whose fields
                       (67 MB each) do not stay in L2, for the two-step
                       kernel against the per-step kernels

  2d_shot_batch_64     64 shots for batched runs: 8 models (seeds 0..7) of
                       (nz, nx) drawn from U{300..800} x U{400..1200}, h = 10 m,
                       3-8 flat layers at random depths with random speeds in
                       1500-4500 m/s; 8 shots per model with sources 2 cells
                       deep spread evenly along the surface; 256 receivers per
                       shot 2 cells deep across the surface; order 8, 10 Hz,
                       40-cell layer, 2000 steps (shot_batch())

  3d_fwi_gradient_256  misfit-gradient workload: 256^3, background 2500 m/s,
                       true model with a +10% Gaussian anomaly (sigma 25
                       cells), 16 shots on a 4 x 4 surface grid, 1500 steps,
                       10 Hz, BF16 checkpoints every 10 steps
                       (fwi_gradient_256())

Every model has no absorbing layer on the top face, which is null Neumann
(as in the paper's listings); the other faces are null Dirichlet behind the
layer.  dt = 0.4 h / c_max (Courant number 0.4).  The damping alpha follows a
standard estimate for a p = 3 profile with 1e-3 reflection:
eta_max = (p + 1) c_max ln(1000) / (2 L), alpha = eta_max / nbl^p, L the layer
width in metres.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class Workload:
    name: str
    ndim: int
    shape: Tuple[int, ...]
    spacing: Tuple[float, ...]
    order: int
    nbl: List[int]
    bc: List[str]
    damp_alpha: float
    damp_degree: int
    dt: float
    n_steps: int
    f_peak: float
    t0: float
    src_pos: np.ndarray
    rec_pos: np.ndarray
    window_radius: int
    velocity: np.ndarray
    density: Optional[np.ndarray] = None
    notes: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return int(np.prod(self.shape))

    @property
    def updates(self) -> int:
        """Grid-point updates of one forward run (all nodes, absorbing layer included)."""
        return self.nodes * self.n_steps


def _alpha(c_max: float, nbl: int, h: float, p: int = 3, refl: float = 1e-3) -> float:
    if nbl == 0:
        return 0.0
    eta_max = (p + 1) * c_max * math.log(1.0 / refl) / (2.0 * nbl * h)
    return eta_max / nbl ** p


def _smooth_noise(shape, sigma, seed):
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(shape).astype(np.float32)
    g = gaussian_filter(g, sigma=sigma, mode="reflect")
    g -= g.mean()
    g /= g.std()
    return g


def layered_velocity(shape, n_layers=8, vmin=1500.0, vmax=4500.0, noise=0.05, sigma=3.0, seed=2201,
                     dips=None, spacing=None):
    """Flat layers (depth index k * nz / n_layers) with a smooth multiplicative perturbation.

    dips: optional list of (dip_degrees, depth_fraction, jump_m_s) planar interfaces
    dipping along x; below each interface the velocity increases by `jump`.
    """
    nz = shape[0]
    z = np.arange(nz)
    layer = np.minimum((z * n_layers) // nz, n_layers - 1)
    v1 = (vmin + layer * (vmax - vmin) / (n_layers - 1)).astype(np.float32)
    v = np.broadcast_to(v1.reshape((nz,) + (1,) * (len(shape) - 1)), shape).astype(np.float32)
    if dips:
        nx = shape[-1]
        hz, hx = spacing[0], spacing[-1]
        zz = (np.arange(nz) * hz).reshape((nz,) + (1,) * (len(shape) - 1))
        xx = (np.arange(nx) * hx).reshape((1,) * (len(shape) - 1) + (nx,))
        for dip, frac, jump in dips:
            z_if = frac * nz * hz + math.tan(math.radians(dip)) * (xx - 0.5 * nx * hx)
            v = v + np.float32(jump) * (zz > z_if).astype(np.float32)
    if noise:
        v = v * (1.0 + np.float32(noise) * _smooth_noise(shape, sigma, seed))
    return np.ascontiguousarray(v, dtype=np.float32)


def _grid_positions(lo, hi, n):
    return np.linspace(lo, hi, n)


def make(name: str, n_steps: Optional[int] = None, shape: Optional[Tuple[int, ...]] = None,
         seed: int = 2201) -> Workload:
    """Workload by name; n_steps / shape override the defaults (shape keeps the recipe)."""
    if name == "2d_homogeneous_256":
        shp = tuple(shape) if shape else (256, 256)
        h = (10.0, 10.0)
        nb = 20
        nbl = [0, nb, nb, nb]
        vel = np.full(shp, 1500.0, dtype=np.float32)
        c_max = 1500.0
        dt = 0.4 * h[0] / c_max
        f = 10.0
        phys_x = (shp[1] - 2 * nb - 1) * h[1]
        src = np.array([[(shp[0] // 2) * h[0], (shp[1] // 2 - nb) * h[1]]])
        rec = np.stack([np.full(64, 20.0), _grid_positions(0.05 * phys_x, 0.95 * phys_x, 64)], 1)
        return Workload(name, 2, shp, h, 8, nbl, ["null_neumann", "null_dirichlet", "null_dirichlet",
                                                   "null_dirichlet"],
                        _alpha(c_max, nb, h[0]), 3, dt, n_steps or 1000, f, 1.0 / f, src, rec, 4, vel)
    if name == "3d_layered_256":
        shp = tuple(shape) if shape else (256, 256, 256)
        h = (10.0, 10.0, 10.0)
        nb = min(40, max(4, shp[1] // 6))
        nbl = [0, nb, nb, nb, nb, nb]
        vel = layered_velocity(shp, seed=seed)
        c_max = float(vel.max())
        dt = 0.4 * h[0] / c_max
        f = 15.0
        py = (shp[1] - 2 * nb - 1) * h[1]
        px = (shp[2] - 2 * nb - 1) * h[2]
        src = np.array([[5 * h[0], 0.5 * py, 0.5 * px]])
        ny_r = nx_r = 64 if shp[1] >= 128 else 8
        yy, xx = np.meshgrid(_grid_positions(0.0, py, ny_r), _grid_positions(0.0, px, nx_r), indexing="ij")
        rec = np.stack([np.full(yy.size, 2 * h[0]), yy.ravel(), xx.ravel()], 1)
        return Workload(name, 3, shp, h, 8, nbl, ["null_neumann"] + ["null_dirichlet"] * 5,
                        _alpha(c_max, nb, h[0]), 3, dt, n_steps or 2000, f, 1.0 / f, src, rec, 4, vel)
    if name == "3d_vd_512x512x384":
        shp = tuple(shape) if shape else (384, 512, 512)
        h = (12.5, 12.5, 12.5)
        nb = min(50, max(8, shp[1] // 6))
        nbl = [0, nb, nb, nb, nb, nb]
        vel = layered_velocity(shp, seed=seed, dips=[(10.0, 0.35, 500.0), (-15.0, 0.65, 500.0)], spacing=h)
        rho = (310.0 * vel.astype(np.float64) ** 0.25).astype(np.float32)
        c_max = float(vel.max())
        dt = 0.4 * h[0] / c_max
        f = 10.0
        py = (shp[1] - 2 * nb - 1) * h[1]
        px = (shp[2] - 2 * nb - 1) * h[2]
        src = np.array([[5 * h[0], 0.5 * py, 0.5 * px]])
        ny_r = nx_r = 128 if shp[1] >= 256 else 8
        yy, xx = np.meshgrid(_grid_positions(0.0, py, ny_r), _grid_positions(0.0, px, nx_r), indexing="ij")
        rec = np.stack([np.zeros(yy.size), yy.ravel(), xx.ravel()], 1)
        return Workload(name, 3, shp, h, 16, nbl, ["null_neumann"] + ["null_dirichlet"] * 5,
                        _alpha(c_max, nb, h[0]), 3, dt, n_steps or 3000, f, 1.0 / f, src, rec, 4, vel, rho)
    if name == "2d_layered_4096":
        shp = tuple(shape) if shape else (4096, 4096)
        h = (5.0, 5.0)
        nb = min(40, max(4, shp[1] // 6))
        nbl = [0, nb, nb, nb]
        vel = layered_velocity(shp, seed=seed)
        c_max = float(vel.max())
        dt = 0.4 * h[0] / c_max
        f = 15.0
        phys_x = (shp[1] - 2 * nb - 1) * h[1]
        src = np.array([[5 * h[0], 0.5 * phys_x]])
        rec = np.stack([np.full(256, 2 * h[0]), _grid_positions(0.0, phys_x, 256)], 1)
        return Workload(name, 2, shp, h, 8, nbl, ["null_neumann", "null_dirichlet", "null_dirichlet",
                                                   "null_dirichlet"],
                        _alpha(c_max, nb, h[0]), 3, dt, n_steps or 1000, f, 1.0 / f, src, rec, 4, vel)
    raise KeyError(name)


def shot_batch(n_models: int = 8, shots_per_model: int = 8, n_steps: Optional[int] = None,
               size_scale: float = 1.0) -> List[Workload]:
    """The shots of 2d_shot_batch_64 (model after model); size_scale shrinks the
    grids for quick tests.  Shots of one model share its velocity array and dt."""
    out = []
    h = (10.0, 10.0)
    nb = 40
    f = 10.0
    for m in range(n_models):
        rng = np.random.default_rng(m)
        nz = max(2 * nb + 20, int(round(int(rng.integers(300, 801)) * size_scale)))
        nx = max(2 * nb + 40, int(round(int(rng.integers(400, 1201)) * size_scale)))
        n_layers = int(rng.integers(3, 9))
        depths = np.sort(rng.choice(np.arange(1, nz), size=n_layers - 1, replace=False))
        speeds = 1500.0 + 3000.0 * rng.random(n_layers)
        v1 = speeds[np.searchsorted(depths, np.arange(nz), side="right")].astype(np.float32)
        vel = np.ascontiguousarray(np.broadcast_to(v1[:, None], (nz, nx)), dtype=np.float32)
        c_max = float(vel.max())
        dt = 0.4 * h[0] / c_max
        phys_x = (nx - 2 * nb - 1) * h[1]
        rec = np.stack([np.full(256, 2 * h[0]), _grid_positions(0.02 * phys_x, 0.98 * phys_x, 256)], 1)
        for k in range(shots_per_model):
            src = np.array([[2 * h[0], (k + 0.5) / shots_per_model * phys_x]])
            out.append(Workload("2d_shot_batch_64/model%d/shot%d" % (m, k), 2, (nz, nx), h, 8, [0, nb, nb, nb],
                                ["null_neumann", "null_dirichlet", "null_dirichlet", "null_dirichlet"],
                                _alpha(c_max, nb, h[0]), 3, dt, n_steps or 2000, f, 1.0 / f, src, rec, 4, vel))
    return out


def shot_batch_3d(n_models: int = 8, shots_per_model: int = 2, n_steps: Optional[int] = None,
                  size_scale: float = 1.0) -> List[Workload]:
    """The shots of 3d_shot_batch_16: 3D grids too small to fill the GPU
    alone, advanced together.  8 layered models (seeds 100..107, 3-6 flat
    layers of 1500-4500 m/s) whose (nz, ny, nx) are drawn from U{48..96} each,
    h = 10 m, order 8, 12-cell absorbing layer on five faces (top null
    Neumann), 2 shots per model 2 cells deep, 8 x 8 receivers 2 cells deep,
    15 Hz Ricker, 1000 steps."""
    out = []
    h = (10.0, 10.0, 10.0)
    nb = 12
    f = 15.0
    for m in range(n_models):
        rng = np.random.default_rng(100 + m)
        shp = tuple(max(2 * nb + 12, int(round(int(rng.integers(48, 97)) * size_scale))) for _ in range(3))
        n_layers = int(rng.integers(3, 7))
        depths = np.sort(rng.choice(np.arange(1, shp[0]), size=n_layers - 1, replace=False))
        speeds = 1500.0 + 3000.0 * rng.random(n_layers)
        v1 = speeds[np.searchsorted(depths, np.arange(shp[0]), side="right")].astype(np.float32)
        vel = np.ascontiguousarray(np.broadcast_to(v1[:, None, None], shp), dtype=np.float32)
        c_max = float(vel.max())
        dt = 0.4 * h[0] / c_max
        py = (shp[1] - 2 * nb - 1) * h[1]
        px = (shp[2] - 2 * nb - 1) * h[2]
        ry, rx = np.meshgrid(_grid_positions(0.05 * py, 0.95 * py, 8), _grid_positions(0.05 * px, 0.95 * px, 8),
                             indexing="ij")
        rec = np.stack([np.full(ry.size, 2 * h[0]), ry.ravel(), rx.ravel()], 1)
        for k in range(shots_per_model):
            src = np.array([[2 * h[0], 0.5 * py, (k + 0.5) / shots_per_model * px]])
            out.append(Workload("3d_shot_batch_16/model%d/shot%d" % (m, k), 3, shp, h, 8, [0, nb, nb, nb, nb, nb],
                                ["null_neumann"] + ["null_dirichlet"] * 5, _alpha(c_max, nb, h[0]), 3, dt,
                                n_steps or 1000, f, 1.0 / f, src, rec, 4, vel))
    return out


def batch_shots(name: str, n_steps: Optional[int] = None) -> List[Workload]:
    """The shots of a batched workload by name."""
    return shot_batch(n_steps=n_steps) if name == "2d_shot_batch_64" else shot_batch_3d(n_steps=n_steps)


@dataclass
class GradientCase:
    """A misfit-gradient workload: true and initial models, one source per shot."""
    base: Workload          # grid, initial (background) model, receivers, wavelet parameters
    v_true: np.ndarray
    shots: np.ndarray       # [n_shots][3] source positions
    checkpoint_every: int


def fwi_gradient_256(n_steps: Optional[int] = None, shape: Optional[Tuple[int, ...]] = None) -> GradientCase:
    """3d_fwi_gradient_256: 256^3, h = 10 m, background 2500 m/s, true model
    with a centred Gaussian anomaly of +10% (sigma 25 cells), constant
    density; 16 shots on a 4 x 4 grid 2 cells deep, 64 x 64 receivers 2 cells
    deep; order 8, 10 Hz Ricker, 1500 steps, checkpoints every 10 steps;
    40-cell absorbing layer, top face null Neumann."""
    shp = tuple(shape) if shape else (256, 256, 256)
    h = (10.0, 10.0, 10.0)
    nb = min(40, max(4, shp[1] // 6))
    nbl = [0, nb, nb, nb, nb, nb]
    v0 = 2500.0
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=np.float64) - (n - 1) / 2.0 for n in shp], indexing="ij")
    bump = np.exp(-(zz ** 2 + yy ** 2 + xx ** 2) / (2.0 * 25.0 ** 2))
    v_true = (v0 * (1.0 + 0.1 * bump)).astype(np.float32)
    v_init = np.full(shp, v0, dtype=np.float32)
    c_max = float(v_true.max())
    dt = 0.4 * h[0] / c_max
    f = 10.0
    py = (shp[1] - 2 * nb - 1) * h[1]
    px = (shp[2] - 2 * nb - 1) * h[2]
    sy, sx = np.meshgrid(_grid_positions(0.125 * py, 0.875 * py, 4), _grid_positions(0.125 * px, 0.875 * px, 4),
                         indexing="ij")
    shots = np.stack([np.full(16, 2 * h[0]), sy.ravel(), sx.ravel()], 1)
    ny_r = nx_r = 64 if shp[1] >= 128 else 8
    ry, rx = np.meshgrid(_grid_positions(0.0, py, ny_r), _grid_positions(0.0, px, nx_r), indexing="ij")
    rec = np.stack([np.full(ry.size, 2 * h[0]), ry.ravel(), rx.ravel()], 1)
    base = Workload("3d_fwi_gradient_256", 3, shp, h, 8, nbl, ["null_neumann"] + ["null_dirichlet"] * 5,
                    _alpha(c_max, nb, h[0]), 3, dt, n_steps or 1500, f, 1.0 / f, shots[:1], rec, 4, v_init)
    return GradientCase(base, v_true, shots, 10)


NAMES = ["2d_homogeneous_256", "3d_layered_256", "3d_vd_512x512x384", "2d_layered_4096"]
GRADIENT_NAMES = ["3d_fwi_gradient_256"]
BATCH_NAMES = ["2d_shot_batch_64", "3d_shot_batch_16"]
