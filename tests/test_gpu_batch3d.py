"""GPU tests of batches of 3D grids (uneven sizes advanced by one launch per step).

A 3D batch runs the pipelined stencil over one work list of (tile, plane)
items of every grid and one launch of every grid's face conditions, receiver
samples and next step's sources; each grid must reproduce, bit for bit, the
run of its grid alone through sw_forward (the same kernels, the same
operations per node), on the direct, the captured and the replayed time
loop.  One grid is also checked against the oracle directly.
"""
import numpy as np
import pytest

import oracle
from paper_2201_05278_b300 import api
from tests.harness import assert_parity

pytestmark = pytest.mark.gpu


class Shot3:
    def __init__(self, shape, spacing, nbl, bc, vel, dt, src, recs, order=8, f_peak=30.0, n_steps=60, alpha=None):
        self.shape, self.spacing, self.nbl, self.bc, self.vel, self.dt = shape, spacing, nbl, bc, vel, dt
        self.src, self.recs, self.order, self.f_peak, self.n_steps = src, recs, order, f_peak, n_steps
        self.t0 = 1.0 / f_peak
        self.alpha = 30.0 / max(nbl) ** 3 if alpha is None else alpha

    def grid(self):
        import torch
        g = api.sw_create_grid(3, self.shape, self.spacing, self.order, self.nbl, self.bc, self.alpha, 3, self.dt)
        api.sw_set_model(g, torch.from_numpy(self.vel).cuda())
        src = np.zeros((0, 3)) if self.src is None else np.array([self.src])
        api.sw_set_acquisition(g, src, np.array(self.recs).reshape(-1, 3),
                               api.sw_ricker(self.f_peak, self.t0, self.dt, self.n_steps))
        return g


def _model(shape, seed):
    rng = np.random.default_rng(seed)
    v = np.empty(shape, np.float32)
    depths = np.sort(rng.integers(1, shape[0], size=2))
    speeds = 1500.0 + 2500.0 * rng.random(3)
    for z in range(shape[0]):
        v[z] = speeds[int(np.searchsorted(depths, z, side="right"))]
    return v * (1.0 + 0.03 * rng.standard_normal(shape)).astype(np.float32)


def _shots(spacings):
    """Five grids of uneven sizes and face conditions; spacings: one per grid."""
    geo = [
        dict(shape=(40, 37, 70), nbl=[0, 6, 5, 4, 6, 7],
             bc=["null_neumann", "null_dirichlet", "null_dirichlet", "none", "null_neumann", "null_dirichlet"]),
        dict(shape=(33, 50, 45), nbl=[4, 4, 0, 6, 5, 5],
             bc=["null_dirichlet", "null_neumann", "null_neumann", "null_dirichlet", "null_dirichlet", "none"]),
        dict(shape=(48, 48, 48), nbl=[0, 8, 8, 8, 8, 8], bc=["null_neumann"] + ["null_dirichlet"] * 5),
        dict(shape=(48, 48, 48), nbl=[0, 8, 8, 8, 8, 8], bc=["null_neumann"] + ["null_dirichlet"] * 5),
        dict(shape=(30, 61, 90), nbl=[0, 5, 6, 6, 9, 9],
             bc=["null_neumann", "null_dirichlet", "null_dirichlet", "null_dirichlet", "null_dirichlet",
                 "null_dirichlet"]),
    ]
    shots = []
    for i, (gm, h) in enumerate(zip(geo, spacings)):
        v = _model(gm["shape"], 10 + i)
        dt = 0.3 * min(h) / float(v.max())
        phys = [(gm["shape"][a] - gm["nbl"][2 * a] - gm["nbl"][2 * a + 1] - 1) * h[a] for a in range(3)]
        # the source: in the middle, or inside an absorbing layer (shallow enough that eta dt stays small)
        src = (0.35 * phys[0], 0.5 * phys[1], -1.3 * h[2]) if i == 1 else tuple(0.3 * p + 0.41 for p in phys)
        recs = [(2.0 * h[0], 0.2 * phys[1] + k * 0.15 * phys[1], 0.1 * phys[2] + k * 0.2 * phys[2]) for k in range(5)]
        shots.append(Shot3(spacing=h, vel=v, dt=dt, src=src, recs=recs if i != 2 else [], **gm))
    return shots


def _alone(shot):
    import torch
    g = shot.grid()
    try:
        assert api.sw_get_stencil_variant(g) == api.SW_STENCIL_TMA
        seis = torch.zeros((shot.n_steps, len(shot.recs)), device="cuda:0")
        fin = torch.zeros(shot.shape, device="cuda:0")
        api.sw_forward(g, shot.n_steps, seis if shot.recs else None, fin)
        return seis.cpu().numpy(), fin.cpu().numpy()
    finally:
        g.close()


@pytest.mark.parametrize("equal_spacing", [True, False])
def test_3d_batch_reproduces_single_runs(cuda_device, equal_spacing):
    import torch
    spacings = [(10.0, 10.0, 10.0)] * 5 if equal_spacing else [(10.0, 9.0, 11.0), (8.0, 9.0, 7.5), (9.0, 9.5, 10.0),
                                                                  (9.0, 9.5, 10.0), (12.0, 10.0, 11.0)]
    shots = _shots(spacings)
    alone = [_alone(s) for s in shots]
    grids = [s.grid() for s in shots]
    n = shots[0].n_steps
    b = api.sw_create_batch(grids)
    try:
        groups, items = api.sw_batch_info(b)
        assert groups == 5
        assert items == sum(((s.shape[2] + 63) // 64) * ((s.shape[1] + 15) // 16) * s.shape[0] for s in shots)
        with pytest.raises(api.SimwaveError):
            api.sw_batch_set_tile(b, 16)
        for rep in range(3):  # direct, captured, replayed
            seis = [torch.full((n, len(s.recs)), -1.0, device="cuda:0") if s.recs else None for s in shots]
            fins = [torch.zeros(s.shape, device="cuda:0") for s in shots]
            api.sw_batch_forward(b, n, seis, fins)
            for i, s in enumerate(shots):
                if s.recs:
                    assert np.array_equal(seis[i].cpu().numpy(), alone[i][0]), (rep, i)
                assert np.array_equal(fins[i].cpu().numpy(), alone[i][1]), (rep, i)
        # a shorter run, host final fields
        fins = [np.zeros(s.shape, np.float32) for s in shots]
        seis = [torch.zeros((n // 2, len(s.recs)), device="cuda:0") if s.recs else None for s in shots]
        api.sw_batch_forward(b, n // 2, seis, fins)
        assert np.array_equal(seis[0].cpu().numpy(), alone[0][0][: n // 2])
        assert np.abs(fins[4]).max() > 0
    finally:
        b.close()
        for g in grids:
            g.close()
    # the grid whose source sits in an absorbing layer, against the oracle
    s = shots[1]
    w = oracle.ricker_samples(s.f_peak, s.dt, n, t0=s.t0)
    s_ref, p_ref = oracle.forward(3, s.shape, s.spacing, s.order, s.vel.astype(np.float64), s.dt, n,
                                  src_pos=[s.src], wavelet=w, rec_pos=s.recs, nbl=s.nbl, bc=s.bc,
                                  damp_alpha=s.alpha, damp_degree=3)
    assert np.abs(s_ref).max() > 0
    assert_parity(alone[1][0], s_ref)
    assert_parity(alone[1][1], p_ref)


def test_3d_batch_with_initial_levels(cuda_device):
    import torch
    shots = _shots([(10.0, 10.0, 10.0)] * 5)[:3]
    rng = np.random.default_rng(7)
    init = rng.standard_normal(shots[0].shape).astype(np.float32)
    grids = [s.grid() for s in shots]
    try:
        api.sw_set_initial_state(grids[0], init, 0.5 * init)
        fin_alone = torch.zeros(shots[0].shape, device="cuda:0")
        seis_alone = torch.zeros((30, len(shots[0].recs)), device="cuda:0")
        api.sw_forward(grids[0], 30, seis_alone, fin_alone)
        b = api.sw_create_batch(grids)
        try:
            seis = [torch.zeros((30, len(s.recs)), device="cuda:0") if s.recs else None for s in shots]
            fins = [torch.zeros(shots[0].shape, device="cuda:0"), None, None]
            api.sw_batch_forward(b, 30, seis, fins)
            assert np.array_equal(fins[0].cpu().numpy(), fin_alone.cpu().numpy())
            assert np.array_equal(seis[0].cpu().numpy(), seis_alone.cpu().numpy())
        finally:
            b.close()
    finally:
        for g in grids:
            g.close()


def test_3d_batch_refuses_what_it_cannot_run(cuda_device):
    import torch
    shots = _shots([(10.0, 10.0, 10.0)] * 4 + [(10.0, 9.0, 11.0)])
    grids = [s.grid() for s in shots]
    try:
        with pytest.raises(api.SimwaveError, match="spacings"):  # equal spacings mixed with unequal ones
            api.sw_create_batch(grids)
        g2 = api.sw_create_grid(2, (40, 50), (10.0, 10.0), 8, [0, 5, 5, 5], ["null_neumann"] + ["null_dirichlet"] * 3,
                                0.01, 3, 1e-3)
        try:
            api.sw_set_model(g2, torch.full((40, 50), 2000.0, device="cuda:0"))
            api.sw_set_acquisition(g2, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(10, np.float32))
            with pytest.raises(api.SimwaveError, match="dimension"):
                api.sw_create_batch([grids[0], g2])
        finally:
            g2.close()
        api.sw_set_model(grids[1], torch.from_numpy(shots[1].vel).cuda(),
                         torch.full(shots[1].shape, 2000.0, device="cuda:0"))
        with pytest.raises(api.SimwaveError, match="constant-density"):
            api.sw_create_batch(grids[:2])
        api.sw_set_stencil_variant(grids[2], api.SW_STENCIL_PLAIN)
        with pytest.raises(api.SimwaveError, match="pipelined"):
            api.sw_create_batch([grids[0], grids[2]])
    finally:
        for g in grids:
            g.close()
