"""GPU tests of batched shots (2D grids of uneven sizes advanced together).

Every shot of a batch must reproduce, bit for bit, the run of its grid alone
(the batched stencil uses the same arithmetic sequence as the single-grid 2D
kernel), whatever the grouping into shared models, the ragged tiles or the
order of the grids; one shot is also checked against the oracle directly.
"""
import numpy as np
import pytest

import oracle
from paper_2201_05278_b300 import api
from tests.harness import FP32_SEIS_TOL, assert_parity, rel_l2

pytestmark = pytest.mark.gpu


class Shot:
    def __init__(self, shape, spacing, nbl, bc, vel, dt, src, recs, order=8, f_peak=25.0, n_steps=70):
        self.shape, self.spacing, self.nbl, self.bc, self.vel, self.dt = shape, spacing, nbl, bc, vel, dt
        self.src, self.recs, self.order, self.f_peak, self.n_steps = src, recs, order, f_peak, n_steps
        self.t0 = 1.0 / f_peak

    def grid(self):
        import torch
        g = api.sw_create_grid(2, self.shape, self.spacing, self.order, self.nbl, self.bc, 30.0 / max(self.nbl) ** 3,
                               3, self.dt)
        api.sw_set_model(g, torch.from_numpy(self.vel).cuda())
        src = np.zeros((0, 2)) if self.src is None else np.array([self.src])
        api.sw_set_acquisition(g, src, np.array(self.recs).reshape(-1, 2),
                               api.sw_ricker(self.f_peak, self.t0, self.dt, self.n_steps))
        return g


def _layered(shape, seed):
    rng = np.random.default_rng(seed)
    v = np.empty(shape, np.float32)
    depths = np.sort(rng.integers(1, shape[0], size=3))
    speeds = 1500.0 + 3000.0 * rng.random(4)
    for z in range(shape[0]):
        v[z] = speeds[int(np.searchsorted(depths, z, side="right"))]
    return v


def _shots():
    m1 = dict(shape=(97, 203), spacing=(10.0, 12.0), nbl=[0, 12, 10, 14],
              bc=["null_neumann", "null_dirichlet", "null_dirichlet", "none"])
    m2 = dict(shape=(130, 77), spacing=(8.0, 8.0), nbl=[6, 9, 7, 5],
              bc=["null_dirichlet", "null_neumann", "null_neumann", "null_dirichlet"])
    m3 = dict(shape=(41, 300), spacing=(9.0, 7.0), nbl=[0, 8, 8, 8],
              bc=["null_neumann", "none", "null_dirichlet", "null_dirichlet"])
    v1, v2, v3 = _layered(m1["shape"], 1), _layered(m2["shape"], 2), _layered(m3["shape"], 3)
    v4 = v1.copy()
    v4[40:60] *= 1.05  # same geometry as model 1, another model
    dt1 = 0.35 * 10.0 / float(max(v1.max(), v4.max()))
    dt2 = 0.35 * 8.0 / float(v2.max())
    dt3 = 0.35 * 7.0 / float(v3.max())
    rec1 = [(20.0, x) for x in np.linspace(30.0, 2000.0, 17)]
    rec2 = [(z, 100.0) for z in np.linspace(50.0, 700.0, 9)]
    a = [Shot(vel=v1, dt=dt1, src=(40.0, sx), recs=rec1, **m1) for sx in (205.0, 1003.7, 1800.0)]
    b = [Shot(vel=v2, dt=dt2, src=(sz, 250.3), recs=rec2, **m2) for sz in (80.0, 400.0)]
    c = Shot(vel=v3, dt=dt3, src=(100.0, 1000.0), recs=[], **m3)
    d = Shot(vel=v4, dt=dt1, src=(40.0, 605.0), recs=rec1, **m1)
    # interleaved, so the shot table's order differs from the grids' order
    return [a[0], b[0], c, a[1], d, b[1], a[2]]


def _alone(shot):
    import torch
    g = shot.grid()
    try:
        seis = torch.zeros((shot.n_steps, len(shot.recs)), device="cuda:0")
        fin = torch.zeros(shot.shape, device="cuda:0")
        api.sw_forward(g, shot.n_steps, seis if shot.recs else None, fin)
        return seis.cpu().numpy(), fin.cpu().numpy()
    finally:
        g.close()


def test_batch_reproduces_single_runs(cuda_device):
    import torch
    shots = _shots()
    alone = [_alone(s) for s in shots]
    grids = [s.grid() for s in shots]
    n = shots[0].n_steps
    b = api.sw_create_batch(grids)
    try:
        assert api.sw_batch_info(b)[0] == 4  # models 1, 2, 3 and the perturbed copy of 1
        rows, us = api.sw_batch_get_tile(b)
        assert rows in (16, 32, 64) and all(t > 0 for t in us) and us[(16, 32, 64).index(rows)] == min(us)
        # the tuned tile: direct, captured, replayed; then every tile height directly
        for rep, tile in enumerate((rows, rows, rows, 16, 32, 64)):
            api.sw_batch_set_tile(b, tile)
            seis = [torch.full((n, len(s.recs)), -1.0, device="cuda:0") if s.recs else None for s in shots]
            fins = [torch.zeros(s.shape, device="cuda:0") for s in shots]
            api.sw_batch_forward(b, n, seis, fins)
            for i, s in enumerate(shots):
                if s.recs:
                    assert np.array_equal(seis[i].cpu().numpy(), alone[i][0]), (rep, i)
                assert np.array_equal(fins[i].cpu().numpy(), alone[i][1]), (rep, i)
        with pytest.raises(api.SimwaveError):
            api.sw_batch_set_tile(b, 48)
        # a shorter run and host final fields
        fins = [np.zeros(s.shape, np.float32) for s in shots]
        seis = [torch.zeros((n // 2, len(s.recs)), device="cuda:0") if s.recs else None for s in shots]
        api.sw_batch_forward(b, n // 2, seis, fins)
        assert np.array_equal(seis[0].cpu().numpy(), alone[0][0][: n // 2])
    finally:
        b.close()
        for g in grids:
            g.close()
    s = shots[3]
    w = oracle.ricker_samples(s.f_peak, s.dt, n, t0=s.t0)
    s_ref, p_ref = oracle.forward(2, s.shape, s.spacing, s.order, s.vel.astype(np.float64), s.dt, n,
                                  src_pos=[s.src], wavelet=w, rec_pos=s.recs, nbl=s.nbl, bc=s.bc,
                                  damp_alpha=30.0 / max(s.nbl) ** 3, damp_degree=3)
    assert_parity(alone[3][0], s_ref)
    assert_parity(alone[3][1], p_ref)


def test_batch_with_initial_levels(cuda_device):
    import torch
    shots = _shots()[:3]
    rng = np.random.default_rng(5)
    init = rng.standard_normal(shots[2].shape).astype(np.float32)
    grids = [s.grid() for s in shots]
    try:
        api.sw_set_initial_state(grids[2], init, init)
        fin_alone = torch.zeros(shots[2].shape, device="cuda:0")
        api.sw_forward(grids[2], 30, None, fin_alone)
        b = api.sw_create_batch(grids)
        try:
            seis = [torch.zeros((30, len(s.recs)), device="cuda:0") if s.recs else None for s in shots]
            fins = [None, None, torch.zeros(shots[2].shape, device="cuda:0")]
            api.sw_batch_forward(b, 30, seis, fins)
            assert np.array_equal(fins[2].cpu().numpy(), fin_alone.cpu().numpy())
        finally:
            b.close()
    finally:
        for g in grids:
            g.close()


def test_batch_errors(cuda_device):
    import torch
    shots = _shots()
    g0, g1 = shots[0].grid(), shots[1].grid()
    g3d = api.sw_create_grid(3, (20, 20, 20), (10.0, 10.0, 10.0), 8, [0] * 6, ["null_dirichlet"] * 6, 0.0, 3, 1e-3)
    api.sw_set_model(g3d, torch.full((20, 20, 20), 1500.0, device="cuda:0"))
    api.sw_set_acquisition(g3d, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(1, np.float32))
    s4 = shots[1]
    s4.order = 4
    g4 = s4.grid()
    try:
        for bad in ([g0, g3d], [g0, g0], [g0, g4]):
            with pytest.raises(api.SimwaveError):
                api.sw_create_batch(bad)
        b = api.sw_create_batch([g0, g1])
        try:
            seis = [torch.zeros((10, len(s.recs)), device="cuda:0") for s in shots[:2]]
            with pytest.raises(api.SimwaveError):  # host seismograms are refused
                api.sw_batch_forward(b, 10, [np.zeros((10, len(shots[0].recs)), np.float32), seis[1]])
            long_seis = [torch.zeros((shots[0].n_steps + 1, len(s.recs)), device="cuda:0") for s in shots[:2]]
            with pytest.raises(api.SimwaveError):  # longer than the wavelets
                api.sw_batch_forward(b, shots[0].n_steps + 1, long_seis)
            api.sw_batch_forward(b, 10, seis)
            api.sw_set_acquisition(g1, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(1, np.float32))
            with pytest.raises(api.SimwaveError):  # a grid changed after the batch was made
                api.sw_batch_forward(b, 10, seis)
        finally:
            b.close()
    finally:
        for g in (g0, g1, g3d, g4):
            g.close()


@pytest.mark.parametrize("order", [2, 6, 10, 16, 20])
def test_batch_all_radii(cuda_device, order):
    """Every space order's batched kernel reproduces the single-grid runs."""
    import torch
    m = dict(shape=(61 + order, 150), spacing=(9.0, 8.0), nbl=[0, 10, 9, 11],
             bc=["null_neumann", "null_dirichlet", "null_neumann", "none"])
    v = _layered(m["shape"], order)
    dt = 0.3 * 8.0 / float(v.max())
    rec = [(27.0, x) for x in np.linspace(40.0, 900.0, 7)]
    shots = [Shot(vel=v, dt=dt, src=(45.0, sx), recs=rec, order=order, n_steps=40, **m) for sx in (200.0, 611.0)]
    m2 = dict(shape=(40, 263), spacing=(8.0, 8.0), nbl=[5, 5, 5, 5], bc=["null_dirichlet"] * 4)
    v2 = _layered(m2["shape"], 100 + order)
    shots.append(Shot(vel=v2, dt=0.3 * 8.0 / float(v2.max()), src=(150.0, 700.0), recs=[(100.0, 500.0)],
                      order=order, n_steps=40, **m2))
    alone = [_alone(s) for s in shots]
    grids = [s.grid() for s in shots]
    b = api.sw_create_batch(grids)
    try:
        assert api.sw_batch_info(b)[0] == 2
        for rows in (16, 32, 64):
            api.sw_batch_set_tile(b, rows)
            seis = [torch.zeros((40, len(s.recs)), device="cuda:0") for s in shots]
            fins = [torch.zeros(s.shape, device="cuda:0") for s in shots]
            api.sw_batch_forward(b, 40, seis, fins)
            for i in range(len(shots)):
                assert np.array_equal(seis[i].cpu().numpy(), alone[i][0])
                assert np.array_equal(fins[i].cpu().numpy(), alone[i][1])
    finally:
        b.close()
        for g in grids:
            g.close()
