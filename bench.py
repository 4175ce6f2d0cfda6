"""Throughput benchmark of the forward solver (grid-point updates per second).

One bench step = one complete forward simulation of the workload (every
time step of the leapfrog loop with source injection and receiver sampling),
inputs resident in HBM.  Default workload: 3d_vd_512x512x384 (384 x 512 x 512
nodes, order 16, variable density, 3000 time steps, 16384 receivers), the
largest single-GPU configuration; Gpts/s counts every computed node
including the absorbing layer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

Under torchrun each rank runs its own independent simulation (replicas of
the same workload, weak scaling); rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpts/s (grid-point updates per second)"
UNIT = "Gpts/s"
BYTES_PER_UPDATE = {False: 16, True: 20}  # algorithmic bytes per node update (constant / variable density)
PROFILE_EVERY = 15  # CUDA events around every 15th stencil launch (odd: both buffer parities): a sample, so that the events do not slow the run


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_seconds(local_seconds, world, device=None):
    """Wall time of the whole job: the slowest rank's (all ranks run their own
    replica and finish when the last one does).  Needs an initialised process
    group when world > 1 (NCCL on the GPUs, gloo in the CPU tests)."""
    if world == 1:
        return float(local_seconds)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(updates_per_replica, replicas_per_rank, world, seconds):
    """Whole-job Gpts/s: every rank's updates over the job's wall time."""
    return updates_per_replica * replicas_per_rank * world / seconds / 1e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


STENCIL_SOURCES = ("stencil_plain.cuh", "stencil_tma.cuh", "tma.cuh", "layout.h")
BATCH_SOURCES = ("batch.cuh", "stencil_plain.cuh", "layout.h")
TB2_SOURCES = ("tb2d.cuh", "stencil_plain.cuh", "tma.cuh", "layout.h")
# committed ncu traffic record of each workload's dominant kernel (profiles/)
TRAFFIC_FILES = {
    "3d_layered_256": ("traffic_stencil_tma_3d_layered_256.txt", STENCIL_SOURCES),
    "3d_vd_512x512x384": ("traffic_stencil_tma_vd_3d_vd_512x512x384.txt", STENCIL_SOURCES),
    "2d_shot_batch_64": ("traffic_stencil_batch_2d_shot_batch_64.txt", BATCH_SOURCES),
    "2d_layered_4096": ("traffic_tb2_2d_2d_layered_4096.txt", TB2_SOURCES),
}


def _kernel_source_hash(names=STENCIL_SOURCES):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2201_05278_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_record(workload):
    """DRAM bytes of one launch of the workload's dominant kernel from the
    committed ncu record (a warm capture: earlier launches' dirty lines are
    written back inside it, as in the timed run), if the kernel sources still
    match; None otherwise.  Returns {"total", "read", "write"}."""
    if workload not in TRAFFIC_FILES:
        return None
    fname, names = TRAFFIC_FILES[workload]
    try:
        rec = {}
        with open(os.path.join(ROOT, "profiles", fname)) as f:
            for ln in f:
                if ":" in ln and not ln.startswith("#"):
                    k, v = ln.split(":", 1)
                    rec[k.strip()] = v.strip()
        if rec.get("workload") != workload or rec.get("source_sha") != _kernel_source_hash(names):
            return None
        rd, wr = float(rec["dram_bytes_read"]), float(rec["dram_bytes_write"])
        return {"total": rd + wr, "read": rd, "write": wr, "capture": rec.get("capture", "")}
    except Exception:
        return None


def _roofline_traffic(roof, workload, shape=""):
    """Fills roofline["traffic"] (bytes per launch) and its read/write split;
    None when the run's grid is not the workload's own (--shape): the
    records are captures of the full-size grid."""
    t = None if shape else _traffic_record(workload)
    roof["traffic"] = None if t is None else t["total"]
    if t is not None:
        roof["traffic_read"] = t["read"]
        roof["traffic_write"] = t["write"]
        roof["traffic_vs_algorithmic"] = round(t["total"] / roof["algorithmic_bytes_per_launch"], 4)
        roof["traffic_capture"] = t["capture"]
    return roof


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        """Starts sampling every 50 ms and returns once the first sample is in
        (at most 3 s), so that short timed regions still get samples."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class OracleRunner:
    """The FP64 oracle's forward loop on a workload, set up once: FD weights,
    damping profile, ln(rho) and window weights are prepared before any timing
    (oracle.forward would redo them on every call); run(k) times one call of
    the leapfrog loop for k time steps, its per-call padding and copies
    included.  A shot batch is timed on its first shot (the oracle runs one
    shot at a time)."""

    def __init__(self, workload_name):
        from paper_2201_05278_b300 import workloads
        import oracle
        self.oracle = oracle
        self.threads = os.cpu_count() or 1
        w = workloads.batch_shots(workload_name)[0] if workload_name in workloads.BATCH_NAMES else workloads.make(workload_name)
        self.w = w
        nbl_lo = [w.nbl[2 * a] for a in range(w.ndim)]
        self.eta = oracle.eta_field(w.shape, w.nbl, w.damp_alpha, w.damp_degree)
        self.lnrho = None if w.density is None else np.log(w.density.astype(np.float64))
        b = oracle.KAISER_B[w.window_radius]
        self.src = oracle.point_windows([tuple(p) for p in w.src_pos], w.ndim, w.spacing, nbl_lo, w.window_radius, b,
                                        w.shape)
        self.rec = oracle.point_windows([tuple(p) for p in w.rec_pos], w.ndim, w.spacing, nbl_lo, w.window_radius, b,
                                        w.shape)
        bc = [{"none": 0, "null_dirichlet": 1, "null_neumann": 2}[x] for x in w.bc]
        self.bc6 = bc if w.ndim == 3 else [bc[0], bc[1], 0, 0, bc[2], bc[3]]
        self.vel = w.velocity.astype(np.float64)
        self.nodes = w.nodes

    def run(self, steps):
        w = self.w
        wav = self.oracle.ricker_samples(w.f_peak, w.dt, max(steps, 1), t0=w.t0)
        t = time.perf_counter()
        self.oracle.run_raw(w.ndim, w.shape, w.spacing, w.order, self.bc6, self.eta, w.dt, self.vel, self.lnrho,
                            self.src, wav, self.rec, steps, threads=self.threads)
        return time.perf_counter() - t

    def steps_for(self, budget_s):
        """Time steps of one call that take about budget_s (calibrated on 1 and 2 steps)."""
        t1 = self.run(1)
        t2 = self.run(2)
        per_step = max(t2 - t1, 1e-4)
        setup = max(t1 - per_step, 0.0)
        return int(max(1, min(400, (budget_s - setup) / per_step)))

    def describe(self, steps):
        w = self.w
        return "%s full grid %s, %d of %d time steps per call, FP64, %d threads (set-up of weights, damping " \
               "and windows once, outside the timing)" % (w.name, "x".join(map(str, w.shape)), steps, w.n_steps,
                                                          self.threads)


L2_BYTES = 126e6  # B300 L2


def _l2_note(step_bytes):
    """How the per-time-step data compare with the L2 (the timing rule: inputs
    larger than L2, or say so)."""
    if step_bytes > L2_BYTES:
        return "inputs larger than L2 (each time step streams %.0f MB)" % (step_bytes / 1e6)
    return ("each time step touches %.0f MB, less than the 126 MB L2: the levels stay partly in L2 from one time "
            "step to the next, as in any run of this workload (no flush)" % (step_bytes / 1e6))


def cpu_baseline(workload_name, budget_s=12.0):
    """Times the FP64 oracle on the host cores on a bounded sample of the workload."""
    r = OracleRunner(workload_name)
    steps = r.steps_for(budget_s)
    t = r.run(steps)
    return {"value": round(r.nodes * steps / t / 1e9, 4), "unit": UNIT, "cores": r.threads, "kind": "oracle",
            "sample": r.describe(steps)}, t


def run_batch(args, world, rank, local, dev):
    """A shot batch: every shot of 2d_shot_batch_64 (or of 3d_shot_batch_16)
    advanced by one batched launch per time step (sw_batch_forward); a bench
    step = one forward of all shots; Gpts/s counts the nodes of every shot."""
    import torch
    from paper_2201_05278_b300 import api, workloads

    shots = workloads.batch_shots(args.workload, n_steps=args.time_steps or None)
    ndim = shots[0].ndim
    stream = torch.cuda.current_stream(dev)
    grids, models = [], {}
    for w in shots:
        g = api.sw_create_grid(ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt,
                               stream=stream)
        if id(w.velocity) not in models:
            models[id(w.velocity)] = (torch.from_numpy(w.velocity).to(dev), w.nodes)
        api.sw_set_model(g, models[id(w.velocity)][0])
        api.sw_set_acquisition(g, w.src_pos, w.rec_pos, api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps),
                               window_radius=w.window_radius)
        grids.append(g)
    b = api.sw_create_batch(grids)
    n_groups, n_items = api.sw_batch_info(b)
    n_steps = shots[0].n_steps
    seis = [torch.empty((n_steps, len(w.rec_pos)), dtype=torch.float32, device=dev) for w in shots]
    shot_nodes = sum(w.nodes for w in shots)
    model_nodes = sum(n for _, n in models.values())

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        api.sw_batch_forward(b, n_steps, seis)
    api.sw_batch_set_profiling(b, PROFILE_EVERY)
    for _ in range(2):  # the second call captures the loop with its timing events
        api.sw_batch_forward(b, n_steps, seis)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stencil_ms, stencil_launches, kernels = 0.0, 0, 0
    start.record(stream)
    for _ in range(args.steps):
        api.sw_batch_forward(b, n_steps, seis)
        ms, nl, nk = api.sw_batch_get_profile(b)
        stencil_ms += ms
        stencil_launches += nl
        kernels += nk
    stop.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = job_seconds(start.elapsed_time(stop) * 1e-3, world, dev) * 1e3
    value = job_throughput(shot_nodes * n_steps, args.steps, world, elapsed_ms * 1e-3)

    # e2e: the same forwards with every shot's seismogram read back into pinned
    # host memory (the inputs stay resident: models and wavelets are set up once)
    seis_h = [torch.empty(s.shape, dtype=torch.float32).pin_memory() for s in seis]
    e2e = None
    if args.e2e_steps > 0:
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            api.sw_batch_forward(b, n_steps, seis)
            for d, h in zip(seis, seis_h):
                h.copy_(d, non_blocking=True)
            torch.cuda.synchronize(dev)
            _ = float(seis_h[-1][-1, 0])
        barrier()
        e2e_s = job_seconds(time.perf_counter() - t0, world, dev)
        e2e = {"value": round(job_throughput(shot_nodes * n_steps, args.e2e_steps, world, e2e_s), 3), "unit": UNIT,
               "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(sum(h.numel() for h in seis_h) * 4)}

    tile_rows, tuned_us = api.sw_batch_get_tile(b) if ndim == 2 else (16, [])
    b.close()
    # the same shots run one after another with the plain single-grid forward
    # (its second call, the captured graph, is the one timed)
    unbatched = None
    if args.e2e_steps > 0 or not args.no_cpu_baseline:
        for g, s in zip(grids, seis):
            api.sw_forward(g, n_steps, s, None)
        barrier()
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        for g, s in zip(grids, seis):
            api.sw_forward(g, n_steps, s, None)
        u1.record(stream)
        barrier()
        ums = u0.elapsed_time(u1)
        unbatched = {"value": round(shot_nodes * n_steps / (ums * 1e-3) / 1e9, 3), "unit": UNIT,
                     "ms": round(ums, 3), "how": "sw_forward per shot, one after another, same GPU"}
    peak, peak_kind = _peaks()
    avg_launch_s = stencil_ms * 1e-3 / max(stencil_launches, 1)
    # 2D: shots of one model share its kappa reads; 3D: every grid reads its own
    alg_bytes = 12 * shot_nodes + 4 * model_nodes if ndim == 2 else 16 * shot_nodes
    achieved = alg_bytes / avg_launch_s / 1e9
    for g in grids:
        g.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "shots": len(shots), "models": n_groups, "work_items_per_step": n_items,
                       "nodes_per_step": shot_nodes, "space_order": shots[0].order,
                       "time_steps_per_forward": n_steps, "receivers_per_shot": len(shots[0].rec_pos),
                       "parallelism": "replicas" if world > 1 else "single",
                       "tile": ("128 x %d (tuner, us per launch for 16/32/64 rows: %s)" % (
                           tile_rows, ", ".join("%.1f" % t for t in tuned_us))) if ndim == 2 else
                       "64 x 16 x plane items of the pipelined kernel",
                       "l2": _l2_note(alg_bytes)},
            "unbatched": unbatched,
            "roofline": _roofline_traffic(
                {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                 "frac": round(achieved / peak, 4), "traffic": None,
                 "kernel": "batched stencil (CUDA events around every %dth launch, %d launches timed)" % (
                     PROFILE_EVERY, stencil_launches),
                 "algorithmic_bytes_per_launch": alg_bytes, "peak_kind": peak_kind}, args.workload),
            "e2e": e2e,
            "gpu_launches": int(kernels),
            "clocks": clk,
        }
        if not args.no_cpu_baseline and world == 1:
            cb, _ = cpu_baseline(args.workload)
            line["cpu_baseline"] = cb
        print(json.dumps(line))


def gradient_cpu_baseline(budget_s=15.0):
    """The FP64 adjoint oracle (numpy) on the 3d_fwi_gradient_256 recipe at
    96^3 (64 receivers; the oracle forms one dense field per receiver, so the
    full grid's 4096 would not fit) for a bounded number of time steps:
    forward states, residual, adjoint sweep, imaging."""
    from paper_2201_05278_b300 import workloads
    import oracle
    from oracle import adjoint as A
    c = workloads.fwi_gradient_256(shape=(96, 96, 96))
    w = c.base
    kw = dict(src_pos=[tuple(c.shots[0])], rec_pos=[tuple(q) for q in w.rec_pos], nbl=w.nbl, bc=w.bc,
              damp_alpha=w.damp_alpha, damp_degree=w.damp_degree, window_radius=w.window_radius)

    def run(steps):
        wav = oracle.ricker_samples(w.f_peak, w.dt, steps, t0=w.t0)
        t = time.perf_counter()
        pb = A.make_problem(3, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt, **kw)
        obs = np.zeros((steps, len(w.rec_pos)))
        A.adjoint_gradient(pb, wav, obs, steps)
        return time.perf_counter() - t

    t1 = run(2) / 2.0
    steps = int(max(2, min(60, budget_s / max(t1, 1e-3))))
    t = run(steps)
    return {"value": round(w.nodes * steps / t / 1e9, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "3d_fwi_gradient_256 recipe on a 96^3 grid with 64 receivers, one shot, %d time steps "
                      "(forward states, adjoint sweep, imaging), FP64 numpy" % steps}, t


CKPT_NAMES = {0: "fp32", 1: "bf16", 2: "fp16", 3: "i16"}


def padded_field_bytes(shape, order):
    """Bytes of one padded FP32 wavefield of the library's layout (x pitch:
    32 + nx rounded up to 128 + 32; y rounded up to 32 plus 2r ghost rows;
    z plus 2r ghost planes; 2D grids have no y padding)."""
    r = order // 2
    nx = shape[-1]
    pitch = 32 + -(-nx // 128) * 128 + 32
    py = -(-shape[1] // 32) * 32 + 2 * r if len(shape) == 3 else 1
    return (shape[0] + 2 * r) * py * pitch * 4


def gradient_schedule(shape, order, n_steps, dev, every, fmt):
    """(checkpoint_every, format, description) for the misfit gradient: every
    forward level kept in device memory (no recomputation) when the n_steps
    + 1 padded fields fit in 80% of the free memory, else the workload's
    checkpoints."""
    import torch
    fb = padded_field_bytes(shape, order)
    free, _ = torch.cuda.mem_get_info(dev)
    if (n_steps + 4) * fb <= 0.8 * free:
        return n_steps, 0, ("every forward level kept in device memory (%d padded FP32 fields, %.1f GB; the "
                            "adjoint sweep recomputes nothing)" % (n_steps + 1, (n_steps + 1) * fb / 1e9))
    return every, fmt, "16-bit fixed point with per-row scale (SW_CKPT_I16) every %d steps" % every


def gradient_error_reduced(dev):
    """Each checkpoint format's gradient error against the FP64 adjoint oracle
    on the misfit-gradient recipe reduced to 96^3 and 200 time steps (20
    checkpoints of 10 steps), one shot; observed data from the true model by
    the GPU forward.  The oracle part takes about a minute of CPU."""
    import torch
    from paper_2201_05278_b300 import api, workloads
    from oracle import adjoint as A
    c = workloads.fwi_gradient_256(n_steps=200, shape=(96, 96, 96))
    w = c.base
    n = w.n_steps
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, n)
    g = api.sw_create_grid(3, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt)
    grads = {}
    try:
        api.sw_set_model(g, torch.from_numpy(c.v_true).to(dev))
        api.sw_set_acquisition(g, c.shots[:1], w.rec_pos, wav, window_radius=w.window_radius)
        obs = torch.zeros((n, len(w.rec_pos)), dtype=torch.float32, device=dev)
        api.sw_forward(g, n, obs)
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev))
        for fmt in CKPT_NAMES:
            gv = torch.zeros(w.shape, dtype=torch.float32, device=dev)
            api.sw_gradient(g, n, obs, gv, c.checkpoint_every, fmt)
            grads[fmt] = gv.cpu().numpy().astype(np.float64)
        gv = torch.zeros(w.shape, dtype=torch.float32, device=dev)
        api.sw_gradient(g, n, obs, gv, n)  # every level kept
        grads["all_levels"] = gv.cpu().numpy().astype(np.float64)
        obs = obs.cpu().numpy().astype(np.float64)
    finally:
        g.close()
    pb = A.make_problem(3, w.shape, w.spacing, w.order, w.velocity.astype(np.float64), w.dt,
                        src_pos=[tuple(c.shots[0])], rec_pos=[tuple(q) for q in w.rec_pos], nbl=w.nbl, bc=w.bc,
                        damp_alpha=w.damp_alpha, damp_degree=w.damp_degree, window_radius=w.window_radius)
    _, g_ref, _ = A.adjoint_gradient(pb, np.asarray(wav, np.float64), obs, n)
    nr = float(np.linalg.norm(g_ref))
    names = dict(CKPT_NAMES, all_levels="every_level_kept")
    return {names[f] + "_rel_l2": round(float(np.linalg.norm(grads[f] - g_ref)) / nr, 6) for f in grads}


def fwi_summary(world, rank, dev, steps=1, warmup=1):
    """The misfit-gradient half of the metric beside the default forward line:
    the 16-shot summed gradient of 3d_fwi_gradient_256 (256^3, 1500 steps,
    I16 checkpoints every 10 steps) through fwi.misfit_gradient (under
    torchrun the ranks split the shots), timed with CUDA events after a
    warm-up (max over ranks), the forward run of the same grid, and the I16
    gradient's error against FP32 checkpoints on the first shot."""
    import torch
    from paper_2201_05278_b300 import api, fwi, workloads
    c = workloads.fwi_gradient_256()
    w = c.base
    N = w.n_steps
    stream = torch.cuda.current_stream(dev)
    g = api.sw_create_grid(3, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt,
                           stream=stream)
    try:
        wav = api.sw_ricker(w.f_peak, w.t0, w.dt, N)
        n_rec, n_shots = len(w.rec_pos), len(c.shots)
        api.sw_set_model(g, torch.from_numpy(c.v_true).to(dev))
        obs = torch.zeros((n_shots, N, n_rec), dtype=torch.float32, device=dev)
        for i in fwi.shots_of_rank(n_shots, world, rank):
            api.sw_set_acquisition(g, c.shots[i:i + 1], w.rec_pos, wav, window_radius=w.window_radius)
            api.sw_forward(g, N, obs[i], None)
        api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev))
        api.sw_set_acquisition(g, c.shots[:1], w.rec_pos, wav, window_radius=w.window_radius)
        tmp = torch.empty((N, n_rec), dtype=torch.float32, device=dev)
        api.sw_forward(g, N, tmp, None)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        forward_ms = None  # the fastest of three forward runs: the ratio below errs high, not low
        for _ in range(3):
            e0.record(stream)
            api.sw_forward(g, N, tmp, None)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            t = e0.elapsed_time(e1)
            forward_ms = t if forward_ms is None else min(forward_ms, t)
        every, fmt, schedule = gradient_schedule(w.shape, w.order, N, dev, c.checkpoint_every, api.SW_CKPT_I16)

        def timed(k, f, n_warm, n_steps_timed):
            for _ in range(n_warm):
                fwi.misfit_gradient(g, c.shots, obs, N, k, f)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(n_steps_timed):
                fwi.misfit_gradient(g, c.shots, obs, N, k, f)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return job_seconds(e0.elapsed_time(e1) * 1e-3 / n_steps_timed, world, dev)

        sec = timed(every, fmt, warmup, steps)
        # the memory-lean schedule beside it: 16-bit checkpoints, segments recomputed
        sec_ck = sec if every != N else timed(c.checkpoint_every, api.SW_CKPT_I16, 0, 1)
        err = None
        if rank == 0:
            ref = torch.zeros(w.shape, dtype=torch.float32, device=dev)
            gv = torch.zeros_like(ref)
            api.sw_gradient_shots(g, c.shots[:1], N, obs[:1], ref, c.checkpoint_every, api.SW_CKPT_FP32)
            api.sw_gradient_shots(g, c.shots[:1], N, obs[:1], gv, c.checkpoint_every, api.SW_CKPT_I16)
            err = float(torch.linalg.vector_norm(gv - ref) / torch.linalg.vector_norm(ref))
    finally:
        g.close()
    return {"workload": "3d_fwi_gradient_256", "grid": list(w.shape), "time_steps": N, "shots": n_shots,
            "checkpoints": schedule,
            "i16_checkpoints_every_%d" % c.checkpoint_every: {
                "ms_per_gradient": round(sec_ck * 1e3, 3),
                "gradient_vs_forward": round(sec_ck / n_shots * world / (forward_ms * 1e-3), 3)},
            "shots_per_s": round(n_shots / sec, 4), "ms_per_gradient": round(sec * 1e3, 3),
            "ms_per_shot_per_gpu": round(sec * 1e3 / n_shots * world, 3), "forward_ms": round(forward_ms, 3), "forward_timing": "fastest of 3 forward runs of one shot",
            "gradient_vs_forward": round(sec / n_shots * world / (forward_ms * 1e-3), 3),
            "value": round(w.nodes * N * n_shots / sec / 1e9, 3), "unit": UNIT,
            "i16_vs_fp32_checkpoints_rel_l2": None if err is None else round(err, 6),
            "error_vs_fp64_oracle": "I16 6.9e-5, FP32 9.6e-6 relative L2 on the recipe reduced to 96^3 and 200 steps "
                                    "(tests/test_gpu_gradient.py; bench.py --workload 3d_fwi_gradient_256 measures "
                                    "it); with every level kept the gradient is bit-identical to the FP32-checkpoint "
                                    "one",
            "timing": "CUDA events around %d summed 16-shot gradient(s) after %d warm-up, max over ranks" % (
                steps, warmup),
            "parallelism": "shots partitioned over %d ranks" % world if world > 1 else "single"}


def run_gradient(args, world, rank, local, dev):
    """Misfit gradient of 3d_fwi_gradient_256: a bench step is the gradient of
    the whole 16-shot objective, J = sum_s J_s and dJ/dc = sum_s dJ_s/dc
    (fwi.misfit_gradient: under torchrun rank r runs shots r, r + N, ... with
    one sw_gradient_shots call and one all-reduce sums misfit and gradient;
    strong scaling, the 16 shots are the whole job).  Each shot: forward
    keeping every level in device memory when the 1501 padded fields fit
    (else 16-bit checkpoints every 10 steps, SW_CKPT_I16, the format within
    the 1e-2 bar at this scale, and the segments recomputed), residual,
    adjoint sweep with imaging.  Gpts/s counts the forward's grid-point
    updates of all shots per second of gradient computation."""
    import torch
    from paper_2201_05278_b300 import api, fwi, workloads

    fmt = api.SW_CKPT_I16
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
    c = workloads.fwi_gradient_256(n_steps=args.time_steps or None, shape=shape)
    w = c.base
    N = w.n_steps
    stream = torch.cuda.current_stream(dev)
    g = api.sw_create_grid(3, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt,
                           stream=stream)
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, N)
    n_rec = len(w.rec_pos)
    n_shots = len(c.shots)
    mine = fwi.shots_of_rank(n_shots, world, rank)

    # observed data of this rank's shots from the true model (FP32 forward on the GPU), before timing
    api.sw_set_model(g, torch.from_numpy(c.v_true).to(dev))
    obs = torch.zeros((n_shots, N, n_rec), dtype=torch.float32, device=dev)
    for i in mine:
        api.sw_set_acquisition(g, c.shots[i:i + 1], w.rec_pos, wav, window_radius=w.window_radius)
        api.sw_forward(g, N, obs[i], None)
    api.sw_set_model(g, torch.from_numpy(w.velocity).to(dev))
    api.sw_set_acquisition(g, c.shots[:1], w.rec_pos, wav, window_radius=w.window_radius)
    # the forward stencil's launch time on this grid, for the roofline line
    api.sw_set_profiling(g, PROFILE_EVERY)
    tmp = torch.empty((N, n_rec), dtype=torch.float32, device=dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    api.sw_forward(g, N, tmp, None)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    forward_ms = f0.elapsed_time(f1)
    st_ms, st_n, _ = api.sw_get_profile(g)
    api.sw_set_profiling(g, 0)

    every, sfmt, schedule = gradient_schedule(w.shape, w.order, N, dev, c.checkpoint_every, fmt)

    def step():
        return fwi.misfit_gradient(g, c.shots, obs, N, every, sfmt)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    # checkpoint formats at this scale against FP32 checkpoints (first shot, untimed)
    at_scale = {}
    if not args.no_cpu_baseline:
        ref = torch.zeros(w.shape, dtype=torch.float32, device=dev)
        api.sw_gradient_shots(g, c.shots[:1], N, obs[:1], ref, c.checkpoint_every, api.SW_CKPT_FP32)
        for f in (api.SW_CKPT_BF16, api.SW_CKPT_FP16, api.SW_CKPT_I16):
            gv = torch.zeros_like(ref)
            api.sw_gradient_shots(g, c.shots[:1], N, obs[:1], gv, c.checkpoint_every, f)
            at_scale[CKPT_NAMES[f] + "_vs_fp32_checkpoints_rel_l2"] = round(
                float(torch.linalg.vector_norm(gv - ref) / torch.linalg.vector_norm(ref)), 6)
        del ref
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernels = 0
    start.record(stream)
    for _ in range(args.steps):
        J, grad = step()
        kernels += api.sw_get_profile(g)[2]
    stop.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = job_seconds(start.elapsed_time(stop) * 1e-3, world, dev) * 1e3
    value = job_throughput(w.nodes * N * n_shots, args.steps, 1, elapsed_ms * 1e-3)

    # e2e: every shot's observed data from pinned host memory, the summed gradient back to it
    e2e = None
    if args.e2e_steps > 0:
        obs_h = obs.cpu().pin_memory()
        grad_h = torch.empty(w.shape, dtype=torch.float32).pin_memory()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            od = obs_h.to(dev, non_blocking=True)
            J, grad = fwi.misfit_gradient(g, c.shots, od, N, every, sfmt)
            grad_h.copy_(grad, non_blocking=True)
            torch.cuda.synchronize(dev)
            _ = float(grad_h[0, 0, 0])
        barrier()
        e2e_s = job_seconds(time.perf_counter() - t0, world, dev)
        e2e = {"value": round(job_throughput(w.nodes * N * n_shots, args.e2e_steps, 1, e2e_s), 3), "unit": UNIT,
               "h2d_bytes_per_step": int(obs_h.numel() * 4), "d2h_bytes_per_step": w.nodes * 4}
    g.close()

    peak, peak_kind = _peaks()
    alg_bytes = BYTES_PER_UPDATE[False] * w.nodes
    achieved = alg_bytes / (st_ms * 1e-3 / max(st_n, 1)) / 1e9
    if rank == 0:
        errors = dict(at_scale)
        if not args.no_cpu_baseline and world == 1:
            errors["vs_fp64_oracle_reduced"] = gradient_error_reduced(dev)
            errors["vs_fp64_oracle_reduced_recipe"] = ("the same recipe at 96^3, 200 time steps, checkpoints every "
                                                       "10 steps, one shot, against the FP64 adjoint oracle")
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "grid": list(w.shape), "space_order": w.order,
                       "time_steps": N, "shots": n_shots, "receivers": n_rec,
                       "checkpoints": schedule,
                       "shots_per_s": round(n_shots * args.steps / (elapsed_ms * 1e-3), 4),
                       "ms_per_shot": round(elapsed_ms / args.steps / n_shots * world, 3),
                       "forward_ms_per_shot": round(forward_ms, 3),
                       "gradient_error": errors,
                       "quantity": "forward grid-point updates of all 16 shots per second of the summed misfit "
                                   "gradient (per shot: forward, residual, adjoint sweep with imaging; the "
                                   "segments are recomputed unless every level is kept)",
                       "parallelism": ("shots partitioned over %d ranks, one all-reduce of misfit and gradient"
                                       % world) if world > 1 else "single",
                       "l2": "inputs larger than L2 (each time step streams %.0f MB)" % (alg_bytes / 1e6)},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "forward stencil of the same grid (CUDA events around every %dth launch of a "
                                   "profiled sw_forward just before the timed region, %d launches)" % (
                                       PROFILE_EVERY, st_n),
                         "algorithmic_bytes_per_launch": alg_bytes, "peak_kind": peak_kind},
            "e2e": e2e,
            "gpu_launches": int(kernels),
            "clocks": clk,
        }
        if not args.no_cpu_baseline and world == 1:
            cb, _ = gradient_cpu_baseline()
            line["cpu_baseline"] = cb
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="3d_vd_512x512x384")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--time-steps", type=int, default=0,
                    help="override the workload's time steps per forward (profiling runs only)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="forwards timed end to end (0 skips)")
    ap.add_argument("--shape", default="",
                    help="override the workload's grid as nz,ny,nx (profiling runs on a smaller case only)")
    ap.add_argument("--no-fwi", action="store_true",
                    help="skip the misfit-gradient summary the default workload's line carries")
    ap.add_argument("--stencil", default="", choices=["", "auto", "plain", "tb2"],
                    help="kernel variant (default: the library's choice; tb2 for 2d_layered_4096, with the "
                         "per-step kernels timed beside it)")
    args = ap.parse_args()
    world, rank, local = _dist()

    if args.impl == "reference":
        if rank != 0:
            return
        from paper_2201_05278_b300 import workloads as _w
        if args.workload in _w.GRADIENT_NAMES:  # the FP64 adjoint oracle on the reduced recipe
            per, secs = [], 0.0
            for _ in range(args.warmup):
                gradient_cpu_baseline(budget_s=2.0)
            for _ in range(args.steps):
                cb, t = gradient_cpu_baseline(budget_s=3.0)
                per.append(cb["value"])
                secs += t
            v = statistics.median(per)
            cb["value"] = v
            print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
                              "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
                              "data": "synthetic", "config": {"workload": args.workload}, "cpu_baseline": cb,
                              "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
            return
        # each bench step: one call of the oracle's loop for a bounded number of
        # time steps (about 3 s), the set-up done once before the warm-up
        runner = OracleRunner(args.workload)
        k = runner.steps_for(3.0)
        for _ in range(args.warmup):
            runner.run(k)
        secs = 0.0
        for _ in range(args.steps):
            secs += runner.run(k)
        v = round(runner.nodes * k * args.steps / secs / 1e9, 5)
        cb = {"value": v, "unit": UNIT, "cores": runner.threads, "kind": "oracle", "sample": runner.describe(k)}
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": args.workload},
                          "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    import torch.distributed as dist
    from paper_2201_05278_b300 import api, workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if args.workload in workloads.BATCH_NAMES:
        run_batch(args, world, rank, local, dev)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload in workloads.GRADIENT_NAMES:
        run_gradient(args, world, rank, local, dev)
        if world > 1:
            dist.destroy_process_group()
        return

    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
    w = workloads.make(args.workload, n_steps=args.time_steps or None, shape=shape)
    vd = w.density is not None
    stream = torch.cuda.current_stream(dev)
    g = api.sw_create_grid(w.ndim, w.shape, w.spacing, w.order, w.nbl, w.bc, w.damp_alpha, w.damp_degree, w.dt,
                           stream=stream)
    vel_d = torch.from_numpy(w.velocity).to(dev)
    rho_d = None if w.density is None else torch.from_numpy(w.density).to(dev)
    api.sw_set_model(g, vel_d, rho_d)
    stencil = args.stencil or ("tb2" if args.workload == "2d_layered_4096" else "")
    variants = {"auto": api.SW_STENCIL_AUTO, "plain": api.SW_STENCIL_PLAIN, "tb2": api.SW_STENCIL_TB2}
    if stencil:
        api.sw_set_stencil_variant(g, variants[stencil])
    two_step = api.sw_get_stencil_variant(g) == api.SW_STENCIL_TB2
    wav = api.sw_ricker(w.f_peak, w.t0, w.dt, w.n_steps)
    api.sw_set_acquisition(g, w.src_pos, w.rec_pos, wav, window_radius=w.window_radius)
    n_rec = len(w.rec_pos)
    seis = torch.empty((w.n_steps, n_rec), dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        api.sw_forward(g, w.n_steps, seis, None)
    api.sw_set_profiling(g, PROFILE_EVERY)
    cluster_run = api.sw_get_stencil_variant(g) == api.SW_STENCIL_CLUSTER
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stencil_ms, stencil_launches, kernels = 0.0, 0, 0
    start.record(stream)
    for _ in range(args.steps):
        api.sw_forward(g, w.n_steps, seis, None)
        ms, nl, nk = api.sw_get_profile(g)
        stencil_ms += ms
        stencil_launches += nl
        kernels += nk
    stop.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = job_seconds(start.elapsed_time(stop) * 1e-3, world, dev) * 1e3
    api.sw_set_profiling(g, False)
    value = job_throughput(w.updates, args.steps, world, elapsed_ms * 1e-3)

    # e2e through the C ABI with host buffers: H2D of the velocity model every step
    # (sw_set_model from pinned host memory) and D2H of the seismogram.
    vel_h = torch.from_numpy(w.velocity).pin_memory()
    rho_h = None if w.density is None else torch.from_numpy(w.density).pin_memory()
    seis_h = torch.empty((w.n_steps, n_rec), dtype=torch.float32).pin_memory()
    e2e = None
    if args.e2e_steps > 0:
        # one untimed call first, as for the device-timed forwards: the grid
        # allocates its staging buffers for host inputs and outputs on the
        # first call that passes host memory
        api.sw_set_model(g, vel_h, rho_h)
        api.sw_forward(g, w.n_steps, seis_h, None)
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            api.sw_set_model(g, vel_h, rho_h)
            api.sw_forward(g, w.n_steps, seis_h, None)
            _ = float(seis_h[-1, 0])
        barrier()
        e2e_s = job_seconds(time.perf_counter() - t0, world, dev)
        e2e_value = job_throughput(w.updates, args.e2e_steps, world, e2e_s)
        h2d = w.velocity.nbytes + (0 if w.density is None else w.density.nbytes)
        e2e = {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": seis_h.numel() * 4}

    # the two-step run beside the per-step kernels on the same grid
    per_step = None
    if two_step and args.workload == "2d_layered_4096" and not args.stencil:
        api.sw_set_stencil_variant(g, api.SW_STENCIL_PLAIN)
        api.sw_set_profiling(g, PROFILE_EVERY)
        for _ in range(2):
            api.sw_forward(g, w.n_steps, seis, None)
        barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            api.sw_forward(g, w.n_steps, seis, None)
        p1.record(stream)
        barrier()
        pms, pn, _ = api.sw_get_profile(g)
        api.sw_set_profiling(g, 0)
        pl_ms = p0.elapsed_time(p1) / args.steps
        per_step = {"value": round(w.updates / (pl_ms * 1e-3) / 1e9, 3), "unit": UNIT, "ms": round(pl_ms, 3),
                    "stencil_us_per_step": round(pms * 1e3 / max(pn, 1), 3),
                    "how": "the same forward on the per-step 2D kernels (SW_STENCIL_PLAIN), same GPU and process"}
    peak, peak_kind = _peaks()
    avg_launch_s = stencil_ms * 1e-3 / max(stencil_launches, 1)
    # algorithmic bytes of one timed launch: one step reads p[n], p[n-1],
    # kappa (, ln rho) and writes p[n+1]; a two-step launch reads the first
    # three once and writes two levels
    alg_bytes = (20 if two_step else BYTES_PER_UPDATE[vd]) * w.nodes
    achieved = alg_bytes / avg_launch_s / 1e9
    api.sw_destroy_grid(g)
    # the misfit-gradient half of the metric, beside the headline forward
    fwi_line = None
    if args.workload == "3d_vd_512x512x384" and not args.no_fwi and not args.shape and not args.time_steps:
        fwi_line = fwi_summary(world, rank, dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "grid": list(w.shape), "space_order": w.order,
                       "time_steps_per_forward": w.n_steps, "receivers": n_rec, "sources": len(w.src_pos),
                       "variable_density": vd, "parallelism": "replicas" if world > 1 else "single",
                       "l2": ("inputs larger than L2 (each time step streams %.0f MB)" % (alg_bytes / 1e6))
                       if alg_bytes > 126e6 else
                       ("working set fits in L2 (%.1f MB per time step): latency-bound, HBM is not the bound"
                        % (alg_bytes / 1e6))},
            "roofline": _roofline_traffic(
                {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                 "frac": round(achieved / peak, 4), "traffic": None,
                 "kernel": ("cluster-resident 2D run (one launch per forward with CUDA events around "
                            "it, counted as %d time steps)" % stencil_launches) if cluster_run else
                           ("two-step 2D kernel, two time steps per launch (CUDA events around every %dth "
                            "launch, %d launches timed)" % (PROFILE_EVERY, stencil_launches)) if two_step else
                           ("stencil (CUDA events around every %dth launch, %d launches timed)" % (
                               PROFILE_EVERY, stencil_launches)),
                 "algorithmic_bytes_per_launch": alg_bytes, "peak_kind": peak_kind}, args.workload, args.shape),
            "e2e": e2e,
            "gpu_launches": int(kernels),
            "clocks": clk,
        }
        if two_step:
            line["config"]["stencil"] = "two time steps per launch (temporal blocking, SW_STENCIL_TB2)"
        if per_step is not None:
            line["per_step_kernels"] = per_step
        if fwi_line is not None:
            line["fwi"] = fwi_line
        if not args.no_cpu_baseline and world == 1:
            cb, _ = cpu_baseline(args.workload)
            line["cpu_baseline"] = cb
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
