#!/usr/bin/env python3
"""Throughput of the SACRA-2D hot path on GB300: cell-updates per second per
RK stage of Z4c + HLLC GRHD on the fixed-mesh-refinement cartoon grid.

Headline workload (default): the unstable-branch migration star (K=100,
Gamma=2, rho_c=7.993e-3 with a 1% pressure depletion, Gamma_th=2, atmosphere
1e-10 of rho_c), equatorial symmetry, 5 FMR levels of 512^2 cells, finest
dx = 0.1, classical RK4, FP64.  One step = the whole hot path: ghost fill /
prolongation, hydro and Z4c right-hand sides, RK combination with algebraic
constraints and primitive recovery for every stage, then restriction +
reflux; the constraint and conservation diagnostics of the state at the start
of each step are formed inside its first stage and read back to the host
every step.  The working set (about 2.5 GB of FP64 state per step) exceeds the
129 MB L2, so no flush is needed.

Beside it on the same line: the mixed-precision form of the same workload;
the stable star (3 levels of 256^2, SSP-RK3) in both forms; the large run
(the migration star at 7 levels of 1024^2, levels 5 and 6 sub-cycled) in
both forms; the batched sweep of 64 stars; the end-to-end rate through the C
ABI with the state copied both ways every step; the roofline of the dominant
kernel and of the whole step against the method's own operation count.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank advances its own replica (independent problems, no
exchange step; weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import ctypes
import dataclasses
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage (Z4c+HLLC), FP64 vs mixed/batched, % of roofline"
UNIT = "cell-updates/s"

# FP64 operations per unit of work of the method (add, sub, mul = 1; an FMA
# = 2; div, sqrt = 1).  Stencil kernels, counted by hand on the minimal FP64
# form: the derivative pass with symmetric pair sums shared between the
# derivative kinds, weights and 1/dx hoisted, zero taps skipped, the mixed x-z
# derivative separable and the lopsided advection at beta != 0 (2139 per cell;
# the kernel forms these sums exactly in integers, so this is FP64-equivalent
# work, not FP64 instructions); the cartoon terms with the interpolation,
# rotation and plane differences folded into one 9-point sum per output (591
# per cell of the plane patch).  Pointwise kernels (no stencil redundancy):
# the FP64 operations their formulation executes per unit, from ncu's
# instruction counters (dfma x 2 + dmul + dadd) on stage 0 of the migration
# star's second step: they include what the data decide (faces between equal
# states take the state's own flux, matter at rest skips its Lorentz factor,
# the recovery's iteration counts).  Units: a cell of the update region; a face
# for the flux kernels; a cell of the plane patch for the cartoon kernel.
METHOD_FLOPS = {
    "k_z4c_derivs": 2139.0, "k_cartoon": 591.0, "k_z4c_point": 2001.0, "k_flux_x": 508.0,
    "k_flux_z": 536.0, "k_hydro_rhs": 391.0, "k_rk_update": 396.0,
}
NOMINAL_FP64_TFLOPS = 1.25


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- distributed plumbing

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if ws > 1:
        import torch
        import torch.distributed as td
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        td.init_process_group(backend=backend)
        dist = td
    return dist, rank, ws, local


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock, max clock and throttle
    reasons of one GPU while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workloads

WORKLOADS = ("migration_5x512", "tov_stable_3x256", "large_7x1024", "shock_tube_400x4")


def workload(name):
    """(RunConfig, per-level initial data) of a named workload."""
    from paper_2502_03223_gb300 import workloads as W
    if name == "tov_stable_3x256":
        cfg, tov = W.config_tov_stable()
        return cfg, [W.tov_level_data(cfg, tov, l) for l in range(cfg.n_levels)]
    if name == "migration_5x512":
        cfg, tov = W.config_migration()
        return cfg, [W.tov_level_data(cfg, tov, l, p_deplete=0.99) for l in range(cfg.n_levels)]
    if name == "large_7x1024":
        # the migration star at 7 levels of 1024^2; the paper's l_fix = 4: levels >= 5 sub-cycle
        cfg, tov = W.config_migration(N=1024, n_levels=7)
        cfg = dataclasses.replace(cfg, name="large_7x1024", subcycle_from=5)
        return cfg, [W.tov_level_data(cfg, tov, l, p_deplete=0.99) for l in range(cfg.n_levels)]
    if name == "shock_tube_400x4":
        cfg = W.config_shock_tube()
        return cfg, [W.shock_tube_data(cfg)]
    raise SystemExit("unknown workload " + name)


def cell_updates_per_step(cfg):
    """Interior cells x RK stages of one (coarse) step; a sub-cycled level
    takes 2^(l - K + 1) steps per coarse step."""
    K = cfg.subcycle_from
    n = 0
    for l in range(cfg.n_levels):
        reps = (1 << (l - K + 1)) if (0 < K < cfg.n_levels and l >= K) else 1
        n += cfg.nx * cfg.nz * reps
    return n * cfg.n_stages


def describe(cfg):
    return {"workload": cfg.name, "levels": cfg.n_levels, "cells_per_level": [cfg.nx, cfg.nz],
            "finest_dx": cfg.dx(cfg.n_levels - 1), "integrator": "SSP-RK3" if cfg.rk else "RK4",
            "stages_per_step": cfg.n_stages, "cell_updates_per_step": cell_updates_per_step(cfg),
            "subcycled_from_level": cfg.subcycle_from if 0 < cfg.subcycle_from < cfg.n_levels else None}


def fp64_peak():
    """Measured FP64 FMA throughput (TFLOP/s) of this GPU by the probe kernel."""
    from paper_2502_03223_gb300 import build as B
    lib = ctypes.CDLL(B.PROBE)
    lib.sacra_probe_fp64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    tf, ms = ctypes.c_double(0), ctypes.c_double(0)
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    rc = lib.sacra_probe_fp64(sms * 8, 256, 2048, 5, ctypes.byref(tf), ctypes.byref(ms))
    return tf.value if rc == 0 else None


def read_traffic(workload_name):
    """DRAM bytes per launch of a kernel from the committed ncu summary of
    this workload (profiles/traffic_<workload>.txt), kept only if the kernel's
    sources still hash to the recorded value (else the counters are stale)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_%s.txt" % workload_name)
    out = {}
    if not os.path.exists(path):
        return out
    for ln in open(path):
        parts = ln.split()
        if len(parts) != 5 or ln.startswith("#"):
            continue
        name, bytes_per_launch, cells_per_launch, digest, files = parts
        h = hashlib.sha256()
        try:
            for fn in files.split(","):
                h.update(open(os.path.join(ROOT, "paper_2502_03223_gb300", "csrc", fn), "rb").read())
        except OSError:
            continue
        if h.hexdigest()[:16] == digest:
            out[name] = (float(bytes_per_launch), float(cells_per_launch))
    return out


# ---------------------------------------------------------------- the reference arm (CPU oracle)

def oracle_sample(cfg, datas, stages=1, full_step=False):
    """Time `stages` RK stages (ghost fill + stage) of the whole hierarchy on
    the CPU oracle, or one whole step (every stage, restriction and reflux)
    with full_step.  Returns (cell-updates, seconds)."""
    import oracle as O
    o = O.Oracle(cfg)
    for l, d in enumerate(datas):
        o.set_level(l, 0, d)
    t0 = time.perf_counter()
    if full_step:
        o.step(cfg.dt, 1)
        n = cell_updates_per_step(cfg)
    else:
        for s in range(stages):
            o.fill(s % cfg.n_stages, cfg.dt)
            o.stage(s % cfg.n_stages, cfg.dt)
        n = cfg.interior_cells * stages
    el = time.perf_counter() - t0
    o.close()
    return n, el


def run_reference(args, dist, rank, ws):
    """The reference arm: the CPU oracle on the host cores, each step one RK
    stage of the workload (a bounded sample), rank 0 only."""
    if rank != 0:
        return
    import oracle as O
    O.build()
    O.set_threads(0)                      # every host core (the per-cell arithmetic does not depend on it)
    cores = O.get_threads()
    cfg, datas = workload(args.workload)
    for _ in range(args.warmup):
        oracle_sample(cfg, datas, 1)
    cells = 0
    el = 0.0
    for _ in range(args.steps):
        c, t = oracle_sample(cfg, datas, 1)
        cells += c
        el += t
    value = cells / el
    conf = describe(cfg)
    conf["reference"] = "CPU oracle (plain FP64 C)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": conf,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: one RK stage (ghost fill + stage) of the whole %s hierarchy, "
                                       "OpenMP over %d threads" % (cfg.name, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- timing helpers

def timed_region(sim, nsteps, dt, dist, with_diag):
    """nsteps graph-replayed steps bracketed by a barrier and a device
    synchronize, timed by CUDA events on the library's stream.  with_diag:
    each step forms the diagnostics of its starting state and reads them
    back.  Returns (ms, launches, last diagnostics or None, clocks)."""
    import torch
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    n0 = sim.launch_count
    barrier(dist)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    diag = None
    if with_diag:
        for _ in range(nsteps):
            diag = sim.step_constraints(dt, 1, use_graph=True)[0]
    else:
        sim.step(dt, nsteps, use_graph=True)
    ev1.record(sim.stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    return ev0.elapsed_time(ev1), sim.launch_count - n0, diag, clocks


def snapshot(sim, cfg):
    """The state of every level (host copies, the layout set_initial_data RAW takes)."""
    out = []
    for l in range(cfg.n_levels):
        a = np.empty(30 * sim.px * sim.pz, dtype=np.float64)
        sim.read_level(l, a)
        out.append(a)
    return out


def restore(sim, snap, dt, warm=2):
    """Back to a snapshot (primitives recovered from it), then `warm` graph steps."""
    from paper_2502_03223_gb300 import sacra2d as S
    for l, a in enumerate(snap):
        sim.set_initial_data(l, S.RAW, a)
    for _ in range(warm):
        sim.step(dt, 1, use_graph=True)
    sim.sync()


def bench_context(cfg, datas, args, dist, ws, repeats, repeat_steps, steps=None, tune=True):
    """Build a context of cfg, warm it up, autotune it (outside the timed
    regions), then time `steps` steps (the line's region) and `repeats` more
    regions of `repeat_steps` steps each.  The star evolves (the migration
    star sheds matter into the atmosphere, which moves work between kernels),
    so every repeat starts from the state the line's region started from (a
    snapshot, restored outside the timed region): the median is over the same
    stretch of evolution.  Returns (sim, result dict); result["_snap"] holds
    the snapshot when repeats > 0."""
    from paper_2502_03223_gb300 import sacra2d as S
    steps = args.steps if steps is None else steps
    sim = S.Sacra(cfg)
    for l, d in enumerate(datas):
        sim.set_initial_data(l, S.PRIM_METRIC, d)
    lockstep = not (0 < cfg.subcycle_from < cfg.n_levels)
    dt = cfg.dt
    for _ in range(args.warmup):
        sim.step(dt, 1, use_graph=True)
    sim.sync()
    tuning = sim.tune(reps=4) if (tune and not args.no_tune) else None
    for _ in range(2):
        sim.step(dt, 1, use_graph=True)
    sim.sync()
    diag0 = sim.constraints() if lockstep else None
    cps = cell_updates_per_step(cfg)
    snap = snapshot(sim, cfg) if repeats > 0 else None
    if snap is not None:
        restore(sim, snap, dt)     # the line's region starts from the snapshot too
    ms, launches, diag_in, clocks = timed_region(sim, steps, dt, dist, lockstep)
    ms = max_over_ranks(dist, ms)
    res = {"value": ws * cps * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "gpu_launches": launches, "clocks": clocks, "tuning": tuning,
           "diagnostics_in_step": lockstep}
    if repeats > 0:
        vals, rclk = [], []
        for _ in range(repeats):
            restore(sim, snap, dt)
            rms, _, _, rc = timed_region(sim, repeat_steps, dt, dist, lockstep)
            rms = max_over_ranks(dist, rms)
            vals.append(ws * cps * repeat_steps / (rms * 1e-3))
            rclk.append(rc.get("sm_mhz"))
        res["repeats"] = {"n": repeats, "steps_each": repeat_steps, "from": "the line's starting state (restored)",
                          "median_value": float(np.median(vals)),
                          "values": vals, "median_ms_per_step": ws * cps / float(np.median(vals)) * 1e3,
                          "sm_mhz": rclk}
    res["_diag_in"] = diag_in
    res["_diag0"] = diag0
    res["_snap"] = snap
    return sim, res


def errors_vs_oracle(cfg, datas, sims, steps=1):
    """Advance the oracle and each simulation `steps` steps from the same
    initial data; per simulation the rest-mass density L1 error relative to
    the oracle and, per output field, the largest error relative to the scale
    of the field's physical group (interior cells of every level)."""
    import oracle as O
    from paper_2502_03223_gb300 import sacra2d as S
    from paper_2502_03223_gb300.workloads import CONS_NAMES, MET_NAMES
    # physical groups sharing one scale: dimensionless metric, curvature, Gt^i,
    # shift, hydro (q_Sy: x_max times the hydro scale, as q_Sphi = x q_Sy)
    groups = [[0, 1, 2, 3, 4, 5, 6, 18], [7, 8, 9, 10, 11, 12, 13, 17], [14, 15, 16],
              [19, 20, 21, 22, 23, 24], [25, 26, 28, 29]]

    def group_scale(B, f, xmax):
        if f == 27:
            return max(float(np.max(np.abs(B[27]))), xmax * max(float(np.max(np.abs(B[i]))) for i in groups[4]))
        g_ = next(g_ for g_ in groups if f in g_)
        return max(float(np.max(np.abs(B[i]))) for i in g_)

    names = MET_NAMES + CONS_NAMES
    o = O.Oracle(cfg)
    for l, d in enumerate(datas):
        o.set_level(l, 0, d)
    o.step(cfg.dt, steps)
    g = 8
    out = []
    for sim in sims:
        for l, d in enumerate(datas):
            sim.set_initial_data(l, S.PRIM_METRIC, d)
        sim.step(cfg.dt, steps, use_graph=False)
        num = den = 0.0
        worst = {}
        for l in range(cfg.n_levels):
            sl = (slice(g, g + cfg.nz), slice(g, g + cfg.nx))
            a = sim.read(l, S.PRIMS, 0)[sl]
            b = o.read(l, 2, 0)[sl]
            num += float(np.abs(a - b).sum())
            den += float(np.abs(b).sum())
            B = [o.read(l, 0, f) for f in range(30)]
            xmax = (cfg.nx + 8) * cfg.dx(l) if cfg.geometry == 1 else 1.0
            for f in range(30):
                sg = group_scale(B, f, xmax)
                e = float(np.max(np.abs(sim.read(l, S.STATE_STEP, f)[sl] - B[f][sl]))) / sg if sg > 0 else 0.0
                worst[names[f]] = max(worst.get(names[f], 0.0), e)
        out.append({"rho_l1_rel": num / den, "steps": steps,
                    "max_group_rel": {k: float("%.3g" % v) for k, v in worst.items()}})
    o.close()
    return out


def run_batch(args, dist, ws):
    """Time whole steps of the batched sweep: n stars of grids {128..512}^2
    with 2-5 levels each (seeded), mixed precision, autotuned, graph-replayed.
    No diagnostics in these steps (the sweep reports throughput only)."""
    import torch
    from paper_2502_03223_gb300 import sacra2d as S
    from paper_2502_03223_gb300 import workloads as W
    stars = W.config_batch_sweep(n_stars=args.batch_stars)
    cfgs = [c for c, _ in stars]
    dt = min(c.dt for c in cfgs)
    t0 = time.perf_counter()
    b = S.SacraBatch(cfgs)
    for i, (c, tov) in enumerate(stars):
        for l in range(c.n_levels):
            b.set_initial_data(i, l, S.PRIM_METRIC, W.tov_level_data(c, tov, l, p_deplete=0.99 if tov.rho_c > 3.2e-3 else 1.0))
    t_init = time.perf_counter() - t0
    b.step(dt, 1, use_graph=False)
    b.sync()
    tuning = b.tune(reps=1) if not args.no_tune else None
    for _ in range(max(args.warmup - 1, 2)):
        b.step(dt, 1, use_graph=True)
    b.sync()
    steps = max(3, min(args.steps, args.batch_steps))

    def timed(nsteps):
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        n0 = b.launch_count
        barrier(dist)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(b.stream)
        b.step(dt, nsteps, use_graph=True)
        ev1.record(b.stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        barrier(dist)
        return max_over_ranks(dist, ev0.elapsed_time(ev1)), b.launch_count - n0, sampler.stop()

    ms, launches, clocks = timed(steps)
    # per-kernel device time of one eager step (events around each launch): the
    # batched kinds against the per-level ghost fill, prolongation, restriction,
    # reflux and recovery launches
    b.profile(True)
    b.step(dt, 1, use_graph=False)
    brep = b.profile_report()
    b.profile(False)
    btot = sum(v[0] for v in brep.values())
    per_level = ("k_parity_x", "k_parity_z", "k_outer", "k_prolong", "k_restrict", "k_reflux", "k_c2p_region",
                 "k_outflow", "k_time_interp")
    kshare = {k: round(v[0] / btot, 4) for k, v in sorted(brep.items(), key=lambda kv: -kv[1][0])}
    klaunch = {k: int(v[1]) for k, v in brep.items()}
    # the learned recovery seed, trained on tuples of this batch's own state
    learned = None
    if not args.no_learned:
        buf = torch.zeros((2_000_000, 10), dtype=torch.float32, device="cuda")
        n = b.mlp_collect(buf)
        if n >= 1000:
            net, rep, _ = S.mlp_train(buf[:n], steps=3000, batch_blocks=32, lr=1e-2, seed=1, kmin=0.2)
            del buf
            b.set_mlp(net)
            b.step(dt, 2, use_graph=True)
            lms, _, lclocks = timed(steps)
            learned = {"ms_per_step": lms / steps, "tuples": n, "train": rep, "clocks": lclocks}
            b.set_mlp(None)
    cells = sum(cell_updates_per_step(c) for c in cfgs)
    if learned is not None:
        learned["value"] = ws * cells * steps / (learned["ms_per_step"] * steps * 1e-3)
        learned["unit"] = UNIT
    diag = b.constraints(0)
    b.close()
    return {"workload": "batch_sweep_%d" % len(cfgs), "value": ws * cells * steps / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps, "n_stars": len(cfgs),
            "cell_updates_per_step": cells, "precision": "mixed", "cuda_graph": True, "tuning": tuning,
            "gpu_launches": launches, "launches_per_step": launches / steps, "clocks": clocks, "init_s": t_init,
            "kernel_share": kshare, "launches_per_kernel_eager_step": klaunch,
            "per_level_share": round(sum(v for k, v in kshare.items() if k in per_level), 4),
            "eager_step_device_ms": btot,
            "learned_seed": learned, "star0_H_L2": diag[0],
            "sizes": sorted(set((c.nx, c.n_levels) for c in cfgs))[:40]}


MIXED_ARITH = ("FP32: reconstruction, Riemann solver, hydro sources, the weighted sums of the Z4c finite "
               "differences (of FP64-exact differences, as FP32 hi/lo splits), the cartoon planes and the Z4c "
               "pointwise algebra; FP64: primitive recovery, algebraic constraints, RK combination, flux "
               "divergence and registers, restriction, prolongation, diagnostics")


def pair_forms(cfg, datas, args, dist, ws, repeats, repeat_steps, steps):
    """FP64 and mixed contexts of one workload, each timed; returns
    (fp64 sim, fp64 result, mixed sim, mixed result)."""
    from paper_2502_03223_gb300 import sacra2d as S
    sim, r64 = bench_context(cfg, datas, args, dist, ws, repeats, repeat_steps, steps=steps)
    if args.fp64_only:
        return sim, r64, None, None
    mcfg = dataclasses.replace(cfg, precision=S.MIXED)
    msim, rmx = bench_context(mcfg, datas, args, dist, ws, repeats, repeat_steps, steps=steps)
    rmx["speedup_vs_fp64"] = rmx["value"] / r64["value"]
    rmx["arith"] = MIXED_ARITH
    return sim, r64, msim, rmx


def strip(d):
    return {k: v for k, v in d.items() if not k.startswith("_")}


def collect_tuples(sim, cfg, buf, off, rounds, steps_between):
    """Recovery tuples (inputs, converged log10 P/D) from the context's own
    state at `rounds` times `steps_between` steps apart, appended to buf at
    row off; returns the new row count."""
    for _ in range(rounds):
        if off >= buf.shape[0]:
            break
        off += sim.mlp_collect(buf[off:])
        sim.step(cfg.dt, steps_between, use_graph=True)
    sim.sync()
    return off


def seed_measurement(sim, cfg, net, steps, dist, ws):
    """The large run with and without the learned seed: Illinois evaluations
    per recovery over one step (counting pass), the stage update's device time
    per launch (profiled eager step) and the step rate (graph-replayed timed
    region), each form from the same state."""
    out = {}
    for name, n in (("without", None), ("with", net)):
        sim.set_mlp(n)
        sim.step(cfg.dt, 1, use_graph=True)       # a graph with this form
        sim.c2p_counting(True)
        sim.c2p_counts(reset=True)
        sim.step(cfg.dt, 1, use_graph=False)
        ev, tried, held, nrec = sim.c2p_counts(reset=True)
        sim.c2p_counting(False)
        sim.profile(True)
        sim.step(cfg.dt, 1, use_graph=False)
        rep = sim.profile_report()
        sim.profile(False)
        rk = rep.get("k_rk_update", (0.0, 1, 0))
        sim.step(cfg.dt, 1, use_graph=True)
        ms, _, _, clocks = timed_region(sim, steps, cfg.dt, dist, False)
        ms = max_over_ranks(dist, ms)
        out[name] = {"value": ws * cell_updates_per_step(cfg) * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                     "evaluations_per_recovery": ev / max(nrec, 1), "recoveries": nrec, "seed_tried": tried,
                     "seed_held": held, "rk_update_ms_per_launch": rk[0] / max(rk[1], 1), "clocks": clocks}
    sim.set_mlp(None)
    return out


def run_native(args, dist, rank, ws, local):
    import torch
    from paper_2502_03223_gb300 import build as B
    B.build()
    from paper_2502_03223_gb300 import sacra2d as S
    torch.cuda.set_device(local)
    cfg, datas = workload(args.workload)
    cps = cell_updates_per_step(cfg)
    reps, rsteps = args.repeats, max(args.steps, args.repeat_steps)

    # ---- the headline workload: FP64 (the line's value) and the mixed form
    sim, r64, msim, rmx = pair_forms(cfg, datas, args, dist, ws, reps, rsteps, args.steps)
    value, ms_step = r64["value"], r64["ms_per_step"]
    diag = sim.constraints() if r64["diagnostics_in_step"] else None
    mixed = strip(rmx) if rmx is not None else None
    if rmx is not None and r64["_diag_in"] is not None and rmx["_diag_in"] is not None:
        # ||H|| of the same starting state of the last timed step, formed in the step
        # (mixed: from the FP32 Ricci scalar of its pointwise pass)
        h64, hmx = r64["_diag_in"][0], rmx["_diag_in"][0]
        mixed["H_L2_in_step"] = {"mixed": hmx, "fp64": h64, "rel_diff": abs(hmx - h64) / h64 if h64 else None}

    # ---- end to end through the C ABI with host buffers: every step the state
    # of all levels goes host -> device from pinned memory (set_initial_data,
    # RAW), one step runs with its diagnostics read back, and the evolved state
    # of all levels comes back device -> host into pinned memory (read_level)
    host_in, host_out = [], []
    for l in range(cfg.n_levels):
        a = torch.empty(30 * sim.px * sim.pz, dtype=torch.float64, pin_memory=True).numpy()
        sim.read_level(l, a)
        host_in.append(a)
        host_out.append(torch.empty(30 * sim.px * sim.pz, dtype=torch.float64, pin_memory=True).numpy())
    e2e_steps = max(3, min(args.steps, 20))
    h2d = sum(a.nbytes for a in host_in)
    d2h = sum(a.nbytes for a in host_out) + ctypes.sizeof(S.SacraDiag)
    sim.sync()
    barrier(dist)
    phase = [0.0, 0.0, 0.0]        # host time in the uploads, the step, the readback
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        for l in range(cfg.n_levels):
            sim.set_initial_data(l, S.RAW, host_in[l])
        tb = time.perf_counter()
        sim.step_constraints(cfg.dt, 1, use_graph=True)
        tc = time.perf_counter()
        for l in range(cfg.n_levels):
            sim.read_level(l, host_out[l])
        td = time.perf_counter()
        phase[0] += tb - ta; phase[1] += tc - tb; phase[2] += td - tc
    el = time.perf_counter() - t0
    el = max_over_ranks(dist, el)
    e2e = {"value": ws * cps * e2e_steps / el, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "steps": e2e_steps, "what": "per step: all levels' state host->device (pinned), one step with its "
                                       "diagnostics read back, all levels' evolved state device->host (pinned)",
           "ms_per_step": {"upload": phase[0] / e2e_steps * 1e3, "step": phase[1] / e2e_steps * 1e3,
                           "readback": phase[2] / e2e_steps * 1e3}}

    # ---- per-kernel device time (eager launches bracketed by CUDA events), from
    # the timed regions' starting state
    if r64.get("_snap") is not None:
        restore(sim, r64["_snap"], cfg.dt)
    sim.profile(True)
    prof_steps = max(2, min(args.steps, 5))
    for _ in range(prof_steps):
        sim.step_constraints(cfg.dt, 1, use_graph=False)
    rep = sim.profile_report()
    sim.profile(False)
    kern = {k: v for k, v in rep.items()}
    dom = max((k for k in kern if k in METHOD_FLOPS), key=lambda k: kern[k][0])
    tot_ms, n_launch, n_cells = kern[dom]
    avg_s = tot_ms * 1e-3 / n_launch
    units_per_launch = n_cells / n_launch
    achieved = METHOD_FLOPS[dom] * units_per_launch / avg_s / 1e12
    peak = fp64_peak()
    traffic = read_traffic(cfg.name).get(dom)
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if peak else None,
                "traffic": (traffic[0] / traffic[1] * units_per_launch) if traffic else None,
                "peak_source": "FP64 FMA probe measured in this run (nominal %.2f TFLOP/s); of measured"
                               % NOMINAL_FP64_TFLOPS,
                "method_flops_per_unit": METHOD_FLOPS[dom], "avg_launch_ms": avg_s * 1e3,
                "units_per_launch": units_per_launch,
                "kernel_share": {k: round(v[0] / sum(x[0] for x in kern.values()), 4) for k, v in
                                 sorted(kern.items(), key=lambda kv: -kv[1][0])[:10]},
                "kernel_frac": {k: round(METHOD_FLOPS[k] * v[2] / (v[0] * 1e-3) / 1e12 / peak, 3)
                                for k, v in kern.items() if k in METHOD_FLOPS and peak}}
    # the whole step: the method's FP64 work of every counted kernel over the device time of
    # every kernel of the profiled steps (ghost fill, restriction and diagnostics count as time only)
    path_flops = sum(METHOD_FLOPS[k] * v[2] for k, v in kern.items() if k in METHOD_FLOPS)
    path_s = sum(v[0] for v in kern.values()) * 1e-3
    roofline["path"] = {"achieved": path_flops / path_s / 1e12, "unit": "TFLOP/s",
                        "frac": (path_flops / path_s / 1e12 / peak) if peak else None,
                        "kernels": sorted(k for k in kern if k in METHOD_FLOPS)}

    # ---- recovery tuples for the learned seed from the migration star's own
    # evolution (FP64 context, 8 times 10 steps apart), before its state is reset
    tuples, ntup, tup_src = None, 0, {}
    if not args.no_learned and not args.no_large:
        tuples = torch.zeros((args.tuples, 10), dtype=torch.float32, device="cuda")
        ntup = collect_tuples(sim, cfg, tuples, 0, 8, 10)
        tup_src[cfg.name] = ntup

    # ---- the same per-kernel breakdown of the mixed-precision step
    if msim is not None:
        if rmx.get("_snap") is not None:
            restore(msim, rmx["_snap"], cfg.dt)
        msim.profile(True)
        for _ in range(prof_steps):
            msim.step_constraints(cfg.dt, 1, use_graph=False)
        mrep = msim.profile_report()
        msim.profile(False)
        mtot = sum(v[0] for v in mrep.values())
        mixed["kernel_share"] = {k: round(v[0] / mtot, 4) for k, v in sorted(mrep.items(), key=lambda kv: -kv[1][0])[:10]}

    # ---- each output's error against the FP64 oracle after one step from the initial data
    if rank == 0 and ws == 1 and not args.no_errors and msim is not None:
        e64, emx = errors_vs_oracle(cfg, datas, [sim, msim], steps=1)
        mixed["err_vs_oracle"] = emx
        mixed["fp64_err_vs_oracle"] = {"rho_l1_rel": e64["rho_l1_rel"],
                                       "max_group_rel": max(e64["max_group_rel"].values()),
                                       "per_field": e64["max_group_rel"]}
    sim.close()
    if msim is not None:
        msim.close()

    # ---- the other workloads, beside the headline
    extra = {}
    if not args.no_extra:
        c2, d2 = workload("tov_stable_3x256")
        s2, a2, m2, b2 = pair_forms(c2, d2, args, dist, ws, 0, 0, args.steps)
        extra["tov_stable_3x256"] = {"config": describe(c2), "fp64": strip(a2), "mixed": strip(b2) if b2 else None}
        if tuples is not None:
            n0 = ntup
            ntup = collect_tuples(s2, c2, tuples, ntup, 10, 20)
            tup_src[c2.name] = ntup - n0
        s2.close()
        if m2 is not None:
            m2.close()
        del d2
    if not args.no_large:
        c5, d5 = workload("large_7x1024")
        s5, a5, m5, b5 = pair_forms(c5, d5, args, dist, ws, 0, 0, args.large_steps)
        if m5 is not None:
            m5.close()
        del d5
        extra["large_7x1024"] = {"config": describe(c5), "fp64": strip(a5), "mixed": strip(b5) if b5 else None}
        if tuples is not None and ntup >= 1000:
            # the learned recovery seed (BF16 MLP) trained by the library's own kernels on the
            # tuples of the smaller runs, tried on every recovery of the large run (kmin = 0)
            t0 = time.perf_counter()
            net, trep, _ = S.mlp_train(tuples[:ntup], steps=3000, batch_blocks=32, lr=1e-2, seed=1, kmin=0.0)
            torch.cuda.synchronize()
            t_train = time.perf_counter() - t0
            del tuples
            tuples = None
            meas = seed_measurement(s5, c5, net, args.large_steps, dist, ws)
            extra["large_7x1024"]["learned_seed"] = {"tuples": ntup, "tuple_sources": tup_src, "train": trep,
                                                     "train_s": t_train, "kmin": 0.0, **meas}
        s5.close()
    batch = None
    if not args.no_batch:
        batch = run_batch(args, dist, ws)

    # ---- CPU oracle on a bounded sample of the headline workload (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        O.set_threads(1)
        c1, t1 = oracle_sample(cfg, datas, 1)
        O.set_threads(0)
        cores = O.get_threads()
        oracle_sample(cfg, datas, 1)              # warm the thread pool
        c, t = oracle_sample(cfg, datas, full_step=True)
        cpu = {"value": c / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "one whole %s step (%d stages with ghost fill, restriction and reflux) of the %s "
                         "hierarchy, OpenMP over %d threads" % ("RK4" if cfg.rk == 0 else "SSP-RK3", cfg.n_stages,
                                                                 cfg.name, cores),
               "single_thread_value": c1 / t1, "single_thread_sample": "one RK stage of the whole hierarchy"}

    if rank == 0:
        conf = describe(cfg)
        conf.update({"parallelism": "replicas" if ws > 1 else "single", "l2": "working set > L2 (no flush)",
                     "cuda_graph": True, "diagnostics_every_step": r64["diagnostics_in_step"]})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": conf,
                "e2e": e2e, "gpu_launches": r64["gpu_launches"], "roofline": roofline, "cpu_baseline": cpu,
                "clocks": r64["clocks"], "repeats": r64.get("repeats"), "tuning": r64["tuning"], "mixed": mixed,
                "extra": extra, "batch": batch}
        if diag is not None and r64["_diag0"] is not None:
            d0 = r64["_diag0"]
            line["diag"] = {"H_L2": diag[0], "Mb": diag[4], "rho_max": diag[6], "Mb_drift": (diag[4] - d0[4]) / d0[4]}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="migration_5x512", choices=WORKLOADS)
    ap.add_argument("--repeats", type=int, default=5, help="further timed regions of the headline (median)")
    ap.add_argument("--repeat-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-errors", action="store_true", help="skip the per-output error report against the oracle")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default launch shapes)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched sweep")
    ap.add_argument("--no-extra", action="store_true", help="skip the stable-star workload")
    ap.add_argument("--no-large", action="store_true", help="skip the 7 x 1024^2 workload")
    ap.add_argument("--fp64-only", action="store_true", help="time the FP64 form only (no mixed contexts)")
    ap.add_argument("--large-steps", type=int, default=6)
    ap.add_argument("--batch-stars", type=int, default=64)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned recovery seed")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--tuples", type=int, default=12_000_000, help="capacity of the learned seed's tuple buffer")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    dist, rank, ws, local = dist_setup()
    try:
        if args.impl == "reference":
            run_reference(args, dist, rank, ws)
        else:
            run_native(args, dist, rank, ws, local)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
