#!/usr/bin/env python3
"""Throughput of the SACRA-2D hot path on GB300: cell-updates per second per
RK stage of Z4c + HLLC GRHD on the fixed-mesh-refinement cartoon grid.

Workload (default): the stable TOV star (K=100, Gamma=2, rho_c=1.28e-3,
Gamma_th=2, atmosphere 1e-10 of rho_c), equatorial symmetry, 3 FMR levels of
256^2 cells, finest dx = 0.25, SSP-RK3, FP64.  One step = the whole hot path:
ghost fill / prolongation, hydro and Z4c right-hand sides, RK combination with
algebraic constraints and primitive recovery for every stage, then
restriction + reflux; the constraint and conservation diagnostics of the state
at the start of each step are formed inside its first stage (from that stage's
derivative pass) and read back to the host every step.  The working set (about
0.7 GB of FP64 state per step) exceeds the 129 MB L2, so no flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank advances its own replica (the path has no exchange
step on one level set; weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import ctypes
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

# Algorithmic FLOPs per unit of work, counted on the oracle's plain
# restatement with its op-counting build (oracle/opcount.cpp), benchmark
# workload, one RK stage.  Unit: a cell of the update region, a face for the
# flux kernels, a cell of the plane patch for the cartoon kernel.
ALG_FLOPS = {
    "k_flux_x": 1071.2, "k_flux_z": 1071.2, "k_hydro_rhs": 1383.2, "k_cartoon": 3481.0,
    "k_z4c_derivs": 5296.0, "k_z4c_point": 4197.0, "k_rk_update": 576.7,
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

def workload(name):
    from paper_2502_03223_gb300 import workloads as W
    if name == "tov_stable_3x256":
        cfg, tov = W.config_tov_stable()
        return cfg, [W.tov_level_data(cfg, tov, l) for l in range(cfg.n_levels)]
    if name == "migration_5x512":
        cfg, tov = W.config_migration()
        return cfg, [W.tov_level_data(cfg, tov, l, p_deplete=0.99) for l in range(cfg.n_levels)]
    if name == "shock_tube_400x4":
        cfg = W.config_shock_tube()
        return cfg, [W.shock_tube_data(cfg)]
    raise SystemExit("unknown workload " + name)


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


def read_traffic():
    """DRAM bytes per launch of a kernel from the committed ncu summary
    (profiles/traffic_tov_stable_3x256.txt), kept only if the kernel's sources
    still hash to the recorded value (else the counters are stale)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_tov_stable_3x256.txt")
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


# ---------------------------------------------------------------- arms

def oracle_sample(cfg, datas, stages=1):
    """Time `stages` RK stages (ghost fill + stage) of the whole hierarchy on
    the CPU oracle (single thread).  Returns (cell-updates, seconds)."""
    import oracle as O
    o = O.Oracle(cfg)
    for l, d in enumerate(datas):
        o.set_level(l, 0, d)
    t0 = time.perf_counter()
    for s in range(stages):
        o.fill(s % cfg.n_stages, cfg.dt)
        o.stage(s % cfg.n_stages, cfg.dt)
    el = time.perf_counter() - t0
    o.close()
    return cfg.interior_cells * stages, el


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
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "levels": cfg.n_levels, "cells_per_level": [cfg.nx, cfg.nz],
                       "integrator": "SSP-RK3" if cfg.rk else "RK4", "reference": "CPU oracle (plain FP64 C)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: one RK stage (ghost fill + stage) of the whole %s hierarchy, "
                                       "OpenMP over %d threads" % (cfg.name, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(sim, dt, steps, dist):
    """K graph-replayed steps, each with the diagnostics of its starting state
    read back, bracketed by a barrier and a device synchronize, timed by CUDA
    events on the library's stream.  Returns (ms, launches, last diagnostics,
    clocks)."""
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
    for _ in range(steps):
        diag = sim.step_constraints(dt, 1, use_graph=True)[0]
    ev1.record(sim.stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    return ev0.elapsed_time(ev1), sim.launch_count - n0, diag, clocks


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
    cells = sum(c.interior_cells * c.n_stages for c in cfgs)
    if learned is not None:
        learned["value"] = ws * cells * steps / (learned["ms_per_step"] * steps * 1e-3)
        learned["unit"] = UNIT
    diag = b.constraints(0)
    b.close()
    return {"workload": "batch_sweep_%d" % len(cfgs), "value": ws * cells * steps / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / steps, "steps": steps, "n_stars": len(cfgs),
            "cell_updates_per_step": cells, "precision": "mixed", "cuda_graph": True, "tuning": tuning,
            "gpu_launches": launches, "clocks": clocks, "init_s": t_init, "learned_seed": learned,
            "star0_H_L2": diag[0], "sizes": sorted(set((c.nx, c.n_levels) for c in cfgs))[:40]}


def run_native(args, dist, rank, ws, local):
    import dataclasses
    import torch
    from paper_2502_03223_gb300 import build as B
    B.build()
    from paper_2502_03223_gb300 import sacra2d as S
    torch.cuda.set_device(local)
    cfg, datas = workload(args.workload)
    sim = S.Sacra(cfg)
    for l, d in enumerate(datas):
        sim.set_initial_data(l, S.PRIM_METRIC, d)
    dt = cfg.dt
    cells_per_step = cfg.interior_cells * cfg.n_stages

    def one_step(graph=True):
        return sim.step_constraints(dt, 1, use_graph=graph)[0]

    for _ in range(args.warmup):
        one_step()
    sim.sync()
    tuning = sim.tune(reps=4) if not args.no_tune else None   # autotuner, outside the timed region
    for _ in range(2):
        one_step()
    sim.sync()
    diag0 = sim.constraints()

    # ---- timed region (device time, CUDA events on the library's stream)
    ms, launches, diag_in, clocks = timed_steps(sim, dt, args.steps, dist)
    diag = sim.constraints()          # the state after the last step (untimed)
    ms_max = max_over_ranks(dist, ms)
    value = ws * cells_per_step * args.steps / (ms_max * 1e-3)

    # ---- the mixed-precision form of the same step, timed the same way
    mcfg = dataclasses.replace(cfg, precision=S.MIXED)
    msim = S.Sacra(mcfg)
    for l, d in enumerate(datas):
        msim.set_initial_data(l, S.PRIM_METRIC, d)
    for _ in range(args.warmup):
        msim.step_constraints(dt, 1, use_graph=True)
    msim.sync()
    mtuning = msim.tune(reps=4) if not args.no_tune else None
    for _ in range(2):
        msim.step_constraints(dt, 1, use_graph=True)
    msim.sync()
    mms, mlaunches, mdiag_in, mclocks = timed_steps(msim, dt, args.steps, dist)
    mms_max = max_over_ranks(dist, mms)
    mvalue = ws * cells_per_step * args.steps / (mms_max * 1e-3)
    mixed = {"value": mvalue, "unit": UNIT, "ms_per_step": mms_max / args.steps, "speedup_vs_fp64": mvalue / value,
             "gpu_launches": mlaunches, "clocks": mclocks, "tuning": mtuning,
             # ||H|| of the same starting state of the last timed step, formed in the step
             # (mixed: from the FP32 Ricci scalar of its pointwise pass)
             "H_L2_in_step": {"mixed": mdiag_in[0], "fp64": diag_in[0],
                              "rel_diff": abs(mdiag_in[0] - diag_in[0]) / diag_in[0]},
             "arith": "FP32 reconstruction, Riemann solver, hydro sources and Z4c algebra; FP64 finite "
                      "differences, primitive recovery, algebraic constraints, RK and flux accumulation"}

    # ---- the batched sweep (independent stars of mixed sizes in one set of
    # persistent launches per stage), mixed precision, one graph per step
    batch = None
    if not args.no_batch:
        batch = run_batch(args, dist, ws)

    # ---- end to end through the C ABI with host buffers: every step the state
    # of all levels goes host -> device from pinned memory (set_initial_data, RAW),
    # one step runs, and the diagnostics come back to the host
    host = []
    for l in range(cfg.n_levels):
        buf = torch.empty(30 * sim.px * sim.pz, dtype=torch.float64, pin_memory=True)
        a = buf.numpy()
        for f in range(30):
            a[f * sim.px * sim.pz:(f + 1) * sim.px * sim.pz] = sim.read(l, S.STATE_STEP, f).ravel()
        host.append(a)
    e2e_steps = max(3, min(args.steps, 20))
    h2d = sum(a.nbytes for a in host)
    d2h = ctypes.sizeof(S.SacraDiag)
    sim.sync()
    barrier(dist)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for l in range(cfg.n_levels):
            sim.set_initial_data(l, S.RAW, host[l])
        one_step()
    el = time.perf_counter() - t0
    el = max_over_ranks(dist, el)
    e2e = ws * cells_per_step * e2e_steps / el

    # ---- per-kernel device time (eager launches bracketed by CUDA events)
    sim.profile(True)
    prof_steps = max(2, min(args.steps, 10))
    for _ in range(prof_steps):
        one_step(graph=False)
    rep = sim.profile_report()
    sim.profile(False)
    kern = {k: v for k, v in rep.items()}
    dom = max((k for k in kern if k in ALG_FLOPS), key=lambda k: kern[k][0])
    tot_ms, n_launch, n_cells = kern[dom]
    avg_s = tot_ms * 1e-3 / n_launch
    units_per_launch = n_cells / n_launch
    if dom == "k_flux_x":
        units_per_launch = n_cells / n_launch * 1.0   # faces ~ cells of the region
    achieved = ALG_FLOPS[dom] * units_per_launch / avg_s / 1e12
    peak = fp64_peak()
    traffic = read_traffic().get(dom)
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if peak else None,
                "traffic": (traffic[0] / traffic[1] * units_per_launch) if traffic else None,
                "peak_source": "FP64 FMA probe measured in this run (nominal %.2f TFLOP/s)" % NOMINAL_FP64_TFLOPS,
                "alg_flops_per_unit": ALG_FLOPS[dom], "avg_launch_ms": avg_s * 1e3,
                "units_per_launch": units_per_launch,
                "kernel_share": {k: round(v[0] / sum(x[0] for x in kern.values()), 4) for k, v in
                                 sorted(kern.items(), key=lambda kv: -kv[1][0])[:8]}}
    # the whole step: the algorithmic FP64 work of every counted kernel over the device time of
    # every kernel of the profiled steps (ghost fill, restriction and diagnostics count as time only)
    path_flops = sum(ALG_FLOPS[k] * v[2] for k, v in kern.items() if k in ALG_FLOPS)
    path_s = sum(v[0] for v in kern.values()) * 1e-3
    roofline["path"] = {"achieved": path_flops / path_s / 1e12, "unit": "TFLOP/s",
                        "frac": (path_flops / path_s / 1e12 / peak) if peak else None,
                        "kernels": sorted(k for k in kern if k in ALG_FLOPS)}

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        O.set_threads(1)
        c1, t1 = oracle_sample(cfg, datas, 1)
        O.set_threads(0)
        cores = O.get_threads()
        oracle_sample(cfg, datas, 1)              # warm the thread pool
        c, t = oracle_sample(cfg, datas, 3)
        cpu = {"value": c / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "one SSP-RK3 step (3 x ghost fill + stage) of the whole %s hierarchy, OpenMP over %d "
                         "threads" % (cfg.name, cores),
               "single_thread_value": c1 / t1}
        if not args.no_errors:
            # each output's error against the FP64 oracle after one step from the initial data
            e64, emx = errors_vs_oracle(cfg, datas, [sim, msim], steps=1)
            mixed["err_vs_oracle"] = emx
            mixed["fp64_err_vs_oracle"] = {"rho_l1_rel": e64["rho_l1_rel"],
                                           "max_group_rel": max(e64["max_group_rel"].values())}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": cfg.name, "levels": cfg.n_levels, "cells_per_level": [cfg.nx, cfg.nz],
                           "finest_dx": cfg.dx(cfg.n_levels - 1), "integrator": "SSP-RK3" if cfg.rk else "RK4",
                           "stages_per_step": cfg.n_stages, "cell_updates_per_step": cells_per_step,
                           "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "working set > L2 (no flush)", "cuda_graph": True},
                "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
                "mixed": mixed, "batch": batch, "tuning": tuning,
                "diag": {"H_L2": diag[0], "Mb": diag[4], "rho_max": diag[6], "Mb_drift": (diag[4] - diag0[4]) / diag0[4]}}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="tov_stable_3x256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-errors", action="store_true", help="skip the per-output error report against the oracle")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default launch shapes)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched sweep")
    ap.add_argument("--batch-stars", type=int, default=64)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned recovery seed")
    ap.add_argument("--batch-steps", type=int, default=5)
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
