"""Batched execution: many independent stars of different grid sizes and
level counts advanced together (one persistent launch per kernel kind and RK
stage over all of them), and the autotuner of those launches.  A star in a
batch must evolve bit for bit as it does alone (the same per-cell arithmetic
in the same order), in FP64 and in the mixed form, with and without graphs;
tuning must not change the state."""
import dataclasses

import numpy as np
import pytest

from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


def _stars(precision=0):
    specs = [(1.28e-3, 2, 32, 0.5), (3.0e-3, 1, 48, 0.5), (6.0e-3, 3, 32, 0.5), (2.0e-3, 2, 40, 0.5)]
    out = []
    for i, (rc, L, N, dxf) in enumerate(specs):
        cfg, tov = W.tov_config("b%d" % i, rho_c=rc, n_levels=L, N=N, dx_fine=dxf, rk=1)
        cfg = dataclasses.replace(cfg, precision=precision)
        out.append((cfg, [W.tov_level_data(cfg, tov, l) for l in range(L)]))
    return out


def _same(a, b):
    return a.shape == b.shape and np.array_equal(a, b)


@pytest.mark.parametrize("precision,use_graph", [(0, False), (0, True), (7, True)])
def test_batch_matches_each_star_alone(precision, use_graph):
    stars = _stars(precision)
    dt = min(c.dt for c, _ in stars)
    batch = S.SacraBatch([c for c, _ in stars])
    for i, (c, ds) in enumerate(stars):
        for l, d in enumerate(ds):
            batch.set_initial_data(i, l, S.PRIM_METRIC, d)
    batch.step(dt, 4, use_graph=use_graph)
    for i, (c, ds) in enumerate(stars):
        alone = S.Sacra(c)
        for l, d in enumerate(ds):
            alone.set_initial_data(l, S.PRIM_METRIC, d)
        alone.step(dt, 4, use_graph=use_graph)
        for l in range(c.n_levels):
            for f in range(30):
                assert _same(batch.read(i, l, S.STATE_STEP, f), alone.read(l, S.STATE_STEP, f)), (i, l, f)
            for f in range(6):
                assert _same(batch.read(i, l, S.PRIMS, f), alone.read(l, S.PRIMS, f)), (i, l, f)
        assert np.array_equal(batch.constraints(i)[:7], alone.constraints()[:7])
        alone.close()


def test_tuning_keeps_the_state_and_picks_valid_shapes():
    cfg, tov = W.tov_config("t", rho_c=1.28e-3, n_levels=2, N=32, dx_fine=0.5, rk=1)
    datas = [W.tov_level_data(cfg, tov, l) for l in range(2)]
    a, b = S.Sacra(cfg), S.Sacra(cfg)
    for l, d in enumerate(datas):
        a.set_initial_data(l, S.PRIM_METRIC, d)
        b.set_initial_data(l, S.PRIM_METRIC, d)
    a.step(cfg.dt, 1)
    b.step(cfg.dt, 1)
    n0 = a.constraints()[8]
    picks = a.tune(reps=1)
    for name, (tx, ty, m) in picks.items():
        assert tx * ty in (128, 256) and m >= 1, (name, tx, ty, m)
    assert a.constraints()[8] == n0          # the fallback counter is restored
    a.step(cfg.dt, 3, use_graph=True)
    b.step(cfg.dt, 3, use_graph=True)
    for l in range(2):
        for f in range(30):
            assert _same(a.read(l, S.STATE_STEP, f), b.read(l, S.STATE_STEP, f)), (l, f)


def test_pinned_shapes_give_the_same_state_mixed():
    """Launch shapes change no value, in the mixed form too, where they also
    decide which FP32 face kernel runs: z-faces on 64 x 4 tiles would need a
    65 KB staging buffer and take the per-face form; the others stage their
    FP32 inputs in shared memory."""
    cfg, tov = W.tov_config("pin", rho_c=1.28e-3, n_levels=2, N=48, dx_fine=0.5, rk=1)
    cfg = dataclasses.replace(cfg, precision=7)
    datas = [W.tov_level_data(cfg, tov, l) for l in range(2)]
    runs = []
    for pins in ({}, {"flux_x": (64, 4, 3), "flux_z": (64, 4, 3), "cartoon": (128, 1, 2), "hydro_rhs": (16, 8, 6),
                      "z4c_point": (64, 2, 4), "rk_update": (128, 1, 1)}):
        sim = S.Sacra(cfg)
        for l, d in enumerate(datas):
            sim.set_initial_data(l, S.PRIM_METRIC, d)
        for kind, (tx, ty, m) in pins.items():
            sim.set_tuning(kind, tx, ty, m)
            assert sim.tuning()[kind] == (tx, ty, m)
        sim.step(cfg.dt, 3, use_graph=True)
        runs.append(sim)
    for l in range(2):
        for f in range(30):
            assert _same(runs[0].read(l, S.STATE_STEP, f), runs[1].read(l, S.STATE_STEP, f)), (l, f)
        for f in range(6):
            assert _same(runs[0].read(l, S.PRIMS, f), runs[1].read(l, S.PRIMS, f)), (l, f)
    with pytest.raises(S.SacraError):
        runs[0].set_tuning("rk_update", 32, 8, 4)       # 256 threads: beyond the kernel's launch bounds
    with pytest.raises(S.SacraError):
        runs[0].set_tuning("flux_x", 32, 4, 5)          # not a candidate grid size
    for r in runs:
        r.close()


def test_batch_tuning_then_graph_steps_match_untuned():
    stars = _stars(7)
    dt = min(c.dt for c, _ in stars)
    runs = []
    for tuned in (False, True):
        batch = S.SacraBatch([c for c, _ in stars])
        for i, (c, ds) in enumerate(stars):
            for l, d in enumerate(ds):
                batch.set_initial_data(i, l, S.PRIM_METRIC, d)
        if tuned:
            batch.tune(reps=1)
        batch.step(dt, 3, use_graph=True)
        runs.append(batch)
    for i, (c, _) in enumerate(stars):
        for l in range(c.n_levels):
            for f in range(30):
                assert _same(runs[0].read(i, l, S.STATE_STEP, f), runs[1].read(i, l, S.STATE_STEP, f)), (i, l, f)


def test_incompatible_stars_are_rejected():
    a, _ = W.tov_config("a", n_levels=1, N=32, dx_fine=0.5, rk=1)
    b, _ = W.tov_config("b", n_levels=1, N=32, dx_fine=0.5, rk=0)      # another integrator
    with pytest.raises(S.SacraError):
        S.SacraBatch([a, b])


def test_batch_mixes_bssn_and_z4c_stars():
    """The formulation is a per-star parameter: a batch holding BSSN and Z4c
    stars advances each exactly as its own context does (Theta stays zero in
    the BSSN stars only)."""
    stars = [(dataclasses.replace(c, bssn=i % 2), ds) for i, (c, ds) in enumerate(_stars(0))]
    dt = min(c.dt for c, _ in stars)
    batch = S.SacraBatch([c for c, _ in stars])
    for i, (c, ds) in enumerate(stars):
        for l, d in enumerate(ds):
            batch.set_initial_data(i, l, S.PRIM_METRIC, d)
    batch.step(dt, 3, use_graph=True)
    for i, (c, ds) in enumerate(stars):
        alone = S.Sacra(c)
        for l, d in enumerate(ds):
            alone.set_initial_data(l, S.PRIM_METRIC, d)
        alone.step(dt, 3, use_graph=True)
        for l in range(c.n_levels):
            for f in range(30):
                assert _same(batch.read(i, l, S.STATE_STEP, f), alone.read(l, S.STATE_STEP, f)), (i, l, f)
        theta = batch.read(i, 0, S.STATE_STEP, 17)
        assert (not np.any(theta)) if c.bssn else np.any(theta), i
        alone.close()
