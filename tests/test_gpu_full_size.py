"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the benchmark uses (graph-replayed steps, batched persistent
launches): the unstable-branch migration star (5 levels of 512^2) in FP64 and
in the mixed form, the 64-star sweep (sampled stars against the oracle), and
the large run (7 levels of 1024^2) with the learned recovery seed and
Berger-Oliger sub-cycling from level 5 (the paper's l_fix = 4)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import G, ZERO_BORN, atmosphere_threshold_cells, both, compare_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    O.set_threads(0)


def _rho_l1(gpu_read, orc, cfg):
    num = den = 0.0
    for l in range(cfg.n_levels):
        a = gpu_read(l)[G:G + cfg.nz, G:G + cfg.nx]
        b = orc.read(l, 2, 0)[G:G + cfg.nz, G:G + cfg.nx]
        num += float(np.abs(a - b).sum())
        den += float(np.abs(b).sum())
    return num / den


def _migration():
    cfg, tov = W.config_migration()
    return cfg, [W.tov_level_data(cfg, tov, l, p_deplete=0.99) for l in range(cfg.n_levels)]


def _compare_all(gpu, orc, cfg):
    """Every cell of every level; cells that flipped at the atmosphere
    threshold are checked to be such flips and counted (at most 1 %: the
    coarse levels are almost all atmosphere)."""
    for l in range(cfg.n_levels):
        ex = atmosphere_threshold_cells(gpu, orc, l, cfg.rho_atm)
        assert ex.mean() <= 1e-2, (l, ex.mean())
        compare_level(gpu, orc, l, 1e-11, which=(S.STATE_STEP, S.PRIMS), excuse=ex, floors=ZERO_BORN)


def test_migration_5x512_fp64_one_step_every_cell():
    cfg, datas = _migration()
    gpu, orc = both(cfg, datas)
    gpu.step(cfg.dt, 1, use_graph=True)
    orc.step(cfg.dt, 1)
    _compare_all(gpu, orc, cfg)
    gpu.close()
    orc.close()


def test_migration_5x512_mixed_error_against_the_fp64_oracle():
    cfg, datas = _migration()
    mixed = dataclasses.replace(cfg, precision=7)
    gpu, orc = both(mixed, datas)
    gpu.tune(reps=1)
    for _ in range(3):
        gpu.step(cfg.dt, 1, use_graph=True)
        orc.step(cfg.dt, 1)
    e = _rho_l1(lambda l: gpu.read(l, S.PRIMS, 0), orc, cfg)
    print("migration 5x512^2, mixed, 3 steps: rho L1 against the FP64 oracle %.2e" % e)
    assert e <= 1e-6
    gpu.close()
    orc.close()


def test_batch_sweep_64_full_size_sampled_stars():
    """All 64 stars advance together (mixed precision, autotuned, graph); three
    stars, the largest and two drawn at random, are compared with the FP64
    oracle run alone."""
    stars = W.config_batch_sweep(n_stars=64)
    cfgs = [c for c, _ in stars]
    dt = min(c.dt for c in cfgs)
    b = S.SacraBatch(cfgs)
    dep = lambda tov: 0.99 if tov.rho_c > 3.2e-3 else 1.0
    for i, (c, tov) in enumerate(stars):
        for l in range(c.n_levels):
            b.set_initial_data(i, l, S.PRIM_METRIC, W.tov_level_data(c, tov, l, p_deplete=dep(tov)))
    b.tune(reps=1)
    b.step(dt, 2, use_graph=True)
    largest = max(range(64), key=lambda i: cfgs[i].interior_cells)
    others = [i for i in range(64) if i != largest]
    picks = [largest] + [int(i) for i in np.random.default_rng(20250203).choice(others, 2, replace=False)]
    for i in picks:
        c, tov = stars[i]
        orc = O.Oracle(dataclasses.replace(c, precision=0))
        for l in range(c.n_levels):
            orc.set_level(l, 0, W.tov_level_data(c, tov, l, p_deplete=dep(tov)))
        orc.step(dt, 2)
        e = _rho_l1(lambda l: b.read(i, l, S.PRIMS, 0), orc, c)
        print("sweep star %d (%d levels of %d^2): rho L1 against the FP64 oracle %.2e" % (i, c.n_levels, c.nx, e))
        assert e <= 1e-6
        orc.close()
    b.close()


def test_large_7x1024_learned_seed_subcycled_one_step_every_cell():
    """The config-3 star at 7 levels of 1024^2 with levels 5 and 6 sub-cycled
    and the learned recovery seed (trained on tuples of a smaller run of the
    same star): one coarse step, every cell against the oracle (which has no
    seed: the seeded recovery must land on the plain one's primitives)."""
    import torch
    cfg, tov = W.config_migration(N=1024, n_levels=7)
    cfg = dataclasses.replace(cfg, subcycle_from=5)
    small, stov = W.config_migration(N=128, n_levels=3)
    sim = S.Sacra(small)
    for l in range(small.n_levels):
        sim.set_initial_data(l, S.PRIM_METRIC, W.tov_level_data(small, stov, l, p_deplete=0.99))
    buf = torch.zeros((400000, 10), dtype=torch.float32, device="cuda")
    parts = []
    for _ in range(6):
        sim.step(small.dt, 3)
        n = sim.mlp_collect(buf)
        parts.append(buf[:n].clone())
    sim.close()
    net, rep, _ = S.mlp_train(torch.cat(parts), steps=3000, batch_blocks=16, lr=1e-2, seed=3, kmin=0.0)
    datas = [W.tov_level_data(cfg, tov, l, p_deplete=0.99) for l in range(cfg.n_levels)]
    gpu, orc = both(cfg, datas)
    del datas
    gpu.set_mlp(net)
    gpu.c2p_counting(True)
    gpu.step(cfg.dt, 1, use_graph=True)
    orc.step(cfg.dt, 1)
    ev, tried, held, nrec = gpu.c2p_counts()
    print("7x1024^2 sub-cycled, learned seed: tried %d, held %d of %d recoveries, %.2f evaluations each"
          % (tried, held, nrec, ev / max(nrec, 1)))
    assert tried > 0
    _compare_all(gpu, orc, cfg)
    gpu.close()
    orc.close()
