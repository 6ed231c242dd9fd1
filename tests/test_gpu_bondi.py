"""Bondi accretion onto the trumpet black hole in Cowling mode (Sec. III):
the CUDA path against the oracle step by step (uniform grid, both Riemann
solvers; three FMR levels, lockstep and sub-cycled), and the paper's
convergence study of eps_L1(rho) at t = 20M on the GPU."""
import math

import numpy as np
import pytest

from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from bondi_common import bondi_l1
from gpu_common import both, compare_level, compare_status

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


def _data(cfg, sol):
    return [W.bondi_level_data(cfg, sol, l) for l in range(cfg.n_levels)]


@pytest.mark.parametrize("N,solver,levels,K", [(64, 0, 1, 0), (64, 1, 1, 0), (32, 0, 3, 0), (32, 0, 3, 1)])
def test_bondi_matches_oracle_every_step(N, solver, levels, K):
    import dataclasses
    cfg, sol = W.bondi_config(N=N, solver=solver, n_levels=levels)
    cfg = dataclasses.replace(cfg, subcycle_from=K)
    gpu, orc = both(cfg, _data(cfg, sol))
    worst = 0.0
    for _ in range(3):
        gpu.step(cfg.dt, 1)
        orc.step(cfg.dt, 1)
        for l in range(levels):
            worst = max(worst, compare_level(gpu, orc, l, 1e-11, which=(S.STATE_STEP, S.PRIMS)))
            compare_status(gpu, orc, l)
    assert worst < 1e-11


def _evolve(N, T, solver=0, levels=1, K=0):
    import dataclasses
    cfg, sol = W.bondi_config(N=N, solver=solver, n_levels=levels)
    cfg = dataclasses.replace(cfg, subcycle_from=K)
    datas = _data(cfg, sol)
    s = S.Sacra(cfg)
    for l, d in enumerate(datas):
        s.set_initial_data(l, S.PRIM_METRIC, d)
    s.step(cfg.dt, int(round(T / cfg.dt)), use_graph=True)
    return cfg, datas, s


def _l1_at(N, T, solver=0, levels=1, K=0):
    cfg, datas, s = _evolve(N, T, solver, levels, K)
    e = bondi_l1(cfg, datas, lambda l: s.read(l, S.PRIMS, 0))
    s.close()
    return e


@pytest.mark.parametrize("solver,levels,K", [(0, 1, 0), (1, 1, 0), (0, 3, 0), (0, 3, 1)])
def test_bondi_convergence_on_the_gpu(solver, levels, K):
    """eps_L1(rho) at t = 20M for N = 32 .. 256 (the paper's study; with three
    levels N is per level and the finest box is 4M) falls at every doubling.
    The measured order is about 1 at this time (the paper reports about 2):
    the error is dominated by an odd-even mode that starts at the staircase
    edge of the held region r < 0.4M and spreads upstream; PPM in
    method-of-lines form does not damp it in smooth monotone flow (see the
    oracle's test_smooth_monotone_flow_has_no_numerical_dissipation and
    test_bondi_smooth_error_is_second_order)."""
    Ns = (32, 64, 128, 256)
    errs = [_l1_at(N, 20.0, solver, levels, K) for N in Ns]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(Ns) - 1)]
    print("Bondi solver %d levels %d K %d: eps_L1(t=20M) %s orders %s" % (solver, levels, K,
          ["%.3e" % e for e in errs], ["%.2f" % o for o in orders]))
    assert errs[-1] < 2e-3
    assert all(o > 0.6 for o in orders), (errs, orders)


def test_bondi_smooth_error_is_second_order():
    """The error averaged over 0.5M x 0.5M blocks (which removes the
    grid-scale noise) between r = 2M and 12M converges at second order at
    t = 5M for N = 128, 256, 512."""
    G = 8
    vals = []
    for N in (128, 256, 512):
        cfg, datas, s = _evolve(N, 5.0)
        sl = (slice(G, G + N), slice(G, G + N))
        e = s.read(0, S.PRIMS, 0)[sl] - datas[0][25][sl]
        s.close()
        X, Z = W.cell_centres(cfg, 0)
        X, Z = X[sl], Z[sl]
        r = np.sqrt(X * X + Z * Z)
        f = N // 32                                   # cells per 0.5M block
        blk = lambda a: a.reshape(32, f, 32, f).mean(axis=(1, 3))
        m = blk(((r > 2.0) & (r < 12.0)).astype(float)) > 0.999
        vals.append(float(np.sum(np.abs(blk(e)) * blk(X) * m)))
    orders = [math.log2(vals[i] / vals[i + 1]) for i in range(2)]
    print("Bondi block-averaged error at t = 5M:", vals, "orders", orders)
    assert min(orders) > 1.8, (vals, orders)
