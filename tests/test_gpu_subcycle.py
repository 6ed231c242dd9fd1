"""Berger-Oliger sub-cycling on the GPU (Sec. II.D): levels >= K take half
their parent's step, with the parent's data interpolated in time for the
child's buffer zone and the reflux weighted by the child's share of the
parent's step.  The CUDA path against the oracle after every coarse step (the
same per-cell criterion as the lockstep parity tests), rest-mass conservation,
graph replay, and the calls a sub-cycled context refuses."""
import dataclasses

import numpy as np
import pytest

from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import G, both, compare_level, compare_status

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


def _tov(L, K, rk, N=32, dx_fine=0.5, seed=0):
    cfg, tov = W.tov_config("tov_sub", rho_c=1.28e-3, n_levels=L, N=N, dx_fine=dx_fine, rk=rk)
    cfg = dataclasses.replace(cfg, subcycle_from=K)
    datas = []
    for l in range(L):
        d = W.tov_level_data(cfg, tov, l)
        d[:25] += W.random_metric_perturbation(cfg, l, np.random.default_rng(seed + 100), amp=1e-3)
        X, Z = W.cell_centres(cfg, l)
        bump = np.exp(-((X - 3.0) ** 2 + (Z - 2.0) ** 2) / 4.0)
        d[26] = 0.05 * bump * X / (np.abs(X) + 1.0)
        d[27] = 0.03 * bump * X / (np.abs(X) + 1.0)
        datas.append(d)
    return cfg, datas


def _blob(L, K, rk, N=48):
    """A frozen-metric flat-space blob crossing the refinement boundaries."""
    cfg = W.RunConfig(n_levels=L, nx=N, nz=N, geometry=1, evolve_spacetime=0, dx0=0.5, dz0=0.5,
                      K=100.0, Gamma=2.0, Gamma_th=2.0, rho_atm=1e-14, rk=rk, subcycle_from=K)
    datas = []
    for l in range(L):
        X, Z = W.cell_centres(cfg, l)
        d = np.zeros((30,) + X.shape)
        d[:25] = W.flat_metric(cfg)
        r2 = ((X - 9.0) ** 2 + (Z - 8.0) ** 2) / 9.0
        bump = np.where(r2 < 1.0, (1.0 - r2) ** 3, 0.0)
        d[25] = 1e-3 * (1.0 + 2.0 * bump)
        d[29] = 100 * d[25] ** 2 * 1.5
        d[26] = 0.3 * bump
        d[28] = 0.2 * bump
        datas.append(d)
    return cfg, datas


@pytest.mark.parametrize("L,K,rk", [(2, 1, 0), (3, 1, 0), (3, 2, 1)])
def test_subcycled_tov_matches_oracle_every_step(L, K, rk):
    cfg, datas = _tov(L, K, rk)
    gpu, orc = both(cfg, datas)
    worst = 0.0
    for _ in range(3):
        gpu.step(cfg.dt, 1)
        orc.step(cfg.dt, 1)
        for l in range(L):
            worst = max(worst, compare_level(gpu, orc, l, 1e-11, which=(S.STATE_STEP, S.PRIMS)))
            compare_status(gpu, orc, l)
    assert worst < 1e-11


def test_subcycled_blob_conserves_mass_and_matches_oracle():
    cfg, datas = _blob(3, 1, 0)
    gpu, orc = both(cfg, datas)
    m0 = gpu.constraints()[4]
    gpu.step(cfg.dt, 4)
    orc.step(cfg.dt, 4)
    m1 = gpu.constraints()[4]
    assert abs(m1 - m0) / m0 < 1e-13, (m0, m1)
    for l in range(3):
        a = gpu.read(l, S.PRIMS, 0)[G:G + 48, G:G + 48]
        b = orc.read(l, 2, 0)[G:G + 48, G:G + 48]
        assert np.abs(a - b).sum() / np.abs(b).sum() < 1e-12, l


def test_subcycled_graph_replay_matches_eager():
    """The first step runs eagerly (no t^{n-1} slice yet); later steps replay
    one captured coarse step."""
    cfg, datas = _tov(3, 1, 1)
    a, b = S.Sacra(cfg), S.Sacra(cfg)
    for l, d in enumerate(datas):
        a.set_initial_data(l, S.PRIM_METRIC, d)
        b.set_initial_data(l, S.PRIM_METRIC, d)
    a.step(cfg.dt, 4, use_graph=False)
    b.step(cfg.dt, 4, use_graph=True)
    for l in range(3):
        for f in range(30):
            assert np.array_equal(a.read(l, S.STATE_STEP, f), b.read(l, S.STATE_STEP, f)), (l, f)
        for f in range(6):
            assert np.array_equal(a.read(l, S.PRIMS, f), b.read(l, S.PRIMS, f)), (l, f)


def test_lockstep_setting_is_the_lockstep_run():
    """K >= n_levels is lockstep: the same launches and results as K = 0."""
    cfg, datas = _tov(2, 0, 1)
    cfg_k = dataclasses.replace(cfg, subcycle_from=2)
    a, b = S.Sacra(cfg), S.Sacra(cfg_k)
    for l, d in enumerate(datas):
        a.set_initial_data(l, S.PRIM_METRIC, d)
        b.set_initial_data(l, S.PRIM_METRIC, d)
    a.step(cfg.dt, 2)
    b.step(cfg.dt, 2)
    for l in range(2):
        for f in range(30):
            assert np.array_equal(a.read(l, S.STATE_STEP, f), b.read(l, S.STATE_STEP, f)), (l, f)


def test_subcycled_context_refuses_stagewise_calls_and_batches():
    cfg, datas = _tov(2, 1, 1)
    s = S.Sacra(cfg)
    for l, d in enumerate(datas):
        s.set_initial_data(l, S.PRIM_METRIC, d)
    with pytest.raises(S.SacraError):
        s.fill(0, cfg.dt)
    with pytest.raises(S.SacraError):
        s.rk_stage(0, cfg.dt)
    with pytest.raises(S.SacraError):
        S.SacraBatch([cfg, cfg])
