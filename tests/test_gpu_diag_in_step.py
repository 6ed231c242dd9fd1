"""Diagnostics formed inside the first RK stage of each step (Sec. II.F.1):
sacra_step_constraints reports, for every step, the constraint norms, rest
mass, angular momentum and maximum density of the state at the start of that
step, computed from the derivatives the stage's own Z4c pass has just formed.
They must equal sacra_constraints called just before the step (which runs its
own ghost fill, cartoon and derivative passes), leave the evolution untouched,
and agree with the oracle's diagnostics of the same state."""
import dataclasses

import numpy as np
import pytest

from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import both

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


def _tov(rk, L=3, N=32, precision=S.FP64, seed=0):
    cfg, tov = W.tov_config("tov_diag", rho_c=1.28e-3, n_levels=L, N=N, dx_fine=0.5, rk=rk)
    cfg = dataclasses.replace(cfg, precision=precision)
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


def _pair(cfg, datas):
    a, b = S.Sacra(cfg), S.Sacra(cfg)
    for l, d in enumerate(datas):
        a.set_initial_data(l, S.PRIM_METRIC, d)
        b.set_initial_data(l, S.PRIM_METRIC, d)
    return a, b


def _separate(sim, dt, n, use_graph):
    rows = []
    for _ in range(n):
        rows.append(sim.constraints())
        sim.step(dt, 1, use_graph=use_graph)
    return np.array(rows)


@pytest.mark.parametrize("rk,use_graph", [(0, False), (1, True)])
def test_in_step_diagnostics_equal_separate_calls_fp64(rk, use_graph):
    cfg, datas = _tov(rk)
    a, b = _pair(cfg, datas)
    n = 4
    la0 = a.launch_count
    ref = _separate(a, cfg.dt, n, use_graph)
    la = a.launch_count - la0
    lb0 = b.launch_count
    got = b.step_constraints(cfg.dt, n, use_graph=use_graph)
    lb = b.launch_count - lb0
    assert got.shape == (n, 9)
    # rest mass, angular momentum, rho_max and the recovery failures need no
    # derivatives: same cells, same fixed-order sums
    assert np.array_equal(got[:, 4:8], ref[:, 4:8]), (got[:, 4:8] - ref[:, 4:8])
    # the fallback counter is read after step i: the separate call's before step i + 1
    assert np.array_equal(got[:-1, 8], ref[1:, 8]), (got[:, 8], ref[:, 8])
    # the momentum-constraint norms come from the stage's batched derivative
    # pass instead of the per-level one; both run the same cell function
    assert np.allclose(got[:, 1:4], ref[:, 1:4], rtol=1e-13, atol=0.0), (got[:, 1:4] - ref[:, 1:4])
    # ||H|| takes the Ricci scalar the stage's FP64 pointwise pass has formed
    # (same function, another kernel, so possibly another contraction of
    # multiply-adds): H cancels terms of order 0.1, so a rounding of 1e-17 in
    # R moves ||H|| (here ~1e-3) by ~1e-14 relative
    assert np.allclose(got[:, 0], ref[:, 0], rtol=1e-10, atol=0.0), (got[:, 0] - ref[:, 0])
    # the evolution is untouched
    for l in range(cfg.n_levels):
        for f in range(30):
            assert np.array_equal(a.read(l, S.STATE_STEP, f), b.read(l, S.STATE_STEP, f)), (l, f)
    # and the cartoon/derivative passes and ghost fills of the separate calls are gone
    assert lb < la, (lb, la)


def test_in_step_diagnostics_match_oracle_at_step_start():
    cfg, datas = _tov(1)
    gpu, orc = both(cfg, datas)
    got = gpu.step_constraints(cfg.dt, 2, use_graph=False)
    do = orc.diag()                       # the initial state = the start of step 0
    assert abs(got[0, 4] - do[4]) < 1e-12 * do[4]          # rest mass
    assert abs(got[0, 0] - do[0]) < 1e-8 * do[0]           # ||H||
    assert np.allclose(got[0, 1:4], do[1:4], rtol=1e-7, atol=1e-14)
    assert got[0, 6] == pytest.approx(do[6], rel=1e-12)    # rho_max
    orc.step(cfg.dt, 1)
    do1 = orc.diag()                      # the start of step 1
    assert abs(got[1, 4] - do1[4]) < 1e-12 * do1[4]
    assert abs(got[1, 0] - do1[0]) < 1e-8 * do1[0]


def test_in_step_diagnostics_mixed_precision():
    cfg, datas = _tov(1, precision=S.MIXED)
    a, b = _pair(cfg, datas)
    n = 3
    ref = _separate(a, cfg.dt, n, True)
    got = b.step_constraints(cfg.dt, n, use_graph=True)
    assert np.array_equal(got[:, 4:7], ref[:, 4:7])        # Mb, J, rho_max: no derivatives involved
    # the momentum constraint: the same kernel on the same FP32 derivatives
    assert np.allclose(got[:, 1:4], ref[:, 1:4], rtol=1e-6, atol=0.0), (got[:, 1:4], ref[:, 1:4])
    # ||H|| takes the FP32 Ricci scalar of the mixed pointwise pass instead of
    # an FP64 Ricci tensor of the FP32 derivatives: terms of order 0.1 rounded
    # at 6e-8 against ||H|| ~ 1e-3 for this perturbed star
    assert np.allclose(got[:, 0], ref[:, 0], rtol=1e-4, atol=0.0), (got[:, 0], ref[:, 0])
    for l in range(cfg.n_levels):
        assert np.array_equal(a.read(l, S.STATE_STEP, 25), b.read(l, S.STATE_STEP, 25)), l


def test_in_step_diagnostics_frozen_metric():
    """Cowling runs (no spacetime evolution) have no derivative pass: only the
    hydrodynamic sums."""
    cfg = W.RunConfig(n_levels=2, nx=48, nz=48, geometry=1, evolve_spacetime=0, dx0=0.5, dz0=0.5,
                      K=100.0, Gamma=2.0, Gamma_th=2.0, rho_atm=1e-14, rk=1)
    datas = []
    for l in range(2):
        X, Z = W.cell_centres(cfg, l)
        d = np.zeros((30,) + X.shape)
        d[:25] = W.flat_metric(cfg)
        r2 = ((X - 9.0) ** 2 + (Z - 8.0) ** 2) / 9.0
        bump = np.where(r2 < 1.0, (1.0 - r2) ** 3, 0.0)
        d[25] = 1e-3 * (1.0 + 2.0 * bump)
        d[29] = 100 * d[25] ** 2 * 1.5
        d[26] = 0.3 * bump
        datas.append(d)
    a, b = _pair(cfg, datas)
    ref = _separate(a, cfg.dt, 3, False)
    got = b.step_constraints(cfg.dt, 3, use_graph=False)
    assert np.array_equal(got[:, :8], ref[:, :8])
    assert np.array_equal(got[:-1, 8], ref[1:, 8])


def test_in_step_diagnostics_refused_when_subcycled():
    cfg, datas = _tov(1, L=2)
    cfg = dataclasses.replace(cfg, subcycle_from=1)
    s = S.Sacra(cfg)
    for l, d in enumerate(datas):
        s.set_initial_data(l, S.PRIM_METRIC, d)
    with pytest.raises(S.SacraError):
        s.step_constraints(cfg.dt, 1)
