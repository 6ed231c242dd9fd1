"""Mixed-precision form of the CUDA path (precision = MIXED): reconstruction,
Riemann solver, hydro sources and the Z4c algebra in FP32, every finite
difference of the state, the primitive recovery, the algebraic constraints and
all accumulation in FP64.  Checked against the FP64 oracle: rest-mass density
L1 error <= 1e-6 relative after 100 steps, the exact properties that do not
depend on the arithmetic (uniform states, Minkowski, rest-mass conservation),
and a per-output error report after one step."""
import dataclasses

import numpy as np
import pytest

from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import G, both, group_scale, STATE_GROUPS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


def _mixed(cfg):
    return dataclasses.replace(cfg, precision=S.MIXED)


def _rho_l1(gpu, orc, cfg, l):
    a = gpu.read(l, S.PRIMS, 0)[G:G + cfg.nz, G:G + cfg.nx]
    b = orc.read(l, 2, 0)[G:G + cfg.nz, G:G + cfg.nx]
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_mixed_shock_tube_rho_l1_after_100_steps():
    cfg = _mixed(W.config_shock_tube())
    d0 = W.shock_tube_data(cfg)
    gpu, orc = both(cfg, [d0])
    gpu.step(cfg.dt, 100)
    orc.step(cfg.dt, 100)
    err = _rho_l1(gpu, orc, cfg, 0)
    assert err <= 1e-6, err
    assert err > 0.0          # the FP32 arithmetic really ran
    # the flux divergence telescopes in FP64: rest mass is conserved to rounding
    m = gpu.read(0, S.STATE_STEP, 25)[G:G + cfg.nz, G:G + cfg.nx].sum()
    m0 = d0[25][G:G + cfg.nz, G:G + cfg.nx].sum()
    assert abs(m - m0) / m0 < 1e-13


def _tov(L=2, N=32, rk=0):
    cfg, tov = W.tov_config("tov_small", rho_c=1.28e-3, n_levels=L, N=N, dx_fine=0.5, rk=rk)
    datas = []
    for l in range(L):
        d = W.tov_level_data(cfg, tov, l)
        d[:25] += W.random_metric_perturbation(cfg, l, np.random.default_rng(100), amp=1e-4)
        datas.append(d)
    return _mixed(cfg), datas


@pytest.mark.parametrize("rk", [0, 1])
def test_mixed_tov_fmr_rho_l1_after_100_steps(rk):
    cfg, datas = _tov(rk=rk)
    gpu, orc = both(cfg, datas)
    gpu.step(cfg.dt, 100, use_graph=True)
    orc.step(cfg.dt, 100)
    for l in range(cfg.n_levels):
        err = _rho_l1(gpu, orc, cfg, l)
        assert 0.0 < err <= 1e-6, (l, err)


def test_mixed_migration_star_rho_l1():
    """The unstable-branch star (pressure depleted by 1%) on a reduced grid."""
    cfg, tov = W.tov_config("migration_small", rho_c=7.993e-3, n_levels=2, N=32, dx_fine=0.4, rk=1)
    datas = [W.tov_level_data(cfg, tov, l, p_deplete=0.99) for l in range(cfg.n_levels)]
    cfg = _mixed(cfg)
    gpu, orc = both(cfg, datas)
    gpu.step(cfg.dt, 100, use_graph=True)
    orc.step(cfg.dt, 100)
    for l in range(cfg.n_levels):
        err = _rho_l1(gpu, orc, cfg, l)
        assert err <= 1e-6, (l, err)


def test_mixed_per_output_errors_one_step():
    """Every output of one RK4 step against the FP64 oracle, relative to the
    scale of its physical group.  Bound: FP32 rounding (6e-8) amplified by the
    cancellation among the O(100) terms of the Ricci tensor and the sources,
    i.e. 1e-5, still far below the truncation error of the scheme."""
    cfg, datas = _tov(L=2, N=32)
    gpu, orc = both(cfg, datas)
    gpu.step(cfg.dt, 1)
    orc.step(cfg.dt, 1)
    report = {}
    for l in range(cfg.n_levels):
        B = [orc.read(l, 0, f) for f in range(30)]
        for f in range(30):
            a = gpu.read(l, S.STATE_STEP, f)[G:G + cfg.nz, G:G + cfg.nx]
            b = B[f][G:G + cfg.nz, G:G + cfg.nx]
            xmax = (cfg.nx + 8) * cfg.dx(l)
            sg = group_scale(B, STATE_GROUPS, f, xmax)
            report[(l, f)] = float(np.max(np.abs(a - b))) / sg if sg > 0 else 0.0
    worst = max(report.values())
    print("mixed one-step worst group-relative error: %.3e at %s" % (worst, max(report, key=report.get)))
    assert worst < 1e-5, sorted(report.items(), key=lambda kv: -kv[1])[:5]


def test_mixed_uniform_state_exact():
    """A uniform boosted fluid on a flat slab: every face computes the same
    FP32 flux and the divergence is taken in FP64, so the mixed path holds the
    state bit for bit, as the FP64 path does."""
    cfg = W.RunConfig(name="uniform", n_levels=1, nx=24, nz=20, geometry=0, evolve_spacetime=0, rk=0,
                      dx0=0.1, dz0=0.1, Gamma=5.0 / 3.0, Gamma_th=5.0 / 3.0, K=0.0, rho_atm=1e-12,
                      precision=S.MIXED)
    d = W.flat_metric(cfg)
    rng = np.random.default_rng(3)
    ux, uz = rng.uniform(-0.3, 0.3, 2)
    pr = np.zeros((6, cfg.pz, cfg.px))
    pr[0] = 1.3; pr[1] = ux; pr[3] = uz; pr[4] = 0.7
    pr[5] = pr[4] / ((cfg.Gamma - 1.0) * pr[0])
    d = np.concatenate([d, pr[[0, 1, 2, 3, 4]]])
    gpu = S.Sacra(cfg)
    gpu.set_initial_data(0, S.PRIM_METRIC, d)
    before = [gpu.read(0, S.STATE_STEP, f) for f in range(30)]
    gpu.step(cfg.dt, 5)
    for f in range(30):
        a = gpu.read(0, S.STATE_STEP, f)[G:G + cfg.nz, G:G + cfg.nx]
        assert np.array_equal(a, before[f][G:G + cfg.nz, G:G + cfg.nx]), f


def test_staged_fp32_faces_equal_the_per_face_form():
    """The FP32 face fluxes of a stage (inputs split once per cell of a tile
    and staged through shared memory) equal, bit for bit, the per-face form
    that splits every input of every face again (the allocation-free entry
    point runs that form): the same FP32 arithmetic on the same values.  A
    moving bump gives faces with velocity; the stellar surface gives faces
    that go to the FP64 solver."""
    import torch
    cfg, tov = W.tov_config("staged32", rho_c=1.28e-3, n_levels=1, N=64, dx_fine=0.5, rk=0)
    cfg = dataclasses.replace(cfg, precision=S.MIXED_FLUX | S.MIXED_SOURCES)
    d = W.tov_level_data(cfg, tov, 0)
    X, Z = W.cell_centres(cfg, 0)
    bump = np.exp(-((X - 4.0) ** 2 + (Z - 3.0) ** 2) / 4.0)
    d[26] = 0.1 * bump * X / (np.abs(X) + 1.0)
    d[28] = 0.05 * bump * Z / (np.abs(Z) + 1.0)
    sim = S.Sacra(cfg)
    sim.set_initial_data(0, S.PRIM_METRIC, d)
    sim.fill(0, cfg.dt)
    P = sim.px * sim.pz
    state = np.stack([sim.read(0, S.STATE_STEP, f) for f in range(30)]).reshape(30 * P)
    prims = np.stack([sim.read(0, S.PRIMS, f) for f in range(6)]).reshape(6 * P)
    sim.rk_stage(0, cfg.dt)
    ref = np.stack([sim.read(0, S.RHS, 25 + v) for v in range(5)])
    dev = torch.device("cuda")
    out = torch.full((5 * P,), float("nan"), dtype=torch.float64, device=dev)
    rc = S.hydro_rhs_noalloc(cfg, 0, torch.from_numpy(state).to(dev).data_ptr(),
                             torch.from_numpy(prims).to(dev).data_ptr(), out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(5, sim.pz, sim.px)
    for v in range(5):
        a = got[v][G:G + cfg.nz, G:G + cfg.nx]
        b = ref[v][G:G + cfg.nz, G:G + cfg.nx]
        assert np.array_equal(a, b), (v, float(np.max(np.abs(a - b))))
