"""The allocation-free hydro right-hand side (for callers that cannot call
cudaMalloc: its face-flux scratch is a static device array) gives the same
rates as the hydro part of sacra_rk_stage, on two calls in a row.  Collected
last so that a failure here comes after every other test has run."""
import numpy as np
import pytest

from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

pytestmark = pytest.mark.gpu
G = 8


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()


@pytest.mark.parametrize("precision", [S.FP64, S.MIXED_FLUX | S.MIXED_SOURCES], ids=["fp64", "mixed_hydro"])
def test_noalloc_hydro_rhs_matches_rk_stage(precision):
    """Same rates as the hydro part of sacra_rk_stage run with the same
    precision bits (the FP32 flux and source kernels in the mixed case)."""
    import dataclasses
    import torch
    cfg, tov = W.tov_config("noalloc", rho_c=1.28e-3, n_levels=1, N=64, dx_fine=0.5, rk=0)
    cfg = dataclasses.replace(cfg, precision=precision)
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
    st_d = torch.from_numpy(state).to(dev)
    pr_d = torch.from_numpy(prims).to(dev)
    for call in range(2):
        out = torch.full((5 * P,), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        rc = S.hydro_rhs_noalloc(cfg, 0, st_d.data_ptr(), pr_d.data_ptr(), out.data_ptr(), stream.cuda_stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(5, sim.pz, sim.px)
        for v in range(5):
            a = got[v][G:G + cfg.nz, G:G + cfg.nx]
            b = ref[v][G:G + cfg.nz, G:G + cfg.nx]
            scale = max(float(np.max(np.abs(ref[[0, 1, 3, 4]][:, G:G + cfg.nz, G:G + cfg.nx]))), 1e-300)
            if v == 2:
                scale *= cfg.nx * cfg.dx0
            assert np.all(np.abs(a - b) <= 1e-11 * np.maximum(np.abs(b), scale)), (precision, call, v)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    cfg, _ = W.config_migration()        # 512^2 cells per level: above the limit
    assert S.hydro_rhs_noalloc(cfg, 0, 1, 1, 1, 0) == -1
