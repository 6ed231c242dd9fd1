"""The FP64 tolerance on the whole dynamical path: Z4c (Sec. II.B) and GRHD
(Sec. II.C) together on a fixed-mesh-refinement hierarchy (Sec. II.D), 100
steps on the GPU (through the C ABI, CUDA-graph replay as the benchmark runs
it) and on the CPU oracle from the same initial data: the rest-mass density
agrees within 1e-9 in the L1 norm on every level.  Cases: the stable star and
the migration star (Sec. III.C.2, 1% pressure depletion), each with
classical RK4 and SSP-RK3, the stable star also with a seeded perturbation of
every metric field and a velocity bump."""
import numpy as np
import pytest

from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import G, STATE_GROUPS, both, group_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


def _case(kind, rk):
    if kind == "stable":
        cfg, tov = W.tov_config("stable_3x48", rho_c=1.28e-3, n_levels=3, N=48, dx_fine=0.5, rk=rk)
        datas = [W.tov_level_data(cfg, tov, l) for l in range(cfg.n_levels)]
    elif kind == "stable_perturbed":
        cfg, tov = W.tov_config("stable_2x48p", rho_c=1.28e-3, n_levels=2, N=48, dx_fine=0.5, rk=rk)
        datas = []
        for l in range(cfg.n_levels):
            d = W.tov_level_data(cfg, tov, l)
            d[:25] += W.random_metric_perturbation(cfg, l, np.random.default_rng(7), amp=1e-3)
            X, Z = W.cell_centres(cfg, l)
            bump = np.exp(-((X - 3.0) ** 2 + (Z - 2.0) ** 2) / 4.0)
            d[26] = 0.05 * bump * X / (np.abs(X) + 1.0)
            datas.append(d)
    else:
        cfg, tov = W.config_migration(N=64, n_levels=3, dx_fine=0.1)
        datas = [W.tov_level_data(cfg, tov, l, p_deplete=0.99) for l in range(cfg.n_levels)]
    return cfg, datas


@pytest.mark.parametrize("kind,rk", [("stable", 1), ("stable", 0), ("migration", 0), ("migration", 1),
                                     ("stable_perturbed", 0)])
def test_rho_l1_after_100_steps_every_level(kind, rk):
    cfg, datas = _case(kind, rk)
    gpu, orc = both(cfg, datas)
    gpu.step(cfg.dt, 100, use_graph=True)
    orc.step(cfg.dt, 100)
    errs = []
    for l in range(cfg.n_levels):
        a = gpu.read(l, S.PRIMS, 0)[G:G + cfg.nz, G:G + cfg.nx]
        b = orc.read(l, 2, 0)[G:G + cfg.nz, G:G + cfg.nx]
        errs.append(float(np.abs(a - b).sum() / np.abs(b).sum()))
    # the metric after 100 steps, for the record: the largest difference per
    # field relative to the largest magnitude of its physical group on the
    # level (the y-components of a star without rotation are rounding noise on
    # both sides, so their own maximum is no scale)
    met, where = 0.0, None
    for l in range(cfg.n_levels):
        B = [orc.read(l, 0, f)[G:G + cfg.nz, G:G + cfg.nx] for f in range(30)]
        for f in range(25):
            a = gpu.read(l, S.STATE_STEP, f)[G:G + cfg.nz, G:G + cfg.nx]
            s = group_scale(B, STATE_GROUPS, f)
            if s > 0 and float(np.max(np.abs(a - B[f]))) / s > met:
                met, where = float(np.max(np.abs(a - B[f]))) / s, (l, f)
    print("%s %s: rho L1 per level %s; worst metric difference %.2e of its group scale (level, field %s)"
          % (kind, "RK4" if rk == 0 else "SSP-RK3", " ".join("%.2e" % e for e in errs), met, where))
    assert max(errs) <= 1e-9, errs
    gpu.close()
    orc.close()
