"""The piecewise polytropic cold EOS and the "adiabatic" (zero-temperature)
EOS on the GPU (Sec. II.C.3; Sec. III migration test): step-by-step parity
with the oracle, the adiabatic star staying on the cold curve, the mixed
form's error, and a batch of stars with different EOS equal to each alone."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import G, both, compare_level, compare_status

pytestmark = pytest.mark.gpu

PWP = ((1e-4, 2.0), (8e-4, 2.5))
K1 = 100.0 * 1e-4 ** (2.0 - 4.0 / 3.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


def _pwp_star(L=2, N=32, adiabatic=0, rk=0, dx_fine=0.5, perturb=True):
    cfg, tov = W.tov_config("pwp", rho_c=1.28e-3, n_levels=L, N=N, dx_fine=dx_fine, rk=rk, K=K1, Gamma=4.0 / 3.0,
                            Gamma_th=5.0 / 3.0, pwp=PWP, eos_adiabatic=adiabatic)
    datas = []
    for l in range(L):
        d = W.tov_level_data(cfg, tov, l)
        if perturb:
            X, Z = W.cell_centres(cfg, l)
            bump = np.exp(-((X - 2.0) ** 2 + (Z - 3.0) ** 2) / 6.0)
            d[26] = 0.04 * bump * X / (np.abs(X) + 1.0)
            d[28] = 0.03 * bump * Z / (np.abs(Z) + 1.0)
        datas.append(d)
    return cfg, datas


def _migration_adiabatic(L=2, N=32):
    cfg, tov = W.tov_config("mig_ad", rho_c=7.993e-3, n_levels=L, N=N, dx_fine=0.25, rk=0, eos_adiabatic=1)
    return cfg, [W.tov_level_data(cfg, tov, l, p_deplete=0.99) for l in range(L)]


@pytest.mark.parametrize("which", ["pwp_hybrid", "pwp_adiabatic", "migration_adiabatic"])
def test_eos_variant_matches_oracle_every_step(which):
    if which == "migration_adiabatic":
        cfg, datas = _migration_adiabatic()
    else:
        cfg, datas = _pwp_star(adiabatic=int(which == "pwp_adiabatic"))
    gpu, orc = both(cfg, datas)
    worst = 0.0
    for _ in range(3):
        gpu.step(cfg.dt, 1)
        orc.step(cfg.dt, 1)
        for l in range(cfg.n_levels):
            worst = max(worst, compare_level(gpu, orc, l, 1e-11, which=(S.STATE_STEP, S.PRIMS)))
            compare_status(gpu, orc, l)
    assert worst < 1e-11


def test_adiabatic_gpu_star_stays_on_the_cold_curve():
    cfg, datas = _pwp_star(adiabatic=1, L=2)
    s = S.Sacra(cfg)
    for l, d in enumerate(datas):
        s.set_initial_data(l, S.PRIM_METRIC, d)
    s.step(cfg.dt, 5, use_graph=True)
    for l in range(cfg.n_levels):
        rho = s.read(l, S.PRIMS, 0)[G:G + cfg.nz, G:G + cfg.nx].ravel()
        P = s.read(l, S.PRIMS, 4)[G:G + cfg.nz, G:G + cfg.nx].ravel()
        eps = s.read(l, S.PRIMS, 5)[G:G + cfg.nz, G:G + cfg.nx].ravel()
        Pc = np.array([O.eos_pcold(cfg, r) for r in rho])
        ec = np.array([O.eos_ecold(cfg, r) for r in rho])
        assert np.allclose(P, Pc, rtol=1e-14, atol=0), l
        assert np.allclose(eps, ec, rtol=1e-14, atol=0), l


def test_mixed_precision_with_pieces():
    cfg, datas = _pwp_star(L=2)
    mixed = dataclasses.replace(cfg, precision=7)
    a, b = S.Sacra(cfg), S.Sacra(mixed)
    for l, d in enumerate(datas):
        a.set_initial_data(l, S.PRIM_METRIC, d)
        b.set_initial_data(l, S.PRIM_METRIC, d)
    a.step(cfg.dt, 2)
    b.step(cfg.dt, 2)
    num = den = 0.0
    for l in range(cfg.n_levels):
        x = a.read(l, S.PRIMS, 0)[G:G + cfg.nz, G:G + cfg.nx]
        y = b.read(l, S.PRIMS, 0)[G:G + cfg.nz, G:G + cfg.nx]
        num += np.abs(x - y).sum()
        den += np.abs(x).sum()
    print("mixed vs FP64, three-piece star, rho L1 after 2 steps: %.2e" % (num / den))
    assert num / den < 1e-6


def test_batch_of_different_eos_equals_each_star_alone():
    stars = [_pwp_star(L=2, N=32, adiabatic=0), _pwp_star(L=1, N=48, adiabatic=1), _migration_adiabatic(L=2, N=32)]
    c0, tov = W.tov_config("single", rho_c=2e-3, n_levels=2, N=40, dx_fine=0.5, rk=0)
    stars.append((c0, [W.tov_level_data(c0, tov, l) for l in range(2)]))
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
                assert np.array_equal(batch.read(i, l, S.STATE_STEP, f), alone.read(l, S.STATE_STEP, f)), (i, l, f)
        alone.close()
