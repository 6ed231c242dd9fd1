"""Pins of the oracle's piecewise polytropic cold EOS and of the "adiabatic"
(zero-temperature) EOS variant (Sec. II.C.3, Sec. III migration test)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2502_03223_gb300 import workloads as W

PWP = ((1e-4, 2.0), (8e-4, 2.5))          # crust Gamma = 4/3 below 1e-4, then 2, then 2.5 above 8e-4
K1 = 100.0 * 1e-4 ** (2.0 - 4.0 / 3.0)     # so that the middle piece is K = 100, Gamma = 2


def _cfg(**kw):
    base = dict(K=K1, Gamma=4.0 / 3.0, Gamma_th=5.0 / 3.0, rho_atm=1e-14, w_max=100.0, c2p_tol=1e-12,
                c2p_maxit=100, geometry=1, pwp=PWP)
    base.update(kw)
    return W.RunConfig(**base)


def test_pieces_are_continuous_and_follow_the_first_law():
    cfg = _cfg()
    for rt, _ in PWP:
        for f in (O.eos_pcold, O.eos_ecold):
            a, b = f(cfg, rt * (1 - 1e-13)), f(cfg, rt)
            assert abs(a - b) <= 1e-11 * abs(b), (f.__name__, rt, a, b)
    assert O.eos_pcold(cfg, 5e-4) == pytest.approx(100.0 * 5e-4 ** 2, rel=1e-13)   # middle piece: K = 100, Gamma = 2
    assert O.eos_gamma_cold(cfg, 5e-5) == 4.0 / 3.0 and O.eos_gamma_cold(cfg, 1e-3) == 2.5
    # zero-temperature first law d eps_c / d rho = P_c / rho^2 inside every piece
    for rho in (2e-6, 3e-5, 2e-4, 6e-4, 2e-3, 5e-3):
        h = rho * 1e-6
        de = (O.eos_ecold(cfg, rho + h) - O.eos_ecold(cfg, rho - h)) / (2 * h)
        assert de == pytest.approx(O.eos_pcold(cfg, rho) / rho ** 2, rel=1e-7), rho


def test_equal_indices_reduce_to_one_polytrope():
    one = _cfg(pwp=(), K=100.0, Gamma=2.0)
    two = _cfg(pwp=((3e-4, 2.0),), K=100.0, Gamma=2.0)
    for rho in (1e-5, 2e-4, 3e-4, 9e-4):
        assert O.eos_pcold(two, rho) == O.eos_pcold(one, rho)
        assert O.eos_ecold(two, rho) == O.eos_ecold(one, rho)


def test_sound_speed_with_pieces():
    cfg = _cfg()
    for rho, eth in ((5e-5, 1e-4), (4e-4, 1e-2), (2e-3, 0.05)):
        eps = O.eos_ecold(cfg, rho) + eth
        P = O.eos_press(cfg, rho, eps)
        hr, he = rho * 1e-6, eps * 1e-6
        dPdr = (O.eos_press(cfg, rho + hr, eps) - O.eos_press(cfg, rho - hr, eps)) / (2 * hr)
        dPde = (O.eos_press(cfg, rho, eps + he) - O.eos_press(cfg, rho, eps - he)) / (2 * he)
        h = 1.0 + eps + P / rho
        assert O.eos_cs2(cfg, rho, eps, P) == pytest.approx((dPdr + P / rho ** 2 * dPde) / h, rel=1e-6)


def test_round_trip_across_pieces():
    cfg = _cfg()
    rng = np.random.default_rng(3)
    rho, u, pfac = W.random_prims(rng, 200, w_max=10.0, log_rho=(-6.0, -2.9))
    for i in range(len(rho)):
        Wc, h = W.random_conformal_metric(rng)
        P = O.eos_pcold(cfg, rho[i]) * (1.0 + pfac[i])
        prim = np.array([rho[i], u[i, 0], u[i, 1], u[i, 2], P, O.eos_eps(cfg, rho[i], P)])
        x = rng.uniform(0.5, 3.0)
        q = O.prim2cons(cfg, prim, Wc, h, x)
        pr, _, st, _ = O.con2prim(cfg, q, Wc, h, x)
        assert st == 0
        assert pr[0] == pytest.approx(rho[i], rel=1e-9)
        assert pr[4] == pytest.approx(P, rel=1e-7)


def test_adiabatic_recovery_uses_D_and_S_only():
    cfg = _cfg(eos_adiabatic=1)
    rng = np.random.default_rng(4)
    rho, u, _ = W.random_prims(rng, 100, w_max=20.0, log_rho=(-6.0, -2.9))
    for i in range(len(rho)):
        Wc, h = W.random_conformal_metric(rng)
        P = O.eos_pcold(cfg, rho[i])
        prim = np.array([rho[i], u[i, 0], u[i, 1], u[i, 2], P, O.eos_ecold(cfg, rho[i])])
        x = rng.uniform(0.5, 3.0)
        q = O.prim2cons(cfg, prim, Wc, h, x)
        hot = q.copy()
        hot[4] *= 1.0 + rng.uniform(0.01, 0.5)          # extra energy: discarded
        a, qa, sa, _ = O.con2prim(cfg, q.copy(), Wc, h, x)
        b, qb, sb, _ = O.con2prim(cfg, hot, Wc, h, x)
        assert sa == sb == 0
        assert np.array_equal(a, b) and np.array_equal(qa, qb)   # E rebuilt from the cold primitives
        assert a[0] == pytest.approx(rho[i], rel=1e-9)
        assert a[4] == O.eos_pcold(cfg, a[0]) and a[5] == O.eos_ecold(cfg, a[0])
        for v in range(3):
            assert a[1 + v] == pytest.approx(u[i, v], rel=1e-8, abs=1e-12)


def test_adiabatic_star_stays_on_the_cold_curve():
    """A three-piece TOV star evolved with the adiabatic EOS keeps P = P_cold(rho)
    and eps = eps_cold(rho) in every interior cell, bit for bit."""
    import dataclasses
    cfg, tov = W.tov_config("pwp_adiabatic", rho_c=1.28e-3, n_levels=1, N=32, dx_fine=1.0, rk=1, K=K1,
                            Gamma=4.0 / 3.0, Gamma_th=5.0 / 3.0, pwp=PWP, eos_adiabatic=1)
    o = O.Oracle(cfg)
    o.set_level(0, 0, W.tov_level_data(cfg, tov, 0))
    o.step(cfg.dt, 3)
    rho, P, eps = (o.read(0, 2, f)[8:40, 8:40] for f in (0, 4, 5))
    assert all(P[k, j] == O.eos_pcold(cfg, rho[k, j]) for k in range(32) for j in range(32))
    assert all(eps[k, j] == O.eos_ecold(cfg, rho[k, j]) for k in range(32) for j in range(32))
    assert rho.max() > 8e-4 and rho.min() < 1e-4 * 1e-3          # the star spans all three pieces
