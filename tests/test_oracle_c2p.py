"""Pins of the oracle's EOS and primitive recovery (Sec. II.C.3-4)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2502_03223_gb300 import workloads as W


def _cfg(**kw):
    base = dict(K=100.0, Gamma=2.0, Gamma_th=2.0, rho_atm=1e-14, w_max=100.0, c2p_tol=1e-12, c2p_maxit=100,
                geometry=1)
    base.update(kw)
    return W.RunConfig(**base)


def test_hybrid_eos_reduces_to_gamma_law():
    # K = 100, Gamma = Gamma_th = 2: P = P_cold + (Gamma_th - 1) rho (eps - eps_cold) = rho eps exactly
    cfg = _cfg()
    rng = np.random.default_rng(0)
    for rho, t in zip(10 ** rng.uniform(-8, -2, 20), 10 ** rng.uniform(-6, 1, 20)):
        eps = 100.0 * rho * (1.0 + t)      # eps >= eps_cold = K rho / (Gamma - 1)
        assert math.isclose(O.eos_press(cfg, rho, eps), rho * eps, rel_tol=1e-13)
        assert math.isclose(O.eos_eps(cfg, rho, rho * eps), eps, rel_tol=1e-12)


def test_sound_speed_is_the_thermodynamic_derivative():
    # c_s^2 = (dP/drho|_eps + P/rho^2 dP/deps|_rho) / h, by central differences
    cfg = _cfg(Gamma=2.5, Gamma_th=5.0 / 3.0, K=30.0)
    for rho, eps_th in ((1e-3, 0.05), (2e-4, 1e-3), (5e-3, 0.3)):
        eps = rho ** 1.5 * 30.0 / 1.5 + eps_th
        P = O.eos_press(cfg, rho, eps)
        hr, he = rho * 1e-6, eps * 1e-6
        dPdr = (O.eos_press(cfg, rho + hr, eps) - O.eos_press(cfg, rho - hr, eps)) / (2 * hr)
        dPde = (O.eos_press(cfg, rho, eps + he) - O.eos_press(cfg, rho, eps - he)) / (2 * he)
        h = 1.0 + eps + P / rho
        cs2 = (dPdr + P / rho ** 2 * dPde) / h
        assert math.isclose(O.eos_cs2(cfg, rho, eps, P), cs2, rel_tol=1e-7)


@pytest.mark.parametrize("geometry", [0, 1])
def test_round_trip_forward_error(geometry):
    """Well-conditioned states (eps not tiny against w^2 eps_machine): the
    recovered primitives equal the ones the conserved state was built from."""
    cfg = _cfg(geometry=geometry)
    rng = np.random.default_rng(42)
    rho, u, pfac = W.random_prims(rng, 300, w_max=10.0, log_rho=(-6.0, -2.0))
    worst = 0.0
    for i in range(len(rho)):
        Wc, h = W.random_conformal_metric(rng)
        P = cfg.K * rho[i] ** cfg.Gamma * (1.0 + pfac[i])
        eps = O.eos_eps(cfg, rho[i], P)
        prim = np.array([rho[i], u[i, 0], u[i, 1], u[i, 2], P, eps])
        x = rng.uniform(0.5, 3.0)
        q = O.prim2cons(cfg, prim, Wc, h, x)
        pr, q2, st, it = O.con2prim(cfg, q, Wc, h, x)
        assert st == 0, st
        un = math.sqrt(u[i] @ u[i])
        for v in range(6):
            scale = max(abs(prim[v]), un if v in (1, 2, 3) else 0.0, 1e-300)
            worst = max(worst, abs(pr[v] - prim[v]) / scale)
    assert worst < 1e-9, worst


@pytest.mark.parametrize("geometry", [0, 1])
def test_round_trip_backward_error(geometry):
    """All random states up to w = 50 over 8 decades of density: the recovered
    primitives reproduce the conserved state (backward error), which is the
    meaningful measure where eps comes from cancelling O(w^2) terms."""
    cfg = _cfg(geometry=geometry)
    rng = np.random.default_rng(43)
    rho, u, pfac = W.random_prims(rng, 400, w_max=50.0, log_rho=(-10.0, -2.0))
    worst = 0.0
    for i in range(len(rho)):
        Wc, h = W.random_conformal_metric(rng)
        P = cfg.K * rho[i] ** cfg.Gamma * (1.0 + pfac[i])
        prim = np.array([rho[i], u[i, 0], u[i, 1], u[i, 2], P, O.eos_eps(cfg, rho[i], P)])
        x = rng.uniform(0.5, 3.0)
        q = O.prim2cons(cfg, prim, Wc, h, x)
        pr, q2, st, it = O.con2prim(cfg, q, Wc, h, x)
        assert st & 1 == 0 and it < 60
        if st == 0:
            q3 = O.prim2cons(cfg, pr, Wc, h, x)
            worst = max(worst, np.max(np.abs(q3 - q)) / np.max(np.abs(q)))
    # the Illinois iteration stops at a relative bracket of c2p_tol = 1e-12 in z
    assert worst < 1e-11, worst


def test_zero_momentum_gives_zero_velocity_exactly():
    cfg = _cfg()
    prim = np.array([1e-3, 0.0, 0.0, 0.0, 100 * 1e-6 * 1.3, 0.0])
    prim[5] = O.eos_eps(cfg, prim[0], prim[4])
    q = O.prim2cons(cfg, prim, 0.8, np.zeros(6), 1.0)
    pr, _, st, it = O.con2prim(cfg, q, 0.8, np.zeros(6), 1.0)
    assert pr[1] == 0.0 and pr[2] == 0.0 and pr[3] == 0.0
    assert math.isclose(pr[0], prim[0], rel_tol=1e-13)


def test_cold_branch_keeps_D_and_S():
    # an energy below the cold curve forces the cold recovery; (D, S_i) must be kept
    cfg = _cfg()
    rho, P = 2e-3, 100 * 4e-6
    prim = np.array([rho, 0.1, -0.05, 0.2, P, O.eos_eps(cfg, rho, P)])
    h = np.array([0.01, 0.002, 0.0, -0.01, 0.003, 0.02])
    q = O.prim2cons(cfg, prim, 0.9, h, 1.0)
    q_bad = q.copy()
    q_bad[4] -= 0.02 * q[4]
    pr, q2, st, it = O.con2prim(cfg, q_bad, 0.9, h, 1.0)
    assert st & 2, st                                   # cold branch taken
    assert math.isclose(pr[4], cfg.K * pr[0] ** cfg.Gamma, rel_tol=1e-12)
    assert np.allclose(q2[:4], q_bad[:4], rtol=1e-10, atol=0)  # D and S_i kept
    assert q2[4] != q_bad[4]                            # E reset from the primitives
    q3 = O.prim2cons(cfg, pr, 0.9, h, 1.0)
    assert np.allclose(q3, q2, rtol=1e-12)


def test_atmosphere_and_velocity_cap():
    cfg = _cfg(rho_atm=1e-8)
    prim = np.array([1e-10, 0.0, 0.0, 0.0, 1e-18, 0.0])
    prim[5] = O.eos_eps(cfg, prim[0], prim[4])
    q = O.prim2cons(cfg, prim, 1.0, np.zeros(6), 1.0)
    pr, q2, st, it = O.con2prim(cfg, q, 1.0, np.zeros(6), 1.0)
    assert st & 4 and pr[0] == 1e-8 and pr[1] == 0.0
    assert math.isclose(pr[4], cfg.K * 1e-16, rel_tol=1e-14)
    # momentum far beyond w_max is rescaled: the recovered Lorentz factor stays below w_max
    cfg2 = _cfg()
    prim = np.array([1e-3, 0.0, 0.0, 0.0, 1e-4, 0.0])
    prim[5] = O.eos_eps(cfg2, prim[0], prim[4])
    q = O.prim2cons(cfg2, prim, 1.0, np.zeros(6), 1.0)
    q[1] = 1e3 * q[4]
    pr, q2, st, it = O.con2prim(cfg2, q, 1.0, np.zeros(6), 1.0)
    assert st & 8
    w = math.sqrt(1.0 + pr[1] ** 2 + pr[2] ** 2 + pr[3] ** 2)
    assert w <= cfg2.w_max * (1 + 1e-9)


def test_atmosphere_decided_by_D_alone():
    """The recovery returns rho = D / w <= D on either branch (w >= 1), so a
    cell with D = rho w < rho_atm always ends in the atmosphere: checked by
    recovering random states (hot, cold-branch and fast ones) with no
    atmosphere and comparing rho with D; with the atmosphere on, such a cell
    returns the atmosphere primitives and the conserved state rebuilt from
    them."""
    cfg0 = _cfg(rho_atm=1e-300)
    rng = np.random.default_rng(5)
    rho, u, pfac = W.random_prims(rng, 200, w_max=30.0, log_rho=(-12.0, -3.0))
    for i in range(len(rho)):
        Wc, h = W.random_conformal_metric(rng)
        P = cfg0.K * rho[i] ** cfg0.Gamma * (1.0 + pfac[i])
        prim = np.array([rho[i], u[i, 0], u[i, 1], u[i, 2], P, O.eos_eps(cfg0, rho[i], P)])
        x = rng.uniform(0.5, 3.0)
        q = O.prim2cons(cfg0, prim, Wc, h, x)
        if i % 3 == 0:
            q[4] *= 0.5                                   # too little energy: cold branch
        D = q[0] * (Wc * Wc * Wc)                        # as the recovery forms it
        pr, _, st, _ = O.con2prim(cfg0, q.copy(), Wc, h, x)
        assert not st & 4 and pr[0] <= D, (i, st, pr[0], D)
        cfg = _cfg(rho_atm=D * 1.5)
        pa, qa, sta, _ = O.con2prim(cfg, q.copy(), Wc, h, x)
        assert sta == 4 and pa[0] == cfg.rho_atm and np.all(pa[1:4] == 0.0)
        assert np.array_equal(qa, O.prim2cons(cfg, pa, Wc, h, x))
