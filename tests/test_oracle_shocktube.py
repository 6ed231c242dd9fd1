"""Pins of the oracle's planar finite-volume update on the special-relativistic
shock tube (Sec. III.B.1): convergence to the exact solution, rest-mass
conservation to round-off, exact preservation of uniform states, and the
cylindrical pressure balance at rest."""
import numpy as np
import pytest

import oracle as O
from oracle.exact_riemann import ExactRiemann
from paper_2502_03223_gb300 import workloads as W

G = 8


def _run(nx, solver=0, t_end=0.4):
    cfg = W.shock_tube_config(nx, 4, solver=solver)
    o = O.Oracle(cfg)
    o.set_level(0, 0, W.shock_tube_data(cfg))
    n = int(round(t_end / cfg.dt))
    m0 = o.read(0, 0, 25)[G:G + cfg.nz, G:G + nx].sum()
    o.step(cfg.dt, n)
    m1 = o.read(0, 0, 25)[G:G + cfg.nz, G:G + nx].sum()
    rho = o.read(0, 2, 0)[G, G:G + nx]
    return cfg, rho, m0, m1


def _l1(nx, rho):
    ex = ExactRiemann(5.0 / 3.0, (10.0, 13.33, 0.0), (1.0, 1e-6, 0.0))
    xs = (np.arange(nx) + 0.5) / nx
    rex = np.array([ex.cell_average_rho(x - 0.5 / nx, x + 0.5 / nx, 0.4) for x in xs])
    return np.abs(rho - rex).mean()


def test_converges_to_the_exact_solution_and_conserves_mass():
    e1 = _l1(100, _run(100)[1])
    cfg, rho, m0, m1 = _run(200)
    e2 = _l1(200, rho)
    assert e2 < 0.6 * e1           # ~1st order at the discontinuities
    assert e2 < 0.05
    assert abs(m1 - m0) / m0 < 1e-13
    # contact (x = 0.786) between the star densities
    ex = ExactRiemann(5.0 / 3.0, (10.0, 13.33, 0.0), (1.0, 1e-6, 0.0))
    mid = 0.5 * (ex.rhoL_star + ex.rhoR_star)
    xs = (np.arange(200) + 0.5) / 200
    sel = (xs > 0.6) & (xs < 0.82)
    xc = xs[sel][np.argmin(np.abs(rho[sel] - mid))]
    assert abs(xc - (0.5 + 0.4 * ex.vstar)) < 3.0 / 200


def test_hllc_more_accurate_than_tvdlf():
    e_h = _l1(100, _run(100, 0)[1])
    e_t = _l1(100, _run(100, 1)[1])
    assert e_h < e_t


@pytest.mark.parametrize("solver", [0, 1])
def test_uniform_state_preserved_bitwise(solver):
    cfg = W.shock_tube_config(32, 4, solver=solver)
    d = W.shock_tube_data(cfg, left=(0.7, 0.3, 0.4), right=(0.7, 0.3, 0.4))
    o = O.Oracle(cfg)
    o.set_level(0, 0, d)
    before = [o.read(0, 0, f).copy() for f in range(25, 30)]
    o.step(cfg.dt, 10)
    after = [o.read(0, 0, f) for f in range(25, 30)]
    for b, a in zip(before, after):
        assert np.array_equal(b[G:-G, G:-G], a[G:-G, G:-G])


def test_cylindrical_rest_state_pressure_balance():
    # uniform fluid at rest on a flat metric in cylindrical geometry: the P/x
    # geometric source balances the area difference of the pressure flux
    cfg = W.RunConfig(n_levels=1, nx=32, nz=32, geometry=1, evolve_spacetime=0, K=100.0, Gamma=2.0,
                      Gamma_th=2.0, dx0=0.5, dz0=0.5, rho_atm=1e-14)
    d = np.zeros((30, cfg.pz, cfg.px))
    d[:25] = W.flat_metric(cfg)
    d[25] = 1e-3
    d[29] = 100 * 1e-6 * 1.5
    o = O.Oracle(cfg)
    o.set_level(0, 0, d)
    o.fill(0, cfg.dt)
    o.stage(0, cfg.dt)
    for f in range(25, 30):
        r = o.read(0, 3, f)[G:G + 28, G:G + 28]   # away from the outer boundary
        q = o.read(0, 0, 25 + 4)[G:G + 28, G:G + 28]
        assert np.max(np.abs(r)) < 1e-13 * np.max(np.abs(q)) / cfg.dx0


@pytest.mark.parametrize("solver", [0, 1])
def test_smooth_monotone_flow_has_no_numerical_dissipation(solver):
    """PPM in method-of-lines form (Sec. II.C.2: the reconstruction feeds the
    Riemann solver at every RK stage) gives equal left and right face states
    wherever the profile is smooth and monotone (no limiter acts): the face
    value is the 4th-order interpolant from both sides.  The Riemann solver's
    dissipation acts on the jump between them, so there it adds none, and a
    small perturbation of any wavelength, down to the 2-cell mode, is carried
    without damping.  This is the property behind the grid-scale noise of the
    Bondi runs: noise excited where a limiter switches is not removed."""
    nx = 128
    cfg = W.shock_tube_config(nx, 4, solver=solver)
    X, _ = W.cell_centres(cfg, 0)
    G = 8
    rho_s = 1.0 + 0.5 * np.tanh((X - 0.5) / 0.15)
    J = np.round(X / cfg.dx0 - 0.5).astype(int)
    v = 0.3
    base = np.zeros((30, cfg.pz, cfg.px))
    base[:25] = W.flat_metric(cfg)
    base[26] = v / np.sqrt(1 - v * v)
    base[29] = 1.0
    runs = []
    for pert in (0.0 * J, 1e-4 * (-1.0) ** J, 1e-4 * np.cos(np.pi * J / 2)):
        d = base.copy()
        d[25] = rho_s + pert
        o = O.Oracle(cfg)
        o.set_level(0, 0, d)
        o.step(cfg.dt, int(0.15 / cfg.dt))
        runs.append(o.read(0, 2, 0)[G + 1, G:G + nx])
    xs = X[G + 1, G:G + nx]
    m = (xs > 0.35) & (xs < 0.75)
    for r in runs[1:]:
        amp = np.sqrt(2 * np.mean((r - runs[0])[m] ** 2))
        assert 0.9e-4 < amp < 2e-4, amp
