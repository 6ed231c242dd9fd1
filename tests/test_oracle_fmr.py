"""Pins of the oracle's FMR operators (Sec. II.D): prolongation and
restriction exact on polynomials of their order, conservative restriction,
and rest-mass conservation to round-off with reflux on a two-level run."""
import numpy as np
import pytest

import oracle as O
from paper_2502_03223_gb300 import workloads as W

G = 8


def _cfg(N=16, L=2, dx0=1.0):
    return W.RunConfig(n_levels=L, nx=N, nz=N, geometry=1, evolve_spacetime=0, dx0=dx0, dz0=dx0, K=100.0,
                       Gamma=2.0, Gamma_th=2.0, rho_atm=1e-14, rk=0)


def _poly(X, Z):
    # even in x and z, degree 6 in each variable (8-point Lagrange is exact to degree 7)
    return 1.0 + 0.01 * X ** 2 - 0.003 * Z ** 2 + 2e-4 * X ** 2 * Z ** 2 + 1e-5 * X ** 4 * Z ** 2 \
        - 3e-6 * X ** 6 + 2e-7 * Z ** 6 * X ** 2


def _data(cfg, level, rho=1e-3, P=2e-4, poly=False):
    X, Z = W.cell_centres(cfg, level)
    d = np.zeros((30, cfg.pz, cfg.px))
    d[:25] = W.flat_metric(cfg)
    if poly:
        d[0] = _poly(X, Z)           # W
        d[13] = 0.1 * _poly(X, Z)    # Khat
    d[25] = rho
    d[29] = P
    return d


def test_prolongation_exact_on_polynomials():
    cfg = _cfg()
    o = O.Oracle(cfg)
    o.set_level(0, 0, _data(cfg, 0, poly=True))
    o.set_level(1, 0, _data(cfg, 1))
    o.fill(0, 0.0)
    X, Z = W.cell_centres(cfg, 1)
    for f, fac in ((0, 1.0), (13, 0.1)):
        got = o.read(1, 0, f)
        ref = fac * _poly(X, Z)
        buf = np.zeros_like(got, dtype=bool)
        buf[G:, G + cfg.nx:] = True          # j > N, k >= 1
        buf[G + cfg.nz:, G:] = True          # k > N, j >= 1
        assert np.max(np.abs(got[buf] - ref[buf])) < 1e-13
    # primitives: constants are reproduced exactly by the limited linear prolongation
    rho = o.read(1, 2, 0)
    assert np.all(rho[G:, G + cfg.nx:] == 1e-3)


def test_restriction_exact_and_conservative():
    cfg = _cfg()
    o = O.Oracle(cfg)
    o.set_level(0, 0, _data(cfg, 0))
    child = _data(cfg, 1, poly=True)
    X, Z = W.cell_centres(cfg, 1)
    rng = np.random.default_rng(4)
    child[25] = 1e-3 * (1.0 + 0.2 * rng.uniform(size=X.shape))   # rough density, positive
    o.set_level(1, 0, child)
    qc = o.read(1, 0, 25)[G:G + 16, G:G + 16]
    xc = (np.arange(1, 17) - 0.5) * cfg.dx(1)
    mass_child = np.sum(qc * xc[None, :]) * cfg.dx(1) ** 2
    o.restrict_reflux()
    qp = o.read(0, 0, 25)[G:G + 8, G:G + 8]
    xp = (np.arange(1, 9) - 0.5) * cfg.dx(0)
    mass_parent = np.sum(qp * xp[None, :]) * cfg.dx(0) ** 2
    assert abs(mass_parent - mass_child) < 1e-15 * mass_child * 64
    Xp, Zp = W.cell_centres(cfg, 0)
    Wp = o.read(0, 0, 0)[G:G + 8, G:G + 8]
    assert np.max(np.abs(Wp - _poly(Xp, Zp)[G:G + 8, G:G + 8])) < 1e-13


@pytest.mark.parametrize("levels,rk", [(2, 0), (3, 0), (2, 1)])
def test_mass_conservation_with_reflux(levels, rk):
    """A compactly supported density blob moving across the refinement
    boundaries on a frozen flat metric, far from the outer boundary: the total
    rest mass over non-covered cells is kept to round-off."""
    cfg = W.RunConfig(n_levels=levels, nx=48, nz=48, geometry=1, evolve_spacetime=0, dx0=0.5, dz0=0.5,
                      K=100.0, Gamma=2.0, Gamma_th=2.0, rho_atm=1e-14, rk=rk)
    o = O.Oracle(cfg)
    for l in range(levels):
        X, Z = W.cell_centres(cfg, l)
        d = _data(cfg, l)
        r2 = ((X - 9.0) ** 2 + (Z - 8.0) ** 2) / 9.0
        bump = np.where(r2 < 1.0, (1.0 - r2) ** 3, 0.0)
        d[25] = 1e-3 * (1.0 + 2.0 * bump)
        d[29] = 100 * d[25] ** 2 * 1.5
        d[26] = 0.3 * bump      # u_x
        d[28] = 0.2 * bump      # u_z
        o.set_level(l, 0, d)
    m0 = o.diag()[4]
    o.step(cfg.dt, 3)
    m1 = o.diag()[4]
    assert abs(m1 - m0) / m0 < 1e-13, (m0, m1)


def _blob(levels, rk, subcycle_from):
    cfg = W.RunConfig(n_levels=levels, nx=48, nz=48, geometry=1, evolve_spacetime=0, dx0=0.5, dz0=0.5,
                      K=100.0, Gamma=2.0, Gamma_th=2.0, rho_atm=1e-14, rk=rk, subcycle_from=subcycle_from)
    o = O.Oracle(cfg)
    for l in range(levels):
        X, Z = W.cell_centres(cfg, l)
        d = _data(cfg, l)
        r2 = ((X - 9.0) ** 2 + (Z - 8.0) ** 2) / 9.0
        bump = np.where(r2 < 1.0, (1.0 - r2) ** 3, 0.0)
        d[25] = 1e-3 * (1.0 + 2.0 * bump)
        d[29] = 100 * d[25] ** 2 * 1.5
        d[26] = 0.3 * bump
        d[28] = 0.2 * bump
        o.set_level(l, 0, d)
    return cfg, o


@pytest.mark.parametrize("levels,K,rk", [(2, 1, 0), (3, 1, 0), (3, 2, 1)])
def test_subcycled_mass_conservation(levels, K, rk):
    """Berger-Oliger sub-cycling (levels >= K take half their parent's step):
    the reflux with the time-weighted fine fluxes keeps the rest mass over
    non-covered cells to round-off."""
    cfg, o = _blob(levels, rk, K)
    m0 = o.diag()[4]
    o.step(cfg.dt, 3)
    m1 = o.diag()[4]
    assert abs(m1 - m0) / m0 < 1e-13, (m0, m1)


def test_subcycling_reproduces_lockstep_to_truncation_error():
    """Sub-cycled and lockstep runs of the same blob over the same time agree
    to the scheme's truncation error, and the lockstep setting of the
    sub-cycling parameter (K >= levels) is the lockstep run bit for bit."""
    steps = 4
    cfg_l, ol = _blob(3, 0, 0)
    ol.step(cfg_l.dt, 2 * steps)             # finest dt both runs
    cfg_s, os_ = _blob(3, 0, 2)
    assert abs(cfg_s.dt - 2 * cfg_l.dt) < 1e-15
    os_.step(cfg_s.dt, steps)
    for l in range(3):
        a = ol.read(l, 2, 0)[G:G + 48, G:G + 48]
        b = os_.read(l, 2, 0)[G:G + 48, G:G + 48]
        assert np.abs(a - b).sum() / np.abs(a).sum() < 5e-5, l
    cfg_k, ok = _blob(3, 0, 3)
    ok.step(cfg_k.dt, 2 * steps)
    for l in range(3):
        assert np.array_equal(ok.read(l, 0, 25), ol.read(l, 0, 25))
