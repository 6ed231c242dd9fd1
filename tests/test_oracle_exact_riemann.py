"""Pins of the exact special-relativistic Riemann solver used as the shock-tube
reference (Sec. III.B.1): the paper's contact position, the Rankine-Hugoniot
jump conditions across the shock and the rarefaction ODE."""
import math

import numpy as np
from scipy.integrate import solve_ivp

from oracle.exact_riemann import ExactRiemann, IdealGas

from golden_values import PAPER


def test_contact_position_of_the_paper():
    # (rho, P, v) = (10, 40/3, 0) | (1, 0, 0), Gamma = 5/3: contact at x = 0.786 for t = 0.4
    e = ExactRiemann(5.0 / 3.0, (10.0, 40.0 / 3.0, 0.0), (1.0, 0.0, 0.0))
    assert abs(0.5 + PAPER["shock_tube_t"] * e.vstar - PAPER["shock_tube_contact_x"]) < 5e-4


def _cons(g, rho, p, v):
    W = 1.0 / math.sqrt(1.0 - v * v)
    h = g.h(rho, p)
    D, S, E = rho * W, rho * h * W * W * v, rho * h * W * W - p
    return np.array([D, S, E]), np.array([D * v, S * v + p, S])


def test_rankine_hugoniot_across_the_shock():
    e = ExactRiemann(5.0 / 3.0, (10.0, 13.33, 0.0), (1.0, 1e-6, 0.0))
    g = e.gas
    Ua, Fa = _cons(g, 1.0, 1e-6, 0.0)
    Ub, Fb = _cons(g, e.rhoR_star, e.pstar, e.vstar)
    res = e.VsR * (Ub - Ua) - (Fb - Fa)
    assert np.max(np.abs(res)) < 1e-10 * np.max(np.abs(Ub))


def test_rarefaction_follows_the_characteristic_ode():
    # dv/dp = -1 / (rho h W^2 c_s) across the left (-) rarefaction, isentropic rho(p)
    e = ExactRiemann(5.0 / 3.0, (10.0, 13.33, 0.0), (1.0, 1e-6, 0.0))
    g = e.gas
    rl, pl = 10.0, 13.33

    def rhs(p, y):
        v = y[0]
        rho = rl * (p / pl) ** (1.0 / g.g)
        return [-(1.0 - v * v) / (rho * g.h(rho, p) * g.cs(rho, p))]

    sol = solve_ivp(rhs, (pl, e.pstar), [0.0], rtol=1e-12, atol=1e-14)
    assert abs(sol.y[0, -1] - e.vstar) < 1e-8
    # continuity of the solution across the fan edges
    head, tail = e.L_head, e.L_tail
    assert np.allclose(e.state(head + 1e-12), e.state(head - 1e-12), rtol=1e-6)
    assert np.allclose(e.state(tail - 1e-12), e.state(tail + 1e-12), rtol=1e-6)
