"""Exact solution of the special-relativistic Riemann problem for an ideal gas
(no tangential velocity), written from the published method of Marti & Mueller
(J. Fluid Mech. 258, 317 (1994); Living Rev. Relativ. 6, 7 (2003)): the star
pressure p* is the root of v*_L(p) = v*_R(p), each side a shock (Taub adiabat
with the Rankine-Hugoniot mass flux) or a rarefaction (Riemann invariant of the
isentrope).  It is the analytic reference of the shock-tube test of Sec. III.B.1
of Lam & Shibata (arXiv:2502.03223).

TEST INFRASTRUCTURE ONLY (part of the oracle).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


class IdealGas:
    def __init__(self, gamma):
        self.g = gamma

    def h(self, rho, p):
        return 1.0 + self.g / (self.g - 1.0) * p / rho

    def cs(self, rho, p):
        return math.sqrt(self.g * p / (rho * self.h(rho, p)))


def _rare_invariant(gas, cs):
    """int c_s drho / rho along the isentrope, closed form for the ideal gas."""
    s = math.sqrt(gas.g - 1.0)
    return math.log((s + cs) / (s - cs)) / s


def rarefaction_v(gas, rho_a, p_a, v_a, p_b, sign):
    """Velocity behind a rarefaction: sign = -1 for the left (-) wave, +1 for the right (+) wave.
    0.5 ln((1+v)/(1-v)) - sign * int c_s drho/rho is constant across the fan."""
    rho_b = rho_a * (p_b / p_a) ** (1.0 / gas.g)
    ja = 0.5 * math.log((1 + v_a) / (1 - v_a)) - sign * _rare_invariant(gas, gas.cs(rho_a, p_a))
    jb = ja + sign * _rare_invariant(gas, gas.cs(rho_b, p_b))
    return math.tanh(jb), rho_b


def shock_state(gas, rho_a, p_a, v_a, p_b, sign):
    """State behind a shock of pressure p_b moving into state a; sign = -1 left, +1 right.
    Returns (v_b, rho_b, V_shock)."""
    g = gas.g
    h_a = gas.h(rho_a, p_a)
    W_a = 1.0 / math.sqrt(1.0 - v_a * v_a)
    A = 1.0 + (g - 1.0) * (p_a - p_b) / (g * p_b)
    B = -(g - 1.0) * (p_a - p_b) / (g * p_b)
    Cq = h_a * (p_a - p_b) / rho_a - h_a * h_a
    h_b = (-B + math.sqrt(B * B - 4.0 * A * Cq)) / (2.0 * A)
    rho_b = g * p_b / ((g - 1.0) * (h_b - 1.0))
    j2 = -(p_b - p_a) / (h_b / rho_b - h_a / rho_a)
    j = math.sqrt(j2)
    r2w2 = rho_a * rho_a * W_a * W_a
    Vs = (r2w2 * v_a + sign * j * math.sqrt(j2 + r2w2 * (1.0 - v_a * v_a))) / (r2w2 + j2)
    Ws = 1.0 / math.sqrt(1.0 - Vs * Vs)
    js = sign * j
    v_b = (h_a * W_a * v_a + Ws * (p_b - p_a) / js) / (h_a * W_a + (p_b - p_a) * (Ws * v_a / js + 1.0 / (rho_a * W_a)))
    return v_b, rho_b, Vs


def wave_v(gas, rho_a, p_a, v_a, p_b, sign):
    if p_b > p_a:
        v, _, _ = shock_state(gas, rho_a, p_a, v_a, p_b, sign)
    else:
        v, _ = rarefaction_v(gas, rho_a, p_a, v_a, p_b, sign)
    return v


class ExactRiemann:
    """Exact self-similar solution; state(xi) samples it at xi = (x - x0)/t."""

    def __init__(self, gamma, left, right):
        self.gas = IdealGas(gamma)
        self.L = tuple(map(float, left))    # (rho, p, v)
        self.R = tuple(map(float, right))
        rl, pl, vl = self.L
        rr, pr, vr = self.R

        def f(p):
            return wave_v(self.gas, rl, pl, vl, p, -1) - wave_v(self.gas, rr, pr, vr, p, +1)

        lo = max(min(pl, pr), 1e-14) * 1e-6 if min(pl, pr) > 0 else 1e-14
        hi = 10.0 * max(pl, pr) + 1.0
        self.pstar = brentq(f, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
        self.vstar = wave_v(self.gas, rl, pl, vl, self.pstar, -1)
        g = self.gas
        # left wave
        if self.pstar > pl:
            _, self.rhoL_star, self.VsL = shock_state(g, rl, pl, vl, self.pstar, -1)
            self.left_shock = True
        else:
            _, self.rhoL_star = rarefaction_v(g, rl, pl, vl, self.pstar, -1)
            self.left_shock = False
            cl = g.cs(rl, pl)
            cs_ = g.cs(self.rhoL_star, self.pstar)
            self.L_head = (vl - cl) / (1 - vl * cl)
            self.L_tail = (self.vstar - cs_) / (1 - self.vstar * cs_)
        # right wave
        if self.pstar > pr:
            _, self.rhoR_star, self.VsR = shock_state(g, rr, pr, vr, self.pstar, +1)
            self.right_shock = True
        else:
            _, self.rhoR_star = rarefaction_v(g, rr, pr, vr, self.pstar, +1)
            self.right_shock = False
            cr = g.cs(rr, pr)
            cs_ = g.cs(self.rhoR_star, self.pstar)
            self.R_head = (vr + cr) / (1 + vr * cr)
            self.R_tail = (self.vstar + cs_) / (1 + self.vstar * cs_)

    def _fan(self, xi, side):
        g = self.gas
        rho_a, p_a, v_a = self.L if side < 0 else self.R

        def f(p):
            v, rho = rarefaction_v(g, rho_a, p_a, v_a, p, side)
            c = g.cs(rho, p)
            lam = (v + side * c) / (1 + side * v * c)
            return lam - xi

        lo, hi = min(self.pstar, p_a), max(self.pstar, p_a)
        p = brentq(f, lo, hi, xtol=1e-15, rtol=1e-14, maxiter=500)
        v, rho = rarefaction_v(g, rho_a, p_a, v_a, p, side)
        return rho, p, v

    def state(self, xi):
        rl, pl, vl = self.L
        rr, pr, vr = self.R
        if xi < self.vstar:
            if self.left_shock:
                return self.L if xi < self.VsL else (self.rhoL_star, self.pstar, self.vstar)
            if xi < self.L_head:
                return self.L
            if xi > self.L_tail:
                return (self.rhoL_star, self.pstar, self.vstar)
            return self._fan(xi, -1)
        if self.right_shock:
            return self.R if xi > self.VsR else (self.rhoR_star, self.pstar, self.vstar)
        if xi > self.R_head:
            return self.R
        if xi < self.R_tail:
            return (self.rhoR_star, self.pstar, self.vstar)
        return self._fan(xi, +1)

    def profile(self, x, t, x0=0.5):
        out = np.array([self.state((xx - x0) / t) for xx in np.asarray(x, dtype=float)])
        return out[:, 0], out[:, 1], out[:, 2]

    def cell_average_rho(self, xl, xr, t, x0=0.5, nsub=64):
        """rho averaged over [xl, xr] by midpoint sub-sampling."""
        s = (np.arange(nsub) + 0.5) / nsub
        xs = xl + (xr - xl) * s
        return float(np.mean(self.profile(xs, t, x0)[0]))
