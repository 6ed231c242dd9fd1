"""Pin of the oracle's hydro source terms (Sec. II.C.1; readings: Eulerian
v_i in the bracket, coefficient 1/W of the d W term, W^-3 on alpha K^ij S_ij)
against the textbook covariant Valencia sources
  s_j = sqrt(gamma) [ (alpha/2) S^ik d_j gamma_ik + S_i d_j beta^i - E d_j alpha ],
  s_E = sqrt(gamma) [ alpha S^ij K_ij - S^j d_j alpha ],
computed here from the physical metric gamma_ij = gt_ij / W^2 (det gt = 1)."""
import math

import numpy as np

import oracle as O
from paper_2502_03223_gb300 import workloads as W

S6 = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]


def _sym(v):
    return np.array([[v[S6[i][j]] for j in range(3)] for i in range(3)])


def test_sources_match_covariant_valencia():
    cfg = W.RunConfig(K=100.0, Gamma=2.0, Gamma_th=5.0 / 3.0)
    rng = np.random.default_rng(21)
    for _ in range(40):
        Wc, h = W.random_conformal_metric(rng, 0.15)
        gt = np.eye(3) + _sym(h)
        gti = np.linalg.inv(gt)
        # derivatives of gt that keep det gt = 1: trace-free with respect to gt
        dh = rng.uniform(-0.05, 0.05, (2, 6))
        for e in range(2):
            m = _sym(dh[e])
            m -= gt * np.einsum("ij,ij", gti, m) / 3.0
            dh[e] = [m[0, 0], m[0, 1], m[0, 2], m[1, 1], m[1, 2], m[2, 2]]
        al = rng.uniform(0.5, 1.0)
        dal = rng.uniform(-0.1, 0.1, 2)
        dW = rng.uniform(-0.1, 0.1, 2)
        db = rng.uniform(-0.1, 0.1, (2, 3))
        A = rng.uniform(-0.05, 0.05, 6)
        K = rng.uniform(-0.1, 0.1)
        rho = 10 ** rng.uniform(-4, -2)
        P = 100 * rho * rho * rng.uniform(1.0, 3.0)
        u = rng.uniform(-1.5, 1.5, 3)
        prim = np.array([rho, *u, P, O.eos_eps(cfg, rho, P)])
        src = O.hydro_source(cfg, prim, al, 0.0, Wc, h, A, K, dal, db, dW, dh, 0.0)

        gam = gt / Wc ** 2
        gami = np.linalg.inv(gam)
        w = math.sqrt(1.0 + u @ gami @ u)
        hh = 1.0 + prim[5] + P / rho
        vd = u / w
        vu = gami @ vd
        E = rho * hh * w * w - P
        Sd = rho * hh * w * w * vd
        Sup = rho * hh * w * w * np.outer(vu, vu) + P * gami
        Kij = (_sym(A) + gt * K / 3.0) / Wc ** 2
        sqg = Wc ** -3
        ref = []
        for e in range(2):
            dgam = _sym(dh[e]) / Wc ** 2 - 2.0 * gt * dW[e] / Wc ** 3
            ref.append(sqg * (0.5 * al * np.einsum("ik,ik", Sup, dgam) + Sd @ db[e] - E * dal[e]))
        dalpha3 = np.array([dal[0], 0.0, dal[1]])
        sE = sqg * (al * np.einsum("ij,ij", Sup, Kij) - (gami @ Sd) @ dalpha3)
        scale = max(abs(ref[0]), abs(ref[1]), abs(sE), 1e-300)
        assert abs(src[1] - ref[0]) < 1e-12 * scale
        assert abs(src[3] - ref[1]) < 1e-12 * scale
        assert abs(src[4] - sE) < 1e-12 * scale
        assert src[0] == 0.0 and src[2] == 0.0


def test_geometric_source_balances_pressure_at_rest():
    # at rest, alpha W^-3 P / x: the area difference of the pressure flux
    cfg = W.RunConfig()
    prim = np.array([1e-3, 0, 0, 0, 2e-4, 0.0])
    prim[5] = O.eos_eps(cfg, 1e-3, 2e-4)
    z2 = np.zeros(2)
    s = O.hydro_source(cfg, prim, 0.8, 0.0, 0.9, np.zeros(6), np.zeros(6), 0.0, z2, np.zeros((2, 3)), z2,
                       np.zeros((2, 6)), 2.5)
    assert abs(s[1] - 0.8 * 0.9 ** -3 * 2e-4 / 2.5) < 1e-18
