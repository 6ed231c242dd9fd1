"""Pin of the oracle's pointwise Z4c right-hand side (Eq. bssn, Eq. K,
Eq. moving_puncture) against the textbook ADM evolution equations.

For data with Theta = 0 and Gt^i = -d_j gt^ij (det gt = 1 by construction),
the Z4c equations must reproduce exactly
  d_t gamma_ij = -2 alpha K_ij + L_beta gamma_ij,
  d_t K_ij = -D_i D_j alpha + alpha (R_ij - 2 K_ik K^k_j + K K_ij)
             - 8 pi alpha (S_ij - gamma_ij (S - E) / 2) + L_beta K_ij,
  d_t Theta = alpha H / 2,
  d_t Gt^i = -d_j (d_t gt^ij) + 2 alpha gt^ik M_k,
with H and M_k the Hamiltonian and momentum constraints.  The derivatives of
a generic analytic metric are exact to ~1e-30; the ADM side is assembled
here from the Christoffel symbols of gamma_ij (an independent route from the
conformal decomposition the oracle uses).  Exact derivatives come from central
differences in 80-digit arithmetic (mpmath)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2502_03223_gb300 import workloads as W

mp = pytest.importorskip("mpmath")

S6 = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]
PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
PI = math.pi
H1 = mp.mpf("1e-15")   # outer difference step (80-digit arithmetic)
H2 = mp.mpf("1e-22")   # inner difference step


def _d1(f, p, k, h):
    a = list(p); b = list(p)
    a[k] += h; b[k] -= h
    return (f(a) - f(b)) / (2 * h)


def _d2(f, p, k, l, h):
    if k == l:
        a = list(p); b = list(p)
        a[k] += h; b[k] -= h
        return (f(a) - 2 * f(p) + f(b)) / (h * h)
    pp, pm, mp_, mm = list(p), list(p), list(p), list(p)
    pp[k] += h; pp[l] += h; pm[k] += h; pm[l] -= h; mp_[k] -= h; mp_[l] += h; mm[k] -= h; mm[l] -= h
    return (f(pp) - f(pm) - f(mp_) + f(mm)) / (4 * h * h)


@pytest.fixture(scope="module")
def setup():
    """A generic analytic 3+1 data set (quadratic-plus polynomials with random
    coefficients, no symmetry) and exact derivatives at one point, obtained by
    central differences in 80-digit arithmetic (truncation ~1e-30)."""
    mp.mp.dps = 80
    rng = np.random.default_rng(11)

    def mons(p):
        x, y, z = p
        return [1, x, y, z, x * x, y * y, z * z, x * y, x * z, y * z, x * y * z]

    def mkpoly(c0, amp):
        c = [mp.mpf(float(v)) for v in rng.uniform(-amp, amp, 11)]
        return lambda p: c0 + sum(ci * m for ci, m in zip(c, mons(p)))

    gam_p = {}
    K_p = {}
    for i, j in PAIRS:
        gam_p[(i, j)] = mkpoly(1 if i == j else 0, 0.08)
        K_p[(i, j)] = mkpoly(0, 0.1)
    alpha_p = mkpoly(1, 0.1)
    beta_p = [mkpoly(0, 0.1) for _ in range(3)]
    B_p = [mkpoly(0, 0.1) for _ in range(3)]

    def sym(pd, p):
        m = mp.matrix(3, 3)
        for (i, j), f in pd.items():
            m[i, j] = m[j, i] = f(p)
        return m

    def gti_of(p):
        # gt^ij = gamma^ij / W^2 = gamma^ij det(gamma)^(1/3)
        g = sym(gam_p, p)
        return mp.inverse(g) * mp.det(g) ** (mp.mpf(1) / 3)

    def gt_inv_entry(i, j):
        return lambda p: gti_of(p)[i, j]

    def fields(p):
        g = sym(gam_p, p)
        K = sym(K_p, p)
        dg = mp.det(g)
        Wv = dg ** (-mp.mpf(1) / 6)
        gi = mp.inverse(g)
        Ktr = sum(gi[i, j] * K[i, j] for i in range(3) for j in range(3))
        out = [Wv]
        for (i, j) in PAIRS:
            out.append(Wv * Wv * g[i, j] - (1 if i == j else 0))
        for (i, j) in PAIRS:
            out.append(Wv * Wv * (K[i, j] - g[i, j] * Ktr / 3))
        out.append(Ktr)
        for i in range(3):
            out.append(-sum(_d1(gt_inv_entry(i, j), p, j, H2) for j in range(3)))
        out.append(mp.mpf(0))
        out.append(alpha_p(p))
        out += [b(p) for b in beta_p]
        out += [b(p) for b in B_p]
        return out

    p0 = [mp.mpf("0.31"), mp.mpf("0.22"), mp.mpf("-0.17")]
    F0 = fields(p0)
    Q = np.array([float(v) for v in F0])
    cache = {}

    def fcall(p):
        key = tuple(mp.nstr(v, 60) for v in p)
        if key not in cache:
            cache[key] = fields(p)
        return cache[key]

    dQ = np.zeros((25, 3))
    ddQ = np.zeros((25, 6))
    for k in range(3):
        vals = [(a - b) / (2 * H1) for a, b in zip(fcall([p0[m] + (H1 if m == k else 0) for m in range(3)]),
                                                    fcall([p0[m] - (H1 if m == k else 0) for m in range(3)]))]
        dQ[:, k] = [float(v) for v in vals]
    for a_, (k, l) in enumerate(PAIRS):
        for f in range(25):
            ddQ[f, a_] = float(_d2(lambda p, f=f: fcall(p)[f], p0, k, l, H1))

    def jet(fun):
        v = fun(p0)
        d = [_d1(fun, p0, k, H1) for k in range(3)]
        dd = [[_d2(fun, p0, k, l, H1) for l in range(3)] for k in range(3)]
        return float(v), np.array([float(t) for t in d]), np.array([[float(t) for t in r] for r in dd])

    g0 = np.zeros((3, 3)); dg = np.zeros((3, 3, 3)); ddg = np.zeros((3, 3, 3, 3))
    K0 = np.zeros((3, 3)); dK = np.zeros((3, 3, 3))
    for (i, j) in PAIRS:
        v, d, dd = jet(gam_p[(i, j)])
        g0[i, j] = g0[j, i] = v
        dg[:, i, j] = dg[:, j, i] = d
        ddg[:, :, i, j] = ddg[:, :, j, i] = dd
        v, d, _ = jet(K_p[(i, j)])
        K0[i, j] = K0[j, i] = v
        dK[:, i, j] = dK[:, j, i] = d
    a0, da, dda = jet(alpha_p)
    b0 = np.zeros(3); db = np.zeros((3, 3))
    for i in range(3):
        v, d, _ = jet(beta_p[i])
        b0[i] = v
        db[:, i] = d

    # d_t gt^ij from the ADM d_t gamma_ij at any point, for -d_j d_t gt^ij
    def dtgti(p):
        g = sym(gam_p, p)
        K = sym(K_p, p)
        al = alpha_p(p)
        be = [b(p) for b in beta_p]
        dgm = [[[_d1(gam_p[tuple(sorted((i, j)))], p, k, H2) for j in range(3)] for i in range(3)] for k in range(3)]
        dbe = [[_d1(beta_p[i], p, k, H2) for i in range(3)] for k in range(3)]
        dtg = mp.matrix(3, 3)
        for i in range(3):
            for j in range(3):
                e = -2 * al * K[i, j]
                for k in range(3):
                    e += be[k] * dgm[k][i][j] + g[k, j] * dbe[i][k] + g[i, k] * dbe[j][k]
                dtg[i, j] = e
        gi = mp.inverse(g)
        Wv = mp.det(g) ** (-mp.mpf(1) / 6)
        dtW = -Wv / 6 * sum(gi[c, d] * dtg[c, d] for c in range(3) for d in range(3))
        dtgt = dtg * Wv * Wv + g * (2 * Wv * dtW)
        gti = gi / (Wv * Wv)
        return -(gti * dtgt * gti)

    div = np.zeros(3)
    for i in range(3):
        div[i] = float(sum(_d1(lambda p, i=i, j=j: dtgti(p)[i, j], p0, j, H1) for j in range(3)))

    rng2 = np.random.default_rng(12)
    E = rng2.uniform(0, 0.05)
    Si = rng2.uniform(-0.02, 0.02, 3)
    Sm = rng2.uniform(-0.02, 0.02, (3, 3))
    Sij = 0.5 * (Sm + Sm.T)
    return dict(Q=Q, dQ=dQ, ddQ=ddQ, g=g0, dg=dg, ddg=ddg, K=K0, dK=dK, a=a0, da=da, dda=dda, b=b0, db=db,
                div=div, E=E, Si=Si, Sij=Sij, Bv=Q[22:25])


def _adm(s):
    g, dg, ddg = s["g"], s["dg"], s["ddg"]
    gi = np.linalg.inv(g)
    # Gamma^k_ij and its derivative
    Gam = 0.5 * (np.einsum("kl,ilj->kij", gi, dg) + np.einsum("kl,jli->kij", gi, dg)
                 - np.einsum("kl,lij->kij", gi, dg))
    dgi = -np.einsum("ka,mab,lb->mkl", gi, dg, gi)           # d_m gamma^kl
    dGam = 0.5 * (np.einsum("mkl,ilj->mkij", dgi, dg) + np.einsum("mkl,jli->mkij", dgi, dg)
                  - np.einsum("mkl,lij->mkij", dgi, dg)) \
        + 0.5 * (np.einsum("kl,milj->mkij", gi, ddg) + np.einsum("kl,mjli->mkij", gi, ddg)
                 - np.einsum("kl,mlij->mkij", gi, ddg))
    # R_ij = d_k Gam^k_ij - d_j Gam^k_ik + Gam^k_kl Gam^l_ij - Gam^k_jl Gam^l_ik
    R = np.einsum("kkij->ij", dGam) - np.einsum("jkik->ij", dGam) \
        + np.einsum("kkl,lij->ij", Gam, Gam) - np.einsum("kjl,lik->ij", Gam, Gam)
    K = s["K"]
    Ktr = np.einsum("ij,ij", gi, K)
    Kmix = gi @ K                                              # K^k_j
    DDa = s["dda"] - np.einsum("kij,k->ij", Gam, s["da"])
    S = np.einsum("ij,ij", gi, s["Sij"])
    a = s["a"]
    b, db = s["b"], s["db"]
    dK = s["dK"]
    Lg = np.einsum("k,kij->ij", b, dg) + np.einsum("kj,ik->ij", g, db) + np.einsum("ik,jk->ij", g, db)
    LK = np.einsum("k,kij->ij", b, dK) + np.einsum("kj,ik->ij", K, db) + np.einsum("ik,jk->ij", K, db)
    dtg = -2 * a * K + Lg
    dtK = -DDa + a * (R - 2 * K @ Kmix + Ktr * K) - 8 * PI * a * (s["Sij"] - 0.5 * g * (S - s["E"])) + LK
    H = np.einsum("ij,ij", gi, R) + Ktr ** 2 - np.einsum("ij,ij", K, gi @ K @ gi) - 16 * PI * s["E"]
    # M_i = D_j K^j_i - D_i K - 8 pi S_i
    Kup = gi @ K                                     # K^j_i  as [j][i]
    dKup = np.einsum("mja,ai->mji", dgi, K) + np.einsum("ja,mai->mji", gi, dK)
    divK = np.einsum("jji->i", dKup) + np.einsum("jjl,li->i", Gam, Kup) - np.einsum("lji,jl->i", Gam, Kup)
    dKtr = np.einsum("mij,ij->m", dgi, K) + np.einsum("ij,mij->m", gi, dK)
    M = divK - dKtr - 8 * PI * s["Si"]
    return dict(R=R, dtg=dtg, dtK=dtK, H=H, M=M, gi=gi)


def _oracle_rhs(s, kappa=0.3, eta=0.7, bssn=0, Q=None):
    cfg = W.RunConfig(kappa=kappa, eta_B=eta, bssn=bssn)
    Q = s["Q"] if Q is None else Q
    dQ, ddQ = s["dQ"], s["ddQ"]
    adv = dQ @ Q[19:22]
    Sij6 = np.array([s["Sij"][i, j] for i, j in PAIRS])
    return O.z4c_point(cfg, Q, dQ, ddQ, adv, s["E"], s["Si"], Sij6, 1.0), adv


def test_ricci_matches_christoffel_definition(setup):
    R = O.ricci_point(setup["Q"], setup["dQ"], setup["ddQ"])
    ref = _adm(setup)["R"]
    for a, (i, j) in enumerate(PAIRS):
        assert abs(R[a] - ref[i, j]) < 1e-11 * (1 + abs(ref[i, j])), (i, j, R[a], ref[i, j])


@pytest.mark.parametrize("bssn", [0, 1])
def test_metric_and_curvature_evolution_match_adm(setup, bssn):
    """Z4c, and the BSSN formulation (Theta frozen at zero, no damping) used
    for the cleaner waveform of Sec. III.C.  With Theta = 0 Z4c reproduces the
    ADM equations for gamma_ij and K_ij (its Theta equation carries the alpha H
    that ADM's d_t K has); BSSN's d_t K is ADM's with the Hamiltonian
    constraint substituted, so its d_t K_ij is ADM's minus gamma_ij alpha H / 3,
    whatever kappa is set to."""
    s = setup
    r, adv = _oracle_rhs(s, bssn=bssn)
    ref = _adm(s)
    Q = s["Q"]
    Wc = Q[0]
    gt = np.eye(3) + np.array([[Q[1 + S6[i][j]] for j in range(3)] for i in range(3)])
    At = np.array([[Q[7 + S6[i][j]] for j in range(3)] for i in range(3)])
    dgt = np.array([[r[1 + S6[i][j]] for j in range(3)] for i in range(3)])
    dAt = np.array([[r[7 + S6[i][j]] for j in range(3)] for i in range(3)])
    dW = r[0]
    K = Q[13] + 2 * Q[17]
    dKt = r[13] + 2 * r[17]
    dtg = dgt / Wc ** 2 - 2 * gt * dW / Wc ** 3
    dtK = (dAt + dgt * K / 3 + gt * dKt / 3) / Wc ** 2 - 2 * (At + gt * K / 3) * dW / Wc ** 3
    assert np.allclose(dtg, ref["dtg"], rtol=0, atol=1e-12)
    expect_K = ref["dtK"] - (s["g"] * s["a"] * ref["H"] / 3 if bssn else 0.0)
    assert np.allclose(dtK, expect_K, rtol=0, atol=1e-11)
    if bssn:
        assert r[17] == 0.0
    else:
        # Theta: alpha H / 2 (damping factor 1, Theta = 0)
        assert abs(r[17] - 0.5 * s["a"] * ref["H"]) < 1e-11


@pytest.mark.parametrize("bssn", [0, 1])
def test_gamma_tilde_evolution_matches_constraint_identity(setup, bssn):
    s = setup
    r, adv = _oracle_rhs(s, bssn=bssn)
    ref = _adm(s)
    Q = s["Q"]
    gt = np.eye(3) + np.array([[Q[1 + S6[i][j]] for j in range(3)] for i in range(3)])
    gti = np.linalg.inv(gt)
    expect = -s["div"] + 2 * s["a"] * gti @ ref["M"]
    assert np.allclose(r[14:17], expect, rtol=0, atol=1e-9), (r[14:17], expect)


def test_gauge_equations(setup):
    s = setup
    eta = 0.7
    r, adv = _oracle_rhs(s, eta=eta)
    Q = s["Q"]
    assert abs(r[18] - (adv[18] - 2 * Q[18] * Q[13])) < 1e-14
    assert np.allclose(r[19:22], adv[19:22] + 0.75 * Q[22:25], atol=1e-15)
    gsrc = r[14:17] - adv[14:17]
    assert np.allclose(r[22:25], adv[22:25] + gsrc - eta * Q[22:25], atol=1e-15)


def test_constraints_match_textbook(setup):
    s = setup
    H, M = O.constraints_point(s["Q"], s["dQ"], s["ddQ"], s["E"], s["Si"])
    ref = _adm(s)
    assert abs(H - ref["H"]) < 1e-11
    assert np.allclose(M, ref["M"], atol=1e-11)


def test_minkowski_rhs_vanishes_exactly():
    Q = np.zeros(25); Q[0] = 1.0; Q[18] = 1.0
    r = O.z4c_point(W.RunConfig(kappa=0.1), Q, np.zeros((25, 3)), np.zeros((25, 6)), np.zeros(25), 0.0,
                    np.zeros(3), np.zeros(6), 1.0)
    assert np.all(r == 0.0)


def test_damping_terms_and_their_absence_in_bssn(setup):
    """The kappa terms of Eq. bssn are linear in kappa: with Gt^i = Gd^i + delta^i
    (delta constant near the point) and Theta = th, Z4c(kappa) - Z4c(0) is
    alpha kappa th in K-hat, -2 alpha kappa delta^i in Gt^i and in B^i (the
    Gamma-driver's source is d_t Gt^i, Eq. moving_puncture) and -2 alpha kappa th
    in Theta, nothing elsewhere.  The BSSN setting drops exactly those terms and
    freezes Theta: it equals Z4c at kappa = 0 except Theta's right-hand side,
    which is zero."""
    s = setup
    Q = s["Q"].copy()
    delta = np.array([0.013, -0.021, 0.008])
    th = 0.017
    Q[14:17] += delta
    Q[17] = th
    kap = 0.3
    a = Q[18]
    r_k, _ = _oracle_rhs(s, kappa=kap, Q=Q)
    r_0, _ = _oracle_rhs(s, kappa=0.0, Q=Q)
    r_b, _ = _oracle_rhs(s, kappa=kap, bssn=1, Q=Q)
    d = r_k - r_0
    expect = np.zeros(25)
    expect[13] = a * kap * th
    expect[14:17] = -2 * a * kap * delta
    expect[22:25] = -2 * a * kap * delta
    expect[17] = -2 * a * kap * th
    assert np.allclose(d, expect, rtol=0, atol=1e-13), (d, expect)
    assert r_b[17] == 0.0
    keep = np.arange(25) != 17
    assert np.array_equal(r_b[keep], r_0[keep])


def test_bssn_keeps_theta_zero_on_the_grid():
    """The BSSN switch on a whole two-level hierarchy of the stable star (with
    a random metric perturbation so that the constraints do not vanish): Theta
    stays exactly zero through the stages, the ghost fill, the prolongation and
    the restriction, and the Z4c run from the same data does grow a Theta."""
    import dataclasses
    cfg, tov = W.tov_config("bssn", rho_c=1.28e-3, n_levels=2, N=16, dx_fine=1.0, rk=1)
    datas = []
    for l in range(2):
        d = W.tov_level_data(cfg, tov, l)
        d[:25] += W.random_metric_perturbation(cfg, l, np.random.default_rng(5), amp=1e-3)
        d[17] = 0.0
        datas.append(d)
    runs = {}
    for bssn in (0, 1):
        c = dataclasses.replace(cfg, bssn=bssn)
        o = O.Oracle(c)
        for l, d in enumerate(datas):
            o.set_level(l, 0, d)
        o.step(c.dt, 3)
        runs[bssn] = [o.read(l, 0, 17) for l in range(2)]
        for l in range(2):
            assert np.all(np.isfinite(o.read(l, 0, 0)))
    for l in range(2):
        assert not np.any(runs[1][l]), l
        assert np.max(np.abs(runs[0][l])) > 1e-8, l
