"""Pins of four oracle parts against what the paper and the mathematics fix,
with no GPU:

* the outer boundary condition of the metric (Sec. II.B.3: Q - Q_inf carried
  outward as an outgoing spherical wave, Q(r, t + tau) - Q_inf =
  (1 - tau / r) (Q - Q_inf)(r - tau, t)), which is exact for Q - Q_inf =
  f(t - r) / r: the ghost values converge to the wave at the order of the
  radial interpolation;
* the prolongation of the primitives into a child's buffer zone (Sec. II.D,
  minmod-limited linear): linear data is reproduced exactly, at a kink the
  smaller one-sided slope is taken and at an extremum none;
* the time interpolation of a parent's data for a sub-cycled child (Sec.
  II.D, second order through t^{n-1}, t^n, t^{n+1}): exact on data quadratic
  in t, first order through t^n, t^{n+1} for a primitive whose three values
  are not monotone, first order everywhere without a t^{n-1} slice;
* the volume reductions of Sec. II.F.1: M_b = int W^-3 rho w dV and
  J = int W^-3 rho h w u_y x dV with dV = 2 pi x dx dz over the cells not
  covered by a finer level, and the L2 norm of the Hamiltonian constraint
  (read as sqrt(int H^2 dV / int dV)), against quadrature of closed forms."""
import dataclasses

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2502_03223_gb300 import workloads as W

G = 8
IW, IAL, IBX, IBZ = 0, 18, 19, 21          # W, alpha, beta^x, beta^z
QD, QSY = 25, 27


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def _cfg(N, L=1, X=32.0, rk=0, **kw):
    return dataclasses.replace(W.RunConfig(), name="pin", n_levels=L, nx=N, nz=N, geometry=1, evolve_spacetime=1,
                               rk=rk, dx0=X / N, dz0=X / N, rho_atm=1e-30, **kw)


def _centres(cfg, level):
    X, Z = W.cell_centres(cfg, level)
    return X, Z


def _flat_data(cfg, level, rho=1e-12, P=None):
    X, Z = _centres(cfg, level)
    d = np.zeros((30,) + X.shape)
    d[IW] = 1.0
    d[IAL] = 1.0
    d[25] = rho
    d[29] = cfg.K * rho ** cfg.Gamma * 3.0 if P is None else P
    return d


# ---------------------------------------------------------------- outer boundary (Sec. II.B.3)

def _pulse(s, A=1.0, r0=34.0, sig=3.0):
    """f(t - r) of an outgoing spherical wave, centred at r = r0 at t = 0."""
    return A * np.exp(-((s + r0) ** 2) / sig ** 2)


def _outer_error(N):
    cfg = _cfg(N)
    X, Z = _centres(cfg, 0)
    r = np.sqrt(X ** 2 + Z ** 2)
    d = _flat_data(cfg, 0)
    amps = {IW: 0.3, IAL: -0.2, IBX: 0.1, IBZ: 0.05}
    for f, a in amps.items():
        d[f] = (1.0 if f in (IW, IAL) else 0.0) + a * _pulse(-r) / r
    o = O.Oracle(cfg)
    o.set_level(0, 0, d)
    dt = 0.5 * cfg.dx0
    s = 1                                   # RK4 stage 1: tau = c_1 dt = dt / 2
    tau = 0.5 * dt
    o.fill(s, dt)
    ghost = np.zeros_like(r, dtype=bool)
    ghost[G:, G:] = True                    # j, k >= 1 ...
    ghost[G:G + N, G:G + N] = False         # ... outside the interior
    err = 0.0
    for f, a in amps.items():
        got = o.read(0, 1, f)
        qinf = 1.0 if f in (IW, IAL) else 0.0
        exact = qinf + a * _pulse(tau - r) / r
        err = max(err, float(np.max(np.abs(got - exact)[ghost])) / abs(a))
    o.close()
    return err


def test_outer_boundary_carries_an_outgoing_spherical_wave():
    """The ghost values equal the wave one sub-step later up to the error of
    the 3 x 3 Lagrange interpolation along the radial line (order 3 in the
    spacing, with tau proportional to it).  A plus sign in (1 - tau / r), a
    tau other than c_s dt, or Q_inf left out of W or alpha leaves an O(dx)
    error and order 1."""
    errs = [_outer_error(N) for N in (32, 64, 128)]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-5, errs
    assert min(orders) > 2.2 and orders[-1] > 2.8, (errs, orders)


# ---------------------------------------------------------------- hydro prolongation (Sec. II.D)

def _prolonged_prims(N, rho_fn, u_fn, P_fn):
    """Two levels; the parent holds the given primitive fields, the child's
    buffer zone [N+1, N+8] is filled by the stage-0 ghost fill.  Returns the
    child's primitive planes and cell centres."""
    cfg = _cfg(N, L=2, X=float(N))          # parent dx = 1, child dx = 1/2
    datas = []
    for l in range(2):
        X, Z = _centres(cfg, l)
        d = _flat_data(cfg, l)
        d[25] = rho_fn(X, Z)
        for i in range(3):
            d[26 + i] = u_fn[i](X, Z)
        d[29] = P_fn(X, Z)
        datas.append(d)
    o = O.Oracle(cfg)
    for l, d in enumerate(datas):
        o.set_level(l, 0, d)
    o.fill(0, 0.5 * cfg.dx(1))
    prims = [o.read(1, 2, f) for f in range(5)]
    Xc, Zc = _centres(cfg, 1)
    o.close()
    return cfg, prims, Xc, Zc


def _buffer_mask(N):
    m = np.zeros((N + 2 * G, N + 2 * G), dtype=bool)
    m[G:, G:] = True
    m[G:G + N, G:G + N] = False
    return m


def test_hydro_prolongation_reproduces_linear_primitives():
    N = 32
    rho = lambda x, z: 1e-3 + 2e-5 * x + 1e-5 * z
    u = [lambda x, z: 0.01 + 1e-3 * x - 2e-3 * z, lambda x, z: -0.02 + 5e-4 * x, lambda x, z: 3e-3 * z - 1e-3 * x]
    P = lambda x, z: 1e-3 + 1e-5 * x + 2e-5 * z       # well above the cold curve K rho^2 ~ 1e-4
    cfg, prims, X, Z = _prolonged_prims(N, rho, u, P)
    m = _buffer_mask(N)
    # children of parent cell 1 (child index 1, 2) next to the axis or the
    # equator see the mirrored profile (a kink at the symmetry plane), where
    # minmod takes no slope: left out here
    m[:G + 2, :] = False
    m[:, :G + 2] = False
    exact = [rho(X, Z)] + [ui(X, Z) for ui in u] + [P(X, Z)]
    for f in range(5):
        np.testing.assert_allclose(prims[f][m], exact[f][m], rtol=1e-13, atol=1e-17, err_msg=str(f))


@pytest.mark.parametrize("axis", ["x", "z"])
def test_hydro_prolongation_minmod_at_a_kink_and_an_extremum(axis):
    """rho piecewise linear in one coordinate with a corner at the centre of
    parent cell m0 = N/2 + 2 (its children lie in the buffer zone): with
    one-sided slopes g and 3g the child values use g (the smaller); with g
    and -g (a peak) they equal the parent value.  A central or MC slope would
    give 2g at the corner."""
    N, g, rho0 = 32, 1e-5, 1e-3
    m0 = N // 2 + 2
    c0 = m0 - 0.5                            # parent dx = 1
    pick = (lambda x, z: x) if axis == "x" else (lambda x, z: z)
    for sR, expect_slope in ((3 * g, g), (-g, 0.0)):
        rho = lambda x, z, sR=sR: rho0 + np.where(pick(x, z) < c0, g * (pick(x, z) - c0), sR * (pick(x, z) - c0))
        zero = lambda x, z: 0.0 * x
        cfg, prims, X, Z = _prolonged_prims(N, rho, [zero, zero, zero], lambda x, z: 1e-3 + 0.0 * x)
        # child cells whose parent is m0: child index 2 m0 - 1 (offset -1/4), 2 m0 (+1/4)
        for jc, off in ((2 * m0 - 1, -0.25), (2 * m0, 0.25)):
            if axis == "x":
                vals = prims[0][G + 2:G + N, G + jc - 1]        # k in the interior rows, j = jc
            else:
                vals = prims[0][G + jc - 1, G + 2:G + N]
            np.testing.assert_allclose(vals, rho0 + off * expect_slope, rtol=0, atol=1e-17)
        # one parent cell further right: both slopes equal sR -> exact linear
        jc = 2 * m0 + 2
        vals = prims[0][G + 2:G + N, G + jc - 1] if axis == "x" else prims[0][G + jc - 1, G + 2:G + N]
        xc = (jc - 0.5) * 0.5
        np.testing.assert_allclose(vals, rho0 + sR * (xc - c0), rtol=1e-13, atol=1e-18)


# ---------------------------------------------------------------- time interpolation (Sec. II.D)

def _slices(cfg, rng):
    shape = (cfg.pz, cfg.px)
    a = rng.normal(size=(31,) + shape)
    b = rng.normal(size=(31,) + shape)
    c = rng.normal(size=(31,) + shape)
    q = lambda t: a + b * t + c * t * t
    return a, b, c, q


@pytest.mark.parametrize("theta", [0.25, 0.5, 0.625, 0.75, 1.0])
def test_time_interpolation_is_exact_on_quadratics_and_drops_to_linear(theta):
    cfg = _cfg(16)
    rng = np.random.default_rng(11)
    a, b, c, q = _slices(cfg, rng)
    old, now, new = q(-1.0), q(0.0), q(1.0)
    o = O.Oracle(cfg)
    met, pr = o.time_interp(0, theta, 1, old[:25], now[:25], new[:25], old[25:], now[25:], new[25:])
    # metric: second order through the three slices, exact on quadratics in t
    np.testing.assert_allclose(met, q(theta)[:25], rtol=1e-13, atol=1e-13)
    # primitives: the quadratic where (p1 - p0)(p0 - p_old) >= 0, else linear through t^n, t^{n+1}
    p_old, p0, p1 = old[25:], now[25:], new[25:]
    mono = (p1 - p0) * (p0 - p_old) >= 0
    assert mono.any() and (~mono).any()
    lin = p0 + theta * (p1 - p0)
    np.testing.assert_allclose(pr[mono], q(theta)[25:][mono], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pr[~mono], lin[~mono], rtol=1e-13, atol=1e-13)
    assert np.max(np.abs(pr[~mono] - q(theta)[25:][~mono])) > 1e-3 or theta == 1.0
    # without a t^{n-1} slice: first order everywhere
    met1, pr1 = o.time_interp(0, theta, 0, old[:25], now[:25], new[:25], old[25:], now[25:], new[25:])
    np.testing.assert_allclose(met1, now[:25] + theta * (new[:25] - now[:25]), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pr1, lin, rtol=1e-13, atol=1e-13)
    o.close()


# ---------------------------------------------------------------- reductions of Sec. II.F.1

def _conformal_data(cfg, level, A=0.3, sig=6.0, rho=1e-6, Omega=0.0):
    X, Z = _centres(cfg, level)
    r2 = X ** 2 + Z ** 2
    psi = 1.0 + A * np.exp(-r2 / sig ** 2)
    d = _flat_data(cfg, level, rho=rho, P=1e-9)
    d[IW] = psi ** -2
    d[27] = Omega * X                     # u_y = Omega x: rigid rotation
    return d


def _oracle_diag(cfg, **kw):
    o = O.Oracle(cfg)
    for l in range(cfg.n_levels):
        o.set_level(l, 0, _conformal_data(cfg, l, **kw))
    d = o.diag()
    o.close()
    return d


@pytest.mark.parametrize("L", [1, 2])
def test_baryon_mass_and_angular_momentum_integrals(L):
    """M_b = int W^-3 rho w dV and J = int W^-3 rho h w u_y x dV over the
    domain [0, X] x [0, Z] (dV = 2 pi x dx dz) for uniform rho, P, rigid
    rotation u_y = Omega x and a conformal factor W = psi^-2: the sums over
    non-covered cells converge at second order (midpoint rule) to the
    quadrature of the closed-form integrands, on one and on two levels."""
    X = 32.0
    A, sig, rho, Om, P = 0.3, 6.0, 1e-6, 0.01, 1e-9
    cfgp = _cfg(32, L=L, X=X)
    eps = O.eos_eps(cfgp, rho, P)
    h = 1.0 + eps + P / rho
    psi6 = lambda x, z: (1.0 + A * np.exp(-(x * x + z * z) / sig ** 2)) ** 6

    def wlor(x, z):          # w = sqrt(1 + gamma^yy u_y^2), gamma^yy = psi^-4 = W^2
        return np.sqrt(1.0 + (Om * x) ** 2 / psi6(x, z) ** (2.0 / 3.0))
    mb_ex = integrate.dblquad(lambda x, z: 2 * np.pi * x * psi6(x, z) * rho * wlor(x, z), 0, X, 0, X,
                              epsabs=0, epsrel=1e-12)[0]
    j_ex = integrate.dblquad(lambda x, z: 2 * np.pi * x * psi6(x, z) * rho * h * wlor(x, z) * Om * x * x, 0, X, 0, X,
                             epsabs=0, epsrel=1e-12)[0]
    emb, ej = [], []
    for N in (32, 64, 128):
        d = _oracle_diag(_cfg(N, L=L, X=X), A=A, sig=sig, rho=rho, Omega=Om)
        emb.append(abs(d[4] - mb_ex) / mb_ex)
        ej.append(abs(d[5] - j_ex) / j_ex)
    for e in (emb, ej):
        orders = [np.log2(e[i] / e[i + 1]) for i in range(2)]
        assert e[-1] < 1e-4 and min(orders) > 1.8, (e, orders)


def test_uniform_mass_is_exact_over_covered_levels():
    """A uniform rest-mass density on a flat metric: the midpoint rule is exact
    for the linear integrand 2 pi x, so M_b = rho pi X^2 Z to round-off on one
    level and on three (the covered parent cells counted once)."""
    X, rho = 32.0, 1e-4
    for L in (1, 3):
        cfg = _cfg(32, L=L, X=X)
        o = O.Oracle(cfg)
        for l in range(L):
            o.set_level(l, 0, _flat_data(cfg, l, rho=rho, P=1e-7))
        d = o.diag()
        o.close()
        assert abs(d[4] - rho * np.pi * X ** 3) < 1e-13 * d[4], (L, d[4])
        assert d[5] == 0.0


def test_hamiltonian_constraint_l2_norm():
    """Time-symmetric conformally flat vacuum data, gamma_ij = psi^4 delta_ij
    with psi = 1 + A exp(-r^2 / sigma^2) (K = At = 0): H = R = -8 psi^-5
    lap(psi).  ||H||_2 = sqrt(int H^2 dV / int dV) over the computational
    domain converges to the quadrature of that closed form (midpoint rule:
    second order), on one level and on two; the momentum constraints vanish."""
    X, A, sig = 32.0, 0.3, 6.0

    def R(x, z):
        r2 = x * x + z * z
        e = np.exp(-r2 / sig ** 2)
        psi = 1.0 + A * e
        lap = A * e * (4.0 * r2 / sig ** 4 - 6.0 / sig ** 2)
        return -8.0 * lap / psi ** 5
    num = integrate.dblquad(lambda x, z: 2 * np.pi * x * R(x, z) ** 2, 0, X, 0, X, epsabs=0, epsrel=1e-12)[0]
    h_ex = np.sqrt(num / (np.pi * X ** 3))
    for L in (1, 2):
        errs = []
        for N in (32, 64, 128):
            d = _oracle_diag(_cfg(N, L=L, X=X), A=A, sig=sig, rho=1e-20)
            errs.append(abs(d[0] - h_ex) / h_ex)
            assert max(abs(d[1]), abs(d[2]), abs(d[3])) < 1e-12 * d[0]
        orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert errs[-1] < 1e-3 and min(orders) > 1.8, (L, errs, orders)
