"""Seeded synthetic inputs for the SACRA-2D hot path.

This module only builds inputs: run configurations, initial data (the
special-relativistic shock tube, TOV stars from a plain ODE solve, smooth
random perturbations) and random states.  It holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle take their inputs from
here without sharing any of the method's code.

Units: G = c = M_sun = 1.  Level arrays are padded with 8 cells on every side:
a plane has shape (nz + 16, nx + 16) and cell (j, k) (interior j, k in
[1, n]) sits at [k + 7, j + 7], its centre at x = (j - 1/2) dx,
z = (k - 1/2) dz.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

G = 8
NMET = 25
# metric field order: W, h_ij (xx,xy,xz,yy,yz,zz), At_ij, Khat, Gt^i, Theta, alpha, beta^i, B^i
MET_NAMES = ["W", "hxx", "hxy", "hxz", "hyy", "hyz", "hzz", "Axx", "Axy", "Axz", "Ayy", "Ayz", "Azz",
             "Khat", "Gx", "Gy", "Gz", "Theta", "alpha", "betax", "betay", "betaz", "Bx", "By", "Bz"]
CONS_NAMES = ["qD", "qSx", "qSy", "qSz", "qE"]
PRIM_NAMES = ["rho", "ux", "uy", "uz", "P", "eps"]


@dataclasses.dataclass
class RunConfig:
    name: str = "custom"
    n_levels: int = 1
    nx: int = 64
    nz: int = 64
    geometry: int = 1          # 0 planar slab, 1 cylindrical (cartoon)
    evolve_spacetime: int = 1
    solver: int = 0            # 0 HLLC (TVDLF fallback), 1 TVDLF
    rk: int = 0                # 0 classical RK4, 1 SSP-RK3
    c2p_maxit: int = 100
    precision: int = 0         # 0 FP64, 1 mixed FP32/FP64 (GPU library only; the oracle is FP64)
    subcycle_from: int = 0     # 0 lockstep; K >= 1: levels >= K take half their parent's step
    hydro_outer: int = 0       # outer hydro boundary: 0 zero-gradient copy, 1 held at the initial data
    eos_adiabatic: int = 0     # 1: zero temperature (P = P_cold, eps = eps_cold), energy equation discarded
    pwp: tuple = ()            # further cold pieces: ((rho_1, Gamma_2), (rho_2, Gamma_3), ...)
    bssn: int = 0              # 1: BSSN (Theta held at zero, no constraint damping) instead of Z4c
    dx0: float = 1.0
    dz0: float = 1.0
    kappa: float = 0.0
    eta_B: float = 1.0
    eps_ko: float = 0.5
    r_z4: float = 1e300
    K: float = 100.0
    Gamma: float = 2.0
    Gamma_th: float = 2.0
    rho_atm: float = 1e-13
    w_max: float = 100.0
    c2p_tol: float = 1e-12
    r_hold: float = 0.0        # > 0: hydro held inside x^2 + z^2 < r_hold^2
    cfl: float = 0.5
    mass: float = 1.0          # total mass M used for kappa and eta_B

    @property
    def px(self):
        return self.nx + 2 * G

    @property
    def pz(self):
        return self.nz + 2 * G

    @property
    def n_stages(self):
        return 4 if self.rk == 0 else 3

    def dx(self, level):
        return self.dx0 / (1 << level)

    def dz(self, level):
        return self.dz0 / (1 << level)

    @property
    def dt(self):
        """Step of the coarse (lockstep) levels: the finest level's CFL step
        times 2 per sub-cycled level."""
        f = self.n_levels - 1
        K = self.subcycle_from
        nsub = 0 if (K <= 0 or K >= self.n_levels) else self.n_levels - K
        return self.cfl * min(self.dx(f), self.dz(f)) * (1 << nsub)

    @property
    def interior_cells(self):
        return self.n_levels * self.nx * self.nz


def cell_centres(cfg: RunConfig, level: int):
    j = np.arange(1 - G, cfg.nx + G + 1)
    k = np.arange(1 - G, cfg.nz + G + 1)
    x = (j - 0.5) * cfg.dx(level)
    z = (k - 0.5) * cfg.dz(level)
    return np.meshgrid(x, z)  # (pz, px)


def flat_metric(cfg: RunConfig):
    m = np.zeros((NMET, cfg.pz, cfg.px))
    m[0] = 1.0     # W
    m[18] = 1.0    # alpha
    return m


# ------------------------------------------------------------------ shock tube

def shock_tube_config(nx=400, nz=4, solver=0, rk=0, cfl=0.4) -> RunConfig:
    """Special-relativistic shock tube on [0, 1], Gamma-law Gamma = 5/3 (K = 0),
    flat metric frozen, outflow boundaries (Marti & Mueller problem 1 with the
    pressures 13.33 | 1e-6 of the benchmark configuration)."""
    dx = 1.0 / nx
    return RunConfig(name="shock_tube_%dx%d" % (nx, nz), n_levels=1, nx=nx, nz=nz, geometry=0, evolve_spacetime=0,
                     solver=solver, rk=rk, dx0=dx, dz0=dx, K=0.0, Gamma=5.0 / 3.0, Gamma_th=5.0 / 3.0,
                     rho_atm=1e-10, cfl=cfl)


def shock_tube_data(cfg: RunConfig, left=(10.0, 13.33, 0.0), right=(1.0, 1e-6, 0.0), x0=0.5):
    """Kind-0 level data: 25 metric planes + (rho, u_x, u_y, u_z, P)."""
    X, Z = cell_centres(cfg, 0)
    d = np.zeros((30, cfg.pz, cfg.px))
    d[:NMET] = flat_metric(cfg)
    L = X < x0
    rho = np.where(L, left[0], right[0])
    P = np.where(L, left[1], right[1])
    v = np.where(L, left[2], right[2])
    d[25] = rho
    d[26] = v / np.sqrt(1.0 - v * v)   # u_x = w v on the flat metric
    d[29] = P
    return d


# ------------------------------------------------------------------ TOV stars

@dataclasses.dataclass
class TOVSolution:
    K: float
    Gamma: float
    rho_c: float
    M: float            # gravitational mass
    Mb: float           # baryon mass
    R_areal: float
    r_iso: float        # isotropic surface radius
    r: np.ndarray       # isotropic radius table (inside)
    rho: np.ndarray
    P: np.ndarray
    psi: np.ndarray
    alpha: np.ndarray   # equilibrium lapse on the table (exterior: isotropic Schwarzschild)


def cold_pieces(K, Gamma, pwp=()):
    """Piecewise polytropic cold curve for the initial data: one entry
    (rho_lo, K_i, Gamma_i, Delta eps_i) per piece, K_(i+1) and Delta eps_(i+1)
    from continuity of P and eps at rho_i."""
    out = [(0.0, K, Gamma, 0.0)]
    for rt, g2 in pwp:
        _, k, g, d = out[-1]
        k2 = k * rt ** (g - g2)
        out.append((rt, k2, g2, d + k * rt ** (g - 1.0) / (g - 1.0) - k2 * rt ** (g2 - 1.0) / (g2 - 1.0)))
    return out


def _piece_of_rho(pieces, rho):
    i = 0
    while i + 1 < len(pieces) and rho >= pieces[i + 1][0]:
        i += 1
    return pieces[i]


def cold_P(pieces, rho):
    rho = np.asarray(rho, dtype=np.float64)
    if len(pieces) == 1:
        return pieces[0][1] * rho ** pieces[0][2]
    out = np.zeros_like(rho)
    for i, (rlo, k, g, _) in enumerate(pieces):
        rhi = pieces[i + 1][0] if i + 1 < len(pieces) else np.inf
        m = (rho >= rlo) & (rho < rhi)
        out[m] = k * rho[m] ** g
    return out


def cold_rho_of_P(pieces, P):
    """Inverse of cold_P (scalar)."""
    i = 0
    while i + 1 < len(pieces) and P >= pieces[i + 1][1] * pieces[i + 1][0] ** pieces[i + 1][2]:
        i += 1
    _, k, g, _ = pieces[i]
    return (P / k) ** (1.0 / g)


def tov_solve(K=100.0, Gamma=2.0, rho_c=1.28e-3, dR=2e-3, pwp=()) -> TOVSolution:
    """Tolman-Oppenheimer-Volkoff equilibrium of the cold curve (one
    polytrope P = K rho^Gamma, or the pieces of cold_pieces) by classical RK4
    in the areal radius R, with the isotropic radius r(R) integrated alongside
    and matched to exterior Schwarzschild at the surface."""
    pieces = cold_pieces(K, Gamma, pwp)

    def eos_e(P):
        if P <= 0.0:
            return 0.0, 0.0
        if not pwp:
            rho = (P / K) ** (1.0 / Gamma)
            return rho, rho + P / (Gamma - 1.0)
        rho = cold_rho_of_P(pieces, P)
        _, k, g, d = _piece_of_rho(pieces, rho)
        return rho, rho * (1.0 + k * rho ** (g - 1.0) / (g - 1.0) + d)

    def rhs(R, y):
        m, P, lnr, mb, nu = y
        rho, e = eos_e(P)
        if P <= 0.0:
            return np.array([0.0, 0.0, 1.0 / (R * math.sqrt(1.0 - 2.0 * m / R)), 0.0, m / (R * (R - 2.0 * m))])
        dm = 4.0 * math.pi * R * R * e
        dnu = (m + 4.0 * math.pi * R ** 3 * P) / (R * (R - 2.0 * m))
        dP = -(e + P) * dnu
        dlnr = 1.0 / (R * math.sqrt(1.0 - 2.0 * m / R))
        dmb = 4.0 * math.pi * R * R * rho / math.sqrt(1.0 - 2.0 * m / R)
        return np.array([dm, dP, dlnr, dmb, dnu])

    if not pwp:
        Pc = K * rho_c ** Gamma
        ec = rho_c + Pc / (Gamma - 1.0)
    else:
        Pc = float(cold_P(pieces, np.array([rho_c]))[0])
        ec = eos_e(Pc)[1]
    R = dR * 1e-3
    y = np.array([4.0 / 3.0 * math.pi * R ** 3 * ec, Pc, math.log(R), 4.0 / 3.0 * math.pi * R ** 3 * rho_c, 0.0])
    Rs, Ys = [R], [y.copy()]
    h = dR
    while True:
        k1 = rhs(R, y)
        k2 = rhs(R + h / 2, y + h / 2 * k1)
        k3 = rhs(R + h / 2, y + h / 2 * k2)
        k4 = rhs(R + h, y + h * k3)
        yn = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if yn[1] <= 0.0:
            if h < 1e-10:
                break
            h *= 0.5
            continue
        R += h
        y = yn
        Rs.append(R)
        Ys.append(y.copy())
        if y[1] < 1e-14 * Pc:
            break
    Rs = np.array(Rs)
    Ys = np.array(Ys)
    M = Ys[-1, 0]
    Rsurf = Rs[-1]
    rsurf = 0.5 * (Rsurf - M + math.sqrt(Rsurf * Rsurf - 2.0 * M * Rsurf))
    lnr = Ys[:, 2] - Ys[-1, 2] + math.log(rsurf)
    r = np.exp(lnr)
    P = np.maximum(Ys[:, 1], 0.0)
    rho = (P / K) ** (1.0 / Gamma) if not pwp else np.array([cold_rho_of_P(pieces, x) if x > 0 else 0.0 for x in P])
    psi = np.sqrt(Rs / r)
    # lapse e^nu matched to sqrt(1 - 2M/R) at the surface
    alpha = np.exp(Ys[:, 4] - Ys[-1, 4]) * math.sqrt(1.0 - 2.0 * M / Rsurf)
    return TOVSolution(K=K, Gamma=Gamma, rho_c=rho_c, M=M, Mb=Ys[-1, 3], R_areal=Rsurf, r_iso=rsurf,
                       r=r, rho=rho, P=P, psi=psi, alpha=alpha)


def cfl_for(rk):
    """The paper's c_CFL = 0.5 belongs to its RK4.  SSP-RK3 reaches only sqrt(3)
    on the imaginary axis against RK4's 2 sqrt(2), and the 1+log gauge modes
    (speed sqrt(2 alpha)) grow with it at 0.5; 0.3 = 0.5 sqrt(3) / (2 sqrt(2))
    keeps the same margin."""
    return 0.5 if rk == 0 else 0.3


def tov_config(name, rho_c=1.28e-3, n_levels=3, N=256, dx_fine=0.25, rk=1, solver=0, f_atm=1e-10,
               K=100.0, Gamma=2.0, Gamma_th=2.0, tov: TOVSolution | None = None, pwp=(),
               eos_adiabatic=0) -> tuple[RunConfig, TOVSolution]:
    if tov is None:
        tov = tov_solve(K, Gamma, rho_c, pwp=pwp)
    dx0 = dx_fine * (1 << (n_levels - 1))
    xmax = dx0 * N
    cfg = RunConfig(name=name, n_levels=n_levels, nx=N, nz=N, geometry=1, evolve_spacetime=1, solver=solver,
                    rk=rk, dx0=dx0, dz0=dx0, kappa=5e-3 / tov.M, eta_B=1.0 / tov.M, eps_ko=0.5, r_z4=xmax / 6.0,
                    K=K, Gamma=Gamma, Gamma_th=Gamma_th, rho_atm=f_atm * rho_c, cfl=cfl_for(rk), mass=tov.M,
                    pwp=tuple(pwp), eos_adiabatic=eos_adiabatic)
    return cfg, tov


def tov_level_data(cfg: RunConfig, tov: TOVSolution, level: int, p_deplete=1.0, equilibrium_lapse=False):
    """Kind-0 level data of a TOV star: W = psi^-2, alpha = psi^-2, h = At =
    Khat = Theta = Gt = beta = B = 0, fluid at rest; atmosphere outside.  A
    pressure depletion factor lowers P on the cold curve (rho scaled so that
    P = K rho^Gamma still holds)."""
    if cfg.pwp and p_deplete != 1.0:
        raise ValueError("pressure depletion is implemented for single-polytrope stars")
    X, Z = cell_centres(cfg, level)
    r = np.sqrt(X * X + Z * Z)
    inside = r < tov.r_iso
    rho = np.where(inside, np.interp(r, tov.r, tov.rho), 0.0)
    psi = np.where(inside, np.interp(r, tov.r, tov.psi), 1.0 + tov.M / (2.0 * np.maximum(r, 1e-300)))
    rho_atm = cfg.rho_atm
    if p_deplete != 1.0:
        rho = rho * p_deplete ** (1.0 / cfg.Gamma)
    rho = np.maximum(rho, rho_atm)
    if cfg.pwp:
        P = cold_P(cold_pieces(cfg.K, cfg.Gamma, cfg.pwp), rho)
    else:
        P = cfg.K * rho ** cfg.Gamma
    d = np.zeros((30, cfg.pz, cfg.px))
    d[0] = psi ** -2
    d[18] = psi ** -2
    if equilibrium_lapse:
        rr = np.maximum(r, 1e-300)
        d[18] = np.where(inside, np.interp(r, tov.r, tov.alpha),
                         (1.0 - tov.M / (2.0 * rr)) / (1.0 + tov.M / (2.0 * rr)))
    d[25] = rho
    d[29] = P
    return d


# ------------------------------------------------------------------ Bondi accretion onto a trumpet black hole

def trumpet_C(M=1.0):
    """C of the maximal trumpet slice of Schwarzschild: alpha^2 = 1 - 2M/R + C^2/R^4."""
    return 3.0 * math.sqrt(3.0) / 4.0 * M * M


def trumpet_r_of_R(R, M=1.0):
    """Coordinate radius r of the maximal trumpet slice at areal radius R >= 3M/2
    (closed form of the paper's Sec. III vacuum test; r = 0 at R = 3M/2)."""
    R = np.asarray(R, dtype=np.float64)
    a = (2.0 * R + M + np.sqrt(4.0 * R * R + 4.0 * M * R + 3.0 * M * M)) / 4.0
    b = (4.0 + 3.0 * math.sqrt(2.0)) * (2.0 * R - 3.0 * M) / (
        8.0 * R + 6.0 * M + 3.0 * np.sqrt(8.0 * R * R + 8.0 * M * R + 6.0 * M * M))
    return a * np.maximum(b, 0.0) ** (1.0 / math.sqrt(2.0))


def trumpet_R_of_r(r, M=1.0):
    """Areal radius R(r) by bisection of trumpet_r_of_R (monotone in R)."""
    r = np.asarray(r, dtype=np.float64)
    lo = np.full_like(r, 1.5 * M)
    hi = r + 3.0 * M
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        below = trumpet_r_of_R(mid, M) < r
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


@dataclasses.dataclass
class BondiSolution:
    M: float
    K: float
    Gamma: float
    R_c: float
    u_c: float          # |u^R| at the critical point
    rho_c: float
    Mdot: float         # accretion rate 4 pi R^2 rho |u^R|
    bern: float         # h^2 (1 - 2M/R + (u^R)^2), constant along the flow


def bondi_solve(M=1.0, K=1.0, Gamma=4.0 / 3.0, R_c=8.0):
    """Transonic (Michel) accretion of a polytrope P = K rho^Gamma onto a
    Schwarzschild black hole, fixed by its critical radius: (u^R)^2 = M / (2 R_c)
    and c_s^2 = u^2 / (1 - 3 u^2) there."""
    u2 = M / (2.0 * R_c)
    cs2 = u2 / (1.0 - 3.0 * u2)
    theta = cs2 / (Gamma * (1.0 - cs2 / (Gamma - 1.0)))       # P / rho with c_s^2 = Gamma P / (rho h)
    rho_c = (theta / K) ** (1.0 / (Gamma - 1.0))
    h_c = 1.0 + Gamma / (Gamma - 1.0) * theta
    u_c = math.sqrt(u2)
    return BondiSolution(M=M, K=K, Gamma=Gamma, R_c=R_c, u_c=u_c, rho_c=rho_c,
                         Mdot=4.0 * math.pi * R_c * R_c * rho_c * u_c,
                         bern=h_c * h_c * (1.0 - 2.0 * M / R_c + u2))


def bondi_rho(sol: BondiSolution, R):
    """Rest-mass density of the transonic solution at areal radius R: the root
    of h^2 (1 - 2M/R + u^2) = const, u = Mdot / (4 pi R^2 rho), on the
    subsonic side (larger rho) outside R_c and the supersonic side inside."""
    R = np.asarray(R, dtype=np.float64)
    g1 = sol.Gamma - 1.0

    def F(y):                      # y = ln rho
        rho = np.exp(y)
        h = 1.0 + sol.Gamma / g1 * sol.K * rho ** g1
        u = sol.Mdot / (4.0 * math.pi * R * R * rho)
        return h * h * (1.0 - 2.0 * sol.M / R + u * u) - sol.bern

    # minimum of F in ln rho (golden section), then bisection on the chosen side
    a = np.full_like(R, math.log(1e-14))
    b = np.full_like(R, math.log(10.0))
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    for _ in range(200):
        c = b - gr * (b - a)
        d = a + gr * (b - a)
        left = F(c) < F(d)
        b = np.where(left, d, b)
        a = np.where(left, a, c)
    ymin = 0.5 * (a + b)
    sub = R > sol.R_c
    lo = np.where(sub, ymin, math.log(1e-14))
    hi = np.where(sub, math.log(10.0), ymin)
    flo = F(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        fm = F(mid)
        same = np.sign(fm) == np.sign(flo)
        lo = np.where(same, mid, lo)
        flo = np.where(same, fm, flo)
        hi = np.where(same, hi, mid)
    return np.exp(0.5 * (lo + hi))


def bondi_trumpet_fields(sol: BondiSolution, x, z):
    """Metric (25 fields) and primitives (rho, u_x, u_y, u_z, P, eps) of the
    Bondi flow on the maximal trumpet slice at cartoon-plane points (x, z):
    W = r/R, alpha^2 = 1 - 2M/R + C^2/R^4, beta^i = C x^i / R^3,
    At_ij = (C / R^3)(delta_ij - 3 x^i x^j / r^2), h = Khat = Theta = Gt = B = 0.
    The fluid's covariant velocity follows from the Schwarzschild solution
    through ingoing Eddington-Finkelstein time v (regular at the horizon):
    the slice is t = v + H(R), H' = -R^2 / (alpha (C + R^2 alpha)), so
    u_R = 1/(s - u^R) + H' s with s = -u_v = sqrt((u^R)^2 + 1 - 2M/R), and
    u_r = u_R dR/dr = u_R R alpha / r."""
    M = sol.M
    C = trumpet_C(M)
    x = np.asarray(x, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    r = np.sqrt(x * x + z * z)
    R = trumpet_R_of_r(r, M)
    alpha = np.sqrt(1.0 - 2.0 * M / R + C * C / R ** 4)
    met = np.zeros((NMET,) + x.shape)
    met[0] = r / R
    met[18] = alpha
    cr3 = C / R ** 3
    met[19] = cr3 * x
    met[21] = cr3 * z
    met[7] = cr3 * (1.0 - 3.0 * x * x / (r * r))
    met[9] = cr3 * (-3.0 * x * z / (r * r))
    met[10] = cr3
    met[12] = cr3 * (1.0 - 3.0 * z * z / (r * r))
    rho = bondi_rho(sol, R)
    uR = -sol.Mdot / (4.0 * math.pi * R * R * rho)           # contravariant, inflow
    s = np.sqrt(uR * uR + 1.0 - 2.0 * M / R)
    Hp = -R * R / (alpha * (C + R * R * alpha))
    u_R = 1.0 / (s - uR) + Hp * s
    u_r = u_R * R * alpha / r
    P = sol.K * rho ** sol.Gamma
    prim = np.zeros((6,) + x.shape)
    prim[0] = rho
    prim[1] = u_r * x / r
    prim[3] = u_r * z / r
    prim[4] = P
    prim[5] = P / ((sol.Gamma - 1.0) * rho)
    return met, prim


def bondi_config(N=64, n_levels=1, solver=0, rk=0, xmax=16.0, r_hold=0.4, cfl=0.5, sol=None):
    """Bondi accretion in Cowling mode (metric frozen at the trumpet slice):
    an ideal gas P = (Gamma - 1) rho eps with Gamma = 4/3 (no cold part, so no
    cold-curve clamp), the flow on the adiabat K = 1 with critical radius 8M,
    box x_max = z_max = 16M over n_levels levels of N^2 (the finest box
    x_max / 2^(n_levels - 1)), hydro held inside r = 0.4M and at the outer
    boundary."""
    if sol is None:
        sol = bondi_solve()
    dx0 = xmax / N
    cfg = RunConfig(name="bondi_%dx%d" % (n_levels, N), n_levels=n_levels, nx=N, nz=N, geometry=1,
                    evolve_spacetime=0, solver=solver, rk=rk, dx0=dx0, dz0=dx0, K=0.0, Gamma=2.0,
                    Gamma_th=sol.Gamma, rho_atm=1e-12 * sol.rho_c, cfl=cfl, mass=sol.M, hydro_outer=1,
                    r_hold=r_hold)
    return cfg, sol


def bondi_level_data(cfg: RunConfig, sol: BondiSolution, level: int):
    """Kind-0 level data (25 metric fields, then rho, u_x, u_y, u_z, P) of the
    Bondi flow on the trumpet slice, ghosts included."""
    X, Z = cell_centres(cfg, level)
    met, prim = bondi_trumpet_fields(sol, X, Z)
    d = np.zeros((30, cfg.pz, cfg.px))
    d[:NMET] = met
    d[25:30] = prim[:5]
    return d


# ------------------------------------------------------------------ configurations

def config_shock_tube():
    """Special-relativistic shock tube, 400 x 4 cells, HLLC, CFL 0.4."""
    return shock_tube_config(400, 4, solver=0, rk=0, cfl=0.4)


def config_tov_stable():
    """Stable TOV star K=100, Gamma=2, rho_c=1.28e-3, 3 levels of 256^2, finest dx 0.25, SSP-RK3."""
    return tov_config("tov_stable_3x256", rho_c=1.28e-3, n_levels=3, N=256, dx_fine=0.25, rk=1)


def config_migration(N=512, n_levels=5, dx_fine=0.1):
    """Unstable TOV (rho_c = 7.993e-3) with a 1% pressure depletion, 5 levels of 512^2, finest dx 0.1, RK4."""
    return tov_config("migration_5x512", rho_c=7.993e-3, n_levels=n_levels, N=N, dx_fine=dx_fine, rk=0)


def config_batch_sweep(n_stars=64, seed=20250203, precision=7, rk=1, dx_fine=0.25,
                       sizes=(128, 256, 384, 512), levels=(2, 3, 4, 5), rho_c=(1e-3, 8e-3)):
    """Batched sweep of independent TOV / migration stars (K=100, Gamma=2):
    central densities uniform in rho_c, grids drawn from `sizes` with a level
    count drawn from `levels`, finest dx = dx_fine, all with one dt.  Returns
    [(RunConfig, TOVSolution)], seeded."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_stars):
        rc = float(rng.uniform(*rho_c))
        N = int(rng.choice(sizes))
        L = int(rng.choice(levels))
        cfg, tov = tov_config("sweep_%02d" % i, rho_c=rc, n_levels=L, N=N, dx_fine=dx_fine, rk=rk)
        cfg.precision = precision
        out.append((cfg, tov))
    return out


# ------------------------------------------------------------------ random inputs

def random_metric_perturbation(cfg: RunConfig, level: int, rng: np.random.Generator, amp=1e-2, nbump=3):
    """Smooth axisymmetric-consistent perturbation of every metric field: a sum
    of Gaussian bumps in (x, z), each field with the parity (odd/even in x and
    z) it has on the cartoon plane, so that ghost fills reproduce it."""
    X, Z = cell_centres(cfg, level)
    L = max(cfg.nx * cfg.dx(level), cfg.nz * cfg.dz(level))
    odd_x = {3, 5, 9, 11, 14, 15, 19, 20, 22, 23}   # hxz hyz Axz Ayz Gx Gy betax betay Bx By
    odd_z = {3, 5, 9, 11, 16, 21, 24}               # hxz hyz Axz Ayz Gz betaz Bz
    out = np.zeros((NMET, cfg.pz, cfg.px))
    for f in range(NMET):
        acc = np.zeros_like(X)
        for _ in range(nbump):
            x0, z0 = rng.uniform(0.1, 0.6, 2) * L
            s = rng.uniform(0.15, 0.3) * L
            a = rng.uniform(-1, 1)
            base = np.zeros_like(X)
            for sx in (1, -1):
                for sz in (1, -1):
                    px_ = sx if f in odd_x else 1
                    pz_ = sz if f in odd_z else 1
                    base += px_ * pz_ * np.exp(-((X - sx * x0) ** 2 + (Z - sz * z0) ** 2) / (s * s))
            acc += a * base
        out[f] = amp * acc
    return out


def random_prims(rng: np.random.Generator, n, w_max=50.0, log_rho=(-10.0, -2.0)):
    """n random primitive states (rho, u_x, u_y, u_z, P-factor) with Lorentz
    factors up to w_max and densities over the given decades."""
    rho = 10.0 ** rng.uniform(*log_rho, n)
    w = 1.0 + (w_max - 1.0) * rng.uniform(0, 1, n) ** 3
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    u = dirs * np.sqrt(w * w - 1.0)[:, None]
    pfac = 10.0 ** rng.uniform(-3, 1, n)
    return rho, u, pfac


def random_conformal_metric(rng: np.random.Generator, amp=0.1):
    """A random symmetric positive-definite gt_ij with det gt = 1 (the algebraic
    constraint the evolution keeps), returned as h_ij = gt_ij - delta_ij in the
    order (xx,xy,xz,yy,yz,zz), and a conformal factor W."""
    a = rng.uniform(-amp, amp, 6)
    a[0] = abs(a[0]); a[3] = abs(a[3]); a[5] = abs(a[5])
    g = np.array([[1 + a[0], a[1], a[2]], [a[1], 1 + a[3], a[4]], [a[2], a[4], 1 + a[5]]])
    g = g * np.linalg.det(g) ** (-1.0 / 3.0)
    h = np.array([g[0, 0] - 1, g[0, 1], g[0, 2], g[1, 1] - 1, g[1, 2], g[2, 2] - 1])
    W = rng.uniform(0.6, 1.0)
    return W, h
