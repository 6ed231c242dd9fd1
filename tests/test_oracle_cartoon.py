"""Pin of the oracle's cartoon y-derivatives (Sec. II.B.2): for an exactly
axisymmetric, regular 3D field (scalars s(varpi^2, z), vectors
a rho + b phi + c z_hat, tensors built from delta, rho, phi, z_hat), the
derivatives d_y, d_yy, d_xy, d_yz obtained from the interpolated-and-rotated
planes must converge at 6th order to the exact 3D derivatives at y = 0."""
import numpy as np
import pytest

import oracle as O
from paper_2502_03223_gb300 import workloads as W

G = 8
PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def _profiles(x, y, z):
    """Cartesian 3D values of all 25 fields (scalars, vectors, tensors)."""
    x, y, z = np.broadcast_arrays(np.asarray(x, dtype=float), np.asarray(y, dtype=float),
                                  np.asarray(z, dtype=float))
    r2 = x * x + y * y
    g1 = np.exp(-(r2 + z * z) / 2.0)
    g2 = np.exp(-((r2 - 0.5) ** 2 + z * z) / 1.5)
    zero, one = np.zeros_like(x), np.ones_like(x)
    rho = np.array([x, y, zero])
    phi = np.array([-y, x, zero])
    zh = np.array([zero, zero, one])

    def vec(a, b, c):
        return a * rho + b * phi + c * zh

    def ten(f1, f2, f3, f4, f5):
        T = np.zeros((3, 3) + np.shape(x))
        for i in range(3):
            for j in range(3):
                T[i, j] = f1 * (i == j) + f2 * rho[i] * rho[j] + f3 * (rho[i] * zh[j] + zh[i] * rho[j]) \
                    + f4 * (phi[i] * rho[j] + rho[i] * phi[j]) + f5 * (phi[i] * zh[j] + zh[i] * phi[j])
        return T

    out = np.zeros((25,) + np.shape(x))
    out[0] = 0.8 + 0.1 * g1
    T1 = ten(0.05 * g1, 0.02 * g2, 0.03 * z * g1, 0.01 * g1, 0.02 * z * g2)
    T2 = ten(0.03 * g2, 0.01 * g1, 0.02 * z * g2, 0.02 * g2, 0.01 * z * g1)
    for a, (i, j) in enumerate(PAIRS):
        out[1 + a] = T1[i, j]
        out[7 + a] = T2[i, j]
    out[13] = 0.1 * g2
    out[14:17] = vec(0.05 * g1, 0.03 * g2, 0.04 * z * g1)
    out[17] = 0.02 * g1
    out[18] = 0.9 - 0.1 * g2
    out[19:22] = vec(0.02 * g2, 0.05 * g1, 0.03 * z * g2)
    out[22:25] = vec(0.01 * g1, 0.02 * g2, 0.05 * z * g1)
    return out


def _exact(x, z, h=1e-4):
    """d_y, d_yy, d_xy, d_yz at y = 0 by 6th-order differences of the 3D field with a tiny step."""
    c1 = np.array([-1, 9, -45, 0, 45, -9, 1]) / 60.0
    c2 = np.array([2, -27, 270, -490, 270, -27, 2]) / 180.0
    offs = np.arange(-3, 4)
    fy = [_profiles(x, o * h, z) for o in offs]
    dy = sum(c * f for c, f in zip(c1, fy)) / h
    dyy = sum(c * f for c, f in zip(c2, fy)) / (h * h)
    dxy = sum(ci * cj * _profiles(x + oi * h, oj * h, z) for ci, oi in zip(c1, offs) for cj, oj in zip(c1, offs)) / (h * h)
    dyz = sum(ci * cj * _profiles(x, oi * h, z + oj * h) for ci, oi in zip(c1, offs) for cj, oj in zip(c1, offs)) / (h * h)
    return dy, dyy, dxy, dyz


def _errors(N, L):
    cfg = W.RunConfig(n_levels=1, nx=N, nz=N, geometry=1, evolve_spacetime=1, dx0=L / N, dz0=L / N, K=100.0)
    X, Z = W.cell_centres(cfg, 0)
    d = np.zeros((30, cfg.pz, cfg.px))
    d[:25] = _profiles(X, 0.0 * X, Z)
    d[25] = 1e-3
    d[29] = 1e-4
    o = O.Oracle(cfg)
    o.set_level(0, 0, d)
    o.fill(0, 0.0)
    # sample cells in the inner part of the level, including the axis region
    js = np.array([1, 2, 3, N // 4, N // 2, N // 2 + 1, 3 * N // 4] * 3)
    ks = np.repeat([1, N // 3, N // 2], 7)
    dQ, ddQ, _ = o.derivs(0, js, ks)
    x = (js - 0.5) * cfg.dx0
    z = (ks - 0.5) * cfg.dz0
    ey, eyy, exy, eyz = _exact(x, z)
    err = 0.0
    for f in range(25):
        err = max(err, np.max(np.abs(dQ[:, f, 1] - ey[f])), np.max(np.abs(ddQ[:, f, 3] - eyy[f])),
                  np.max(np.abs(ddQ[:, f, 1] - exy[f])), np.max(np.abs(ddQ[:, f, 4] - eyz[f])))
    return err


def test_cartoon_derivatives_sixth_order():
    e1 = _errors(32, 4.0)
    e2 = _errors(64, 4.0)
    assert e2 < 1e-5
    assert e1 / e2 > 40.0, (e1, e2)       # 2^6 = 64 for 6th order


def test_cartoon_edge_formula_matches_planes():
    """Eq. cartoon_bnd (used beyond the level edge) agrees with the plane
    construction where both exist (the analytic d_xy of an axisymmetric field)."""
    N, L = 64, 4.0
    cfg = W.RunConfig(n_levels=1, nx=N, nz=N, geometry=1, evolve_spacetime=1, dx0=L / N, dz0=L / N, K=100.0)
    X, Z = W.cell_centres(cfg, 0)
    d = np.zeros((30, cfg.pz, cfg.px))
    d[:25] = _profiles(X, 0.0 * X, Z)
    d[25] = 1e-3
    d[29] = 1e-4
    o = O.Oracle(cfg)
    o.set_level(0, 0, d)
    o.fill(0, 0.0)
    js = np.array([N + 1, N + 2, N + 3, N + 4])
    ks = np.array([N // 2] * 4)
    dQ, ddQ, _ = o.derivs(0, js, ks)
    x = (js - 0.5) * cfg.dx0
    z = (ks - 0.5) * cfg.dz0
    _, _, exy, _ = _exact(x, z)
    for f in (1, 2, 3, 4, 5, 7, 8, 9, 10, 11, 14, 15, 19, 20, 22, 23):
        assert np.max(np.abs(ddQ[:, f, 1] - exy[f])) < 1e-6, f
