"""Helpers shared by the GPU parity tests: run the CUDA library and the CPU
oracle on the same seeded inputs and compare them cell by cell."""
import numpy as np

import oracle as O
from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

G = 8
ST_COLD, ST_ATM = 2, 4


def both(cfg, datas):
    gpu = S.Sacra(cfg)
    orc = O.Oracle(cfg)
    for l, d in enumerate(datas):
        gpu.set_initial_data(l, S.PRIM_METRIC, d)
        orc.set_level(l, 0, d)
    return gpu, orc


# Physical groups of fields sharing one scale.  A value formed by cancelling
# terms of magnitude T carries a rounding error ~1e-16 T whatever its own size
# (finite differences of smooth data, Theta ~ alpha H / 2 with H ~ 0, the
# momentum increment of a nearly uniform state), so the per-cell relative
# criterion uses max(|b|, S_group) with S_group the largest magnitude of the
# group on the level.
STATE_GROUPS = [[0, 1, 2, 3, 4, 5, 6, 18],            # W, h_ij, alpha (dimensionless metric)
                [7, 8, 9, 10, 11, 12, 13, 17],        # At_ij, Khat, Theta (curvature)
                [14, 15, 16],                         # Gt^i
                [19, 20, 21, 22, 23, 24],             # beta^i, B^i
                [25, 26, 28, 29],                     # q_D, q_Sx, q_Sz, q_E
                [27]]                                 # q_Sy (x q_Sy in cylindrical geometry: x * group 5)
PRIM_GROUPS = [[0], [1, 2, 3], [4], [5]]              # rho, u_i, P, eps

# Gt^i, beta^i and B^i are zero in conformally flat initial data: after one
# step they are dt times right-hand sides of cancelling O(1) terms, rounded at
# ~1e-16 x dt x O(1) x (number of terms) ~ 1e-15 absolute (measured up to
# 1.5e-15), while their own maximum is ~3e-5: the floor 1e-3 allows 1e-14.
ZERO_BORN = {f: 1e-3 for f in (14, 15, 16, 19, 20, 21, 22, 23, 24)}
# Velocities are derived, u_i = S_i / (rho h w): a momentum that agrees to the
# round-off of its group scale (~1e-16 rho_max, compared in the state planes)
# gives a velocity difference ~1e-16 rho_max / rho, so in low-density cells
# the velocity bound carries the factor max(1, VEL_COND rho_max / rho).
VEL_COND = 1e-4


def group_scale(planes, groups, f, xmax=1.0):
    if groups is STATE_GROUPS and f == 27:
        # q_Sphi = x q_Sy: x times the momentum / energy scale
        return max(float(np.max(np.abs(planes[27]))),
                   xmax * max(float(np.max(np.abs(planes[i]))) for i in (25, 26, 28, 29)))
    for g in groups:
        if f in g:
            return max(float(np.max(np.abs(planes[i]))) for i in g)
    raise KeyError(f)


def atmosphere_threshold_cells(gpu, orc, level, rho_atm, rel=1e-9):
    """Cells where one side reset to the atmosphere and the other did not,
    with the density at the threshold on both sides (|rho / rho_atm - 1| <=
    rel): the decision rho < rho_atm taken on values that differ by rounding.
    Both outcomes are valid; the velocities of such a cell (S / (D h) with S
    at round-off, against 0) are not comparable."""
    sa = gpu.read(level, S.STATUS, 0).astype(np.int64)
    sb = orc.read(level, 4, 0).astype(np.int64)
    ra = gpu.read(level, S.PRIMS, 0)
    rb = orc.read(level, 2, 0)
    flip = (sa & ST_ATM) != (sb & ST_ATM)
    at = (np.abs(ra / rho_atm - 1.0) <= rel) & (np.abs(rb / rho_atm - 1.0) <= rel)
    return flip & at


# Cells beyond the per-cell bound (at most max_frac of a field's cells) are
# excused only as branch decisions taken on values that differ by rounding:
# within STATUS_REACH cells of a cell whose recovery status differs between
# the two sides (a discontinuous branch: atmosphere, cold clamp, iteration
# count, whose effect spreads through the stencils) the error may reach
# EXCUSE_NEAR_FLIP of the group scale; anywhere else (a PPM or minmod limiter
# switching at a point where its branches meet) only EXCUSE_ELSEWHERE.
STATUS_REACH = 4
EXCUSE_NEAR_FLIP = 1e-6
EXCUSE_ELSEWHERE = 1e-9
# worst ratio and excused cells seen by compare_level since the last reset
STATS = {"worst": 0.0, "excused": 0, "excused_worst": 0.0, "cells": 0, "masked": 0}


def reset_stats():
    STATS.update(worst=0.0, excused=0, excused_worst=0.0, cells=0, masked=0)


def stats_line():
    return ("worst ratio %.2e of the group scale within the bound; %d of %d compared values excused "
            "(worst %.2e); %d in the caller's mask of checked flips"
            % (STATS["worst"], STATS["excused"], STATS["cells"], STATS["excused_worst"], STATS["masked"]))


def status_flip_zone(gpu, orc, level, reach=STATUS_REACH):
    """Cells within `reach` (Chebyshev distance) of a cell whose observable
    recovery status differs between the two sides."""
    a = _observable_status(gpu.read(level, S.STATUS, 0))
    b = _observable_status(orc.read(level, 4, 0))
    flip = a != b
    if not flip.any():
        return flip
    z = flip.copy()
    for dk in range(-reach, reach + 1):
        for dj in range(-reach, reach + 1):
            z |= np.roll(np.roll(flip, dk, axis=0), dj, axis=1)
    return z


def compare_level(gpu, orc, level, tol=1e-11, which=(0, 1, 2), max_frac=1e-3, report=None, excuse=None,
                  floors=None):
    """Compare the state / primitive / rhs planes of a level cell by cell:
    |a - b| <= tol * max(|b|, S_group).  At most max_frac of the cells may
    exceed tol, each as a branch decision taken on values that differ by
    rounding (see EXCUSE_NEAR_FLIP / EXCUSE_ELSEWHERE); cells in the boolean
    mask `excuse` (a flip checked separately to be valid on both sides) are
    left out.  floors = {state field: S}: a lower bound on S_group for fields
    whose own maximum understates the size of the terms they are computed
    from (see the caller).  Returns the worst ratio of the cells within tol."""
    worst = 0.0
    zone = status_flip_zone(gpu, orc, level)
    for w in which:
        prim = w == S.PRIMS
        nf = 6 if prim else 30
        A = [gpu.read(level, w, f) for f in range(nf)]
        B = [orc.read(level, w, f) for f in range(nf)]
        groups = PRIM_GROUPS if prim else STATE_GROUPS
        cfg = gpu.cfg
        xmax = max(1.0, (cfg.nx + 8) * cfg.dx(level)) if cfg.geometry == 1 else 1.0
        for f in range(nf):
            a, b = A[f], B[f]
            sg = group_scale(B, groups, f, xmax)
            if floors and not prim and f in floors:
                sg = max(sg, floors[f])
            scale = None
            if prim and f in (1, 2, 3):
                sg = max(sg, 1.0)          # velocities: units of c
                rho = B[0]
                cond = np.maximum(1.0, VEL_COND * float(np.max(rho)) / np.maximum(rho, 1e-300))
                scale = np.maximum(np.abs(b), sg) * cond
            if scale is None:
                scale = np.maximum(np.abs(b), sg)
            with np.errstate(divide="ignore", invalid="ignore"):
                r = np.where(scale > 0, np.abs(a - b) / scale, np.where(a == b, 0.0, np.inf))
            bad = ~(r <= tol)
            if excuse is not None:
                bad &= ~excuse
            frac = float(bad.mean())
            within = r <= tol
            worst = max(worst, float(np.max(r[within])) if np.any(within) else 0.0)
            if excuse is not None:
                STATS["masked"] += int((excuse & ~within).sum())
            STATS["cells"] += r.size
            if np.any(bad):
                STATS["excused"] += int(bad.sum())
                STATS["excused_worst"] = max(STATS["excused_worst"], float(np.max(r[bad])))
                near = bad & zone
                far = bad & ~zone
                assert not np.any(r[near] > EXCUSE_NEAR_FLIP), (level, w, f, float(np.max(r[near])))
                assert not np.any(r[far] > EXCUSE_ELSEWHERE), (level, w, f, float(np.max(r[far])))
            if report is not None and frac > 0:
                report.append((level, w, f, frac, float(np.max(r))))
            assert frac <= max_frac, (level, w, f, frac, float(np.nanmax(r)))
    STATS["worst"] = max(STATS["worst"], worst)
    return worst


def _observable_status(st):
    """A cell reset to the atmosphere takes the atmosphere's primitives
    whether or not its solve hit the cold-curve clamp first, so the clamp
    bit is dropped where the atmosphere bit is set."""
    st = np.asarray(st).astype(np.int64)
    return np.where(st & ST_ATM, st & ~ST_COLD, st)


def compare_status(gpu, orc, level, max_frac=1e-3):
    a = _observable_status(gpu.read(level, S.STATUS, 0))
    b = _observable_status(orc.read(level, 4, 0))
    frac = float(np.mean(a != b))
    assert frac <= max_frac, frac
    return frac
