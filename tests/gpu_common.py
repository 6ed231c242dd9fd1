"""Helpers shared by the GPU parity tests: run the CUDA library and the CPU
oracle on the same seeded inputs and compare them cell by cell."""
import numpy as np

import oracle as O
from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

G = 8


def both(cfg, datas):
    gpu = S.Sacra(cfg)
    orc = O.Oracle(cfg)
    for l, d in enumerate(datas):
        gpu.set_initial_data(l, S.PRIM_METRIC, d)
        orc.set_level(l, 0, d)
    return gpu, orc


def rel_mismatch(a, b, tol, floor_frac=1e-6):
    """Cells where |a - b| > tol * max(|b|, floor_frac * max|b|) (the
    per-cell relative criterion with a field-scaled floor near zero)."""
    scale = np.maximum(np.abs(b), floor_frac * np.max(np.abs(b)))
    bad = np.abs(a - b) > tol * scale
    bad &= ~((scale == 0) & (a == b))
    return bad


def compare_level(gpu, orc, level, tol=1e-11, which=(0, 1, 2), fields=None, max_frac=1e-3, report=None):
    """Compare the stage/step state, primitives and rhs planes of a level.
    Returns the worst relative error; asserts that the fraction of cells
    beyond tol stays below max_frac (cells where a discrete branch flipped)."""
    worst = 0.0
    for w in which:
        nf = 6 if w == S.PRIMS else 30
        for f in (fields if fields is not None and w != S.PRIMS else range(nf)):
            a = gpu.read(level, w, f)
            b = orc.read(level, w, f)
            bad = rel_mismatch(a, b, tol)
            scale = np.maximum(np.abs(b), 1e-6 * np.max(np.abs(b)))
            with np.errstate(divide="ignore", invalid="ignore"):
                r = np.where(scale > 0, np.abs(a - b) / scale, np.where(a == b, 0.0, np.inf))
            worst = max(worst, float(np.max(r[~bad])) if np.any(~bad) else 0.0)
            frac = bad.mean()
            if report is not None and frac > 0:
                report.append((level, w, f, frac, float(np.max(r))))
            assert frac <= max_frac, (level, w, f, frac, float(np.nanmax(r)))
    return worst
