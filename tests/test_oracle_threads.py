"""The oracle's parallel loops change no result: one RK step of a two-level
TOV hierarchy with velocity perturbations is bit for bit the same with one
worker thread and with several."""
import numpy as np

import oracle as O
from paper_2502_03223_gb300 import workloads as W


def _run(threads):
    O.set_threads(threads)
    cfg, tov = W.tov_config("thr", rho_c=1.28e-3, n_levels=2, N=24, dx_fine=0.5, rk=0)
    o = O.Oracle(cfg)
    for l in range(2):
        d = W.tov_level_data(cfg, tov, l)
        d[:25] += W.random_metric_perturbation(cfg, l, np.random.default_rng(5), amp=1e-4)
        X, Z = W.cell_centres(cfg, l)
        d[26] = 0.05 * np.exp(-((X - 3) ** 2 + (Z - 2) ** 2) / 4.0) * X / (np.abs(X) + 1.0)
        o.set_level(l, 0, d)
    o.step(cfg.dt, 2)
    out = [o.read(l, w, f) for l in range(2) for w, nf in ((0, 30), (2, 6)) for f in range(nf)]
    fb = o.fallbacks()
    o.close()
    return out, fb


def test_thread_count_does_not_change_results():
    a, fa = _run(1)
    b, fb = _run(4)
    O.set_threads(0)
    assert fa == fb
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
