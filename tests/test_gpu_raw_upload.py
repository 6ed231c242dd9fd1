"""Saving and restoring a level's state (sacra_read_level, then
sacra_set_initial_data with SACRA_RAW, whose copy arrives in row chunks while
the primitives of the chunks already there are recovered): every row of the
restored context holds the state and primitives of the running one, from
pageable and from pinned host buffers, and it evolves as the original does.
The upload recovers the primitives of every cell again, which can rewrite the
conserved variables of a cell at the level of rounding (a state reset to the
atmosphere or clamped to the cold curve, recovered once more, may take the
other branch), so the comparison is against each field's group scale.  A row
left out by the chunking would leave its primitives at zero."""
import numpy as np
import pytest

from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import STATE_GROUPS, group_scale

pytestmark = pytest.mark.gpu
G = 8


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


@pytest.mark.parametrize("pinned", [False, True])
def test_restored_state_evolves_like_the_original(pinned):
    import torch
    cfg, tov = W.tov_config("raw", rho_c=1.28e-3, n_levels=3, N=56, dx_fine=0.5, rk=0)
    datas = []
    for l in range(cfg.n_levels):
        d = W.tov_level_data(cfg, tov, l)
        X, Z = W.cell_centres(cfg, l)
        bump = np.exp(-((X - 3.0) ** 2 + (Z - 2.0) ** 2) / 4.0)
        d[26] = 0.05 * bump * X / (np.abs(X) + 1.0)
        datas.append(d)
    a = S.Sacra(cfg)
    for l, d in enumerate(datas):
        a.set_initial_data(l, S.PRIM_METRIC, d)
    a.step(cfg.dt, 3, use_graph=True)
    n = 30 * a.px * a.pz
    saved = []
    for l in range(cfg.n_levels):
        h = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy() if pinned else np.empty(n)
        a.read_level(l, h)
        saved.append(h)
    b = S.Sacra(cfg)
    for l in range(cfg.n_levels):
        b.set_initial_data(l, S.RAW, saved[l])
    inner = (slice(G, G + cfg.nz), slice(G, G + cfg.nx))

    def close(tol):
        for l in range(cfg.n_levels):
            A = [a.read(l, S.STATE_STEP, f)[inner] for f in range(30)]
            B = [b.read(l, S.STATE_STEP, f)[inner] for f in range(30)]
            for f in range(30):
                s = group_scale(A, STATE_GROUPS, f, xmax=(cfg.nx + 8) * cfg.dx(l))
                assert float(np.max(np.abs(B[f] - A[f]))) <= tol * s, (l, f)
            for f in range(6):
                pa, pb = a.read(l, S.PRIMS, f)[inner], b.read(l, S.PRIMS, f)[inner]
                s = max(float(np.max(np.abs(pa))), 1.0 if f in (1, 2, 3) else 0.0)
                assert float(np.max(np.abs(pb - pa))) <= tol * s, (l, f)

    close(1e-12)
    a.step(cfg.dt, 2, use_graph=True)
    b.step(cfg.dt, 2, use_graph=True)
    close(1e-11)
    a.close()
    b.close()
