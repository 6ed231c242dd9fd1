"""The learned seed of the primitive recovery: the GPU training kernels'
gradient against the FP64 oracle (oracle/mlp.py), training on tuples the
solver generates, the seeded recovery against the plain one (the Illinois
iteration as judge: same primitives to its tolerance), and what the seed
gains (Illinois function evaluations per recovery)."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2502_03223_gb300 import sacra2d as S
from paper_2502_03223_gb300 import workloads as W

from gpu_common import G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_03223_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()


def _oracle_inputs(tuples, p):
    xh = (tuples[:, :9].astype(np.float64) - p["in_mu"]) / p["in_sd"]
    th = (tuples[:, 9].astype(np.float64) - p["out_mu"]) / p["out_sd"]
    return xh, th


def test_network_size():
    assert S.load().sacra_mlp_bytes() == 10096        # 16-byte aligned
    assert M.n_params() == S.MLP_NPARAM


def test_gpu_gradient_matches_oracle():
    import torch
    rng = np.random.default_rng(7)
    n = 3000
    x = rng.normal(size=(n, 9)) * rng.uniform(0.5, 3.0, 9) + rng.uniform(-2, 2, 9)
    y = np.tanh(x[:, :3].sum(axis=1)) + 0.1 * x[:, 3] - 0.05 * x[:, 4] ** 2
    tuples = torch.tensor(np.column_stack([x, y]), dtype=torch.float32, device="cuda")
    for steps in (0, 50):                      # the initial network and a partly trained one
        net, _, _ = S.mlp_train(tuples, steps=steps, batch_blocks=8, lr=3e-3, seed=11)
        g, loss = S.mlp_grad(tuples, net)
        p = S.mlp_unpack(net.cpu().numpy())
        xh, th = _oracle_inputs(tuples.cpu().numpy(), p)
        theta = M.flatten(p)
        g64 = M.grad(theta, xh, th)
        assert abs(loss - M.loss(theta, xh, th)) <= 1e-5 * M.loss(theta, xh, th)
        scale = np.max(np.abs(g64))
        err = np.abs(g.astype(np.float64) - g64)
        assert np.max(err) <= 2e-5 * scale, (steps, np.max(err) / scale)
        big = np.abs(g64) > 1e-2 * scale
        assert np.max(err[big] / np.abs(g64[big])) < 1e-3


def _moving_star(N=64, L=2, seed=3):
    cfg, tov = W.tov_config("mlp", rho_c=2.0e-3, n_levels=L, N=N, dx_fine=0.4, rk=1)
    datas = []
    rng = np.random.default_rng(seed)
    for l in range(L):
        d = W.tov_level_data(cfg, tov, l)
        X, Z = W.cell_centres(cfg, l)
        amp = rng.uniform(0.05, 0.15, 3)
        bump = np.exp(-(X ** 2 + Z ** 2) / (0.6 * tov.r_iso) ** 2)
        d[26] = amp[0] * bump * np.tanh(X)                 # u_x, odd in x
        d[27] = amp[1] * bump * np.tanh(X)                 # u_y (rotation)
        d[28] = amp[2] * bump * np.tanh(Z)                 # u_z, odd in z
        d[29] *= 1.0 + 0.02 * bump                         # a little heat
        datas.append(d)
    return cfg, datas


def _sim(cfg, datas):
    s = S.Sacra(cfg)
    for l, d in enumerate(datas):
        s.set_initial_data(l, S.PRIM_METRIC, d)
    return s


@pytest.fixture(scope="module")
def trained():
    import torch
    cfg, datas = _moving_star()
    sim = _sim(cfg, datas)
    buf = torch.zeros((200000, 10), dtype=torch.float32, device="cuda")
    parts = []
    for _ in range(12):                         # tuples from several moments of the evolution
        sim.step(cfg.dt, 2)
        n = sim.mlp_collect(buf)
        parts.append(buf[:n].clone())
    tuples = torch.cat(parts)
    net, rep, hist = S.mlp_train(tuples, steps=6000, batch_blocks=16, lr=1e-2, seed=5, record_loss=True)
    return cfg, datas, tuples, net, rep, hist


def test_training_on_solver_tuples(trained):
    cfg, datas, tuples, net, rep, hist = trained
    assert tuples.shape[0] > 2000
    assert np.mean(hist[-100:]) < 0.05 * np.mean(hist[:10])      # the loss falls by > 20x
    assert rep["val_rms_log10"] < 0.05                             # held out: P/D within ~12 %
    assert 1e-5 <= rep["delta"] <= 0.05 + 1e-6


def test_seeded_recovery_equals_plain_and_gains(trained):
    cfg, datas, tuples, net, rep, hist = trained
    plain, seeded = _sim(cfg, datas), _sim(cfg, datas)
    seeded.set_mlp(net)
    for s in (plain, seeded):
        s.c2p_counting(True)
    plain.step(cfg.dt, 1)
    seeded.step(cfg.dt, 1)
    for l in range(cfg.n_levels):
        for f in range(6):
            a, b = seeded.read(l, S.PRIMS, f), plain.read(l, S.PRIMS, f)
            scale = max(np.max(np.abs(b)), 1e-300) if f in (1, 2, 3) else np.abs(b)
            assert np.all(np.abs(a - b) <= 1e-11 * np.maximum(scale, 1e-300) + 1e-300), (l, f)
        assert np.array_equal(seeded.read(l, S.STATUS, 0), plain.read(l, S.STATUS, 0))
    ev_p, _, _, n_p = plain.c2p_counts()
    ev_s, tried, held, n_s = seeded.c2p_counts()
    assert n_p == n_s and tried > 0
    assert held >= 0.95 * tried
    print("Illinois evaluations per recovery: plain %.3f, seeded %.3f (seed held in %.1f%% of %d tries)"
          % (ev_p / n_p, ev_s / n_s, 100.0 * held / tried, tried))
    assert ev_s < ev_p


def test_seed_gain_in_a_relativistic_flow():
    """A relativistic shock tube (left state v = 0.9, w = 2.3, hitting a dense
    counter-flow): the plain bracket needs ~9 master-function evaluations per
    recovery; the trained seed cuts that by more than 20 % (measured 33 %;
    tuples, split and training are deterministic) with the same primitives
    (the Illinois iteration judges every seeded solve)."""
    import torch
    cfg = W.shock_tube_config(400, 4, solver=0, rk=0, cfl=0.4)
    d = W.shock_tube_data(cfg, left=(1.0, 1.0, 0.9), right=(10.0, 0.01, -0.5))

    def mk():
        s = S.Sacra(cfg)
        s.set_initial_data(0, S.PRIM_METRIC, d)
        return s
    sim = mk()
    buf = torch.zeros((50000, 10), dtype=torch.float32, device="cuda")
    parts = []
    for _ in range(20):
        sim.step(cfg.dt, 5)
        n = sim.mlp_collect(buf)
        parts.append(buf[:n].clone())
    net, rep, _ = S.mlp_train(torch.cat(parts), steps=6000, batch_blocks=16, lr=1e-2, seed=5)
    plain, seeded = mk(), mk()
    plain.step(cfg.dt, 50)
    seeded.step(cfg.dt, 50)
    seeded.set_mlp(net)
    for s in (plain, seeded):
        s.c2p_counting(True)
    plain.step(cfg.dt, 1)
    seeded.step(cfg.dt, 1)
    for f in range(6):
        a, b = seeded.read(0, S.PRIMS, f), plain.read(0, S.PRIMS, f)
        assert np.all(np.abs(a - b) <= 1e-11 * np.maximum(np.abs(b), 1.0 if f in (1, 2, 3) else 0.0) + 1e-300), f
    ep, es = plain.c2p_counts(), seeded.c2p_counts()
    print("relativistic tube: Illinois evaluations per recovery plain %.3f, seeded %.3f; held-out RMS of "
          "log10(P/D) %.4f, delta %.3g" % (ep[0] / ep[3], es[0] / es[3], rep["val_rms_log10"], rep["delta"]))
    assert es[2] >= 0.99 * es[1]
    assert es[0] / es[3] < 0.8 * ep[0] / ep[3]
