"""Pins of the oracle's network gradient (oracle/mlp.py): backpropagation
against central finite differences of the loss, a closed form in the
linear regime, and the BF16 rounding against exactly representable cases."""
import numpy as np

from oracle import mlp as M


def _problem(seed=0, n=40, scale=0.3):
    rng = np.random.default_rng(seed)
    theta = rng.normal(scale=scale, size=M.n_params())
    xh = rng.normal(size=(n, M.N_IN))
    th = rng.normal(size=n)
    return theta, xh, th


def test_backprop_matches_central_differences():
    theta, xh, th = _problem()
    g = M.grad(theta, xh, th)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(M.n_params(), 60, replace=False), [M.n_params() - 1]])   # incl. b3
    fd = M.fd_grad(theta, xh, th, idx, h=1e-5)
    rel = np.abs(fd - g[idx]) / np.maximum(np.abs(g[idx]), 1e-3 * np.max(np.abs(g)))
    assert np.max(rel) < 1e-6, np.max(rel)


def test_gradient_in_the_linear_output_layer_is_least_squares():
    # only w3, b3 enter linearly: dL/dw3 = (2/n) H2^T (yh - t), dL/db3 = (2/n) sum (yh - t)
    theta, xh, th = _problem(2)
    p = M.unflatten(theta)
    h2 = np.tanh(np.tanh(xh @ p["w1"].T + p["b1"]) @ p["w2"].T + p["b2"])
    res = h2 @ p["w3"] + p["b3"] - th
    g = M.unflatten(M.grad(theta, xh, th))
    assert np.allclose(g["w3"], 2.0 / len(th) * h2.T @ res, rtol=1e-13, atol=1e-15)
    assert abs(g["b3"] - 2.0 / len(th) * res.sum()) < 1e-13


def test_zero_hidden_weights_decouple_the_input_layer():
    # with w2 = 0 the output does not depend on the first layer: its gradient vanishes
    theta, xh, th = _problem(3)
    p = M.unflatten(theta)
    p["w2"][:] = 0.0
    g = M.unflatten(M.grad(M.flatten(p), xh, th))
    assert np.all(g["w1"] == 0.0) and np.all(g["b1"] == 0.0)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 0.0, 3.0 * 2.0 ** -20])
    want = np.array([1.0, 1.0 + 2.0 ** -7, 1.0, 1.0 + 2.0 ** -7, -2.5, 0.0, 3.0 * 2.0 ** -20])
    assert np.array_equal(M.bf16_round(vals), want)
    # 1 + 3 * 2^-8 is a tie between 1 + 2^-7 and 1 + 2^-6: even mantissa wins
    assert M.bf16_round([1.0 + 3 * 2.0 ** -8])[0] == 1.0 + 2.0 ** -6
