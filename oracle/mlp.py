"""Oracle of the learned primitive-recovery seed: a 9 -> 64 -> 64 -> 1 tanh
network (plain numpy, FP64), its mean-squared loss and the gradient of that
loss by backpropagation, written from the definitions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the tests check the GPU
training kernels' gradients against this one, and pin this one against
central finite differences.

Network (weights as the GPU stores them, row-major):
    xh = (x - in_mu) / in_sd                      x: 9 features
    a1 = W1 xh + b1,  h1 = tanh(a1)               W1: 64 x 9
    a2 = W2 h1 + b2,  h2 = tanh(a2)               W2: 64 x 64
    yh = w3 . h2 + b3                              w3: 64
    y  = out_mu + out_sd * yh
Loss over n samples with normalised targets th = (t - out_mu) / out_sd:
    L = (1 / n) sum (yh - th)^2
"""
import numpy as np

N_IN, N_H = 9, 64
# parameter blocks in the GPU's flat order
SHAPES = [("w1", (N_H, N_IN)), ("b1", (N_H,)), ("w2", (N_H, N_H)), ("b2", (N_H,)), ("w3", (N_H,)), ("b3", ())]


def n_params():
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(p, xh):
    """xh: (n, 9) normalised inputs.  Returns yh (n,) and the activations."""
    a1 = xh @ p["w1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["w2"].T + p["b2"]
    h2 = np.tanh(a2)
    yh = h2 @ p["w3"] + p["b3"]
    return yh, (h1, h2)


def loss(theta, xh, th):
    p = unflatten(theta)
    yh, _ = forward(p, xh)
    return float(np.mean((yh - th) ** 2))


def grad(theta, xh, th):
    """dL/dtheta by backpropagation (chain rule through the three layers)."""
    p = unflatten(theta)
    n = xh.shape[0]
    yh, (h1, h2) = forward(p, xh)
    e = 2.0 * (yh - th) / n                       # dL/dyh
    g = {"w3": h2.T @ e, "b3": np.sum(e)}
    d2 = np.outer(e, p["w3"]) * (1.0 - h2 * h2)   # dL/da2
    g["w2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["w2"]) * (1.0 - h1 * h1)         # dL/da1
    g["w1"] = d1.T @ xh
    g["b1"] = d1.sum(axis=0)
    return flatten(g)


def fd_grad(theta, xh, th, idx, h=1e-6):
    """Central finite difference of the loss along the listed parameters."""
    out = []
    for i in idx:
        tp = np.array(theta, dtype=np.float64)
        tm = tp.copy()
        tp[i] += h
        tm[i] -= h
        out.append((loss(tp, xh, th) - loss(tm, xh, th)) / (2.0 * h))
    return np.array(out)


def bf16_round(a):
    """Round FP32 values to bfloat16 (nearest, ties to even) and back to FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
