"""FP64 CPU oracle of the learned restart pruner (not part of the paper's method).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may use it.

The pruner is a small multilayer perceptron that reads, for one restart of one component, the
kurtosis alpha (Eq. 2) of the restart's row at the first five fixed-point iterations and the
step distance min(||b - b_prev||, ||b + b_prev||) of those iterations, the reduced dimension n,
log T, and how far the restart's objective Upsilon (Eq. 1) at iteration 5 lies below the best
one among the restarts still running then; it returns the probability that the restart ends
at the direction the component picks (Algorithm 2's global optimum). Upsilon is evaluated with
alpha clamped at -1.999 so that the gap stays finite for binary-like directions. Layout of the
parameter vector (float32 on the device, float64 here), shared with the library:

    mean[13], scale[13]            feature standardisation  x_hat = (x - mean) * scale
    W1[64][13], b1[64]             h1 = relu(W1 x_hat + b1)
    W2[64][64], b2[64]             h2 = relu(W2 h1 + b2)
    w3[64], b3                     logit = w3 . h2 + b3,  p = sigmoid(logit)

Loss (weighted binary cross-entropy, mean over the batch):
    L = -(1/B) sum_s [ w_pos y_s log p_s + (1 - y_s) log(1 - p_s) ]
whose derivative with respect to the logit is (1/B) (p_s (w_pos y_s + 1 - y_s) - w_pos y_s).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 13, 64
ALPHA_CLAMP = -1.999
SIZES = [("mean", (N_IN,)), ("scale", (N_IN,)), ("W1", (N_HID, N_IN)), ("b1", (N_HID,)),
         ("W2", (N_HID, N_HID)), ("b2", (N_HID,)), ("w3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(params: np.ndarray) -> dict:
    """Views of the named blocks of a flat parameter vector (layout above)."""
    out, off = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(params[off:off + k], dtype=np.float64).reshape(shape)
        off += k
    return out


def pack(blocks: dict) -> np.ndarray:
    return np.concatenate([np.asarray(blocks[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def upsilon_clamped(alpha) -> np.ndarray:
    """Eq. 1 with alpha clamped at ALPHA_CLAMP (finite everywhere)."""
    a = np.maximum(np.asarray(alpha, dtype=np.float64), ALPHA_CLAMP)
    return a - 2.0 * np.log(a / 2.0 + 1.0)


def features(alpha_traj: np.ndarray, step_traj: np.ndarray, n: int, T: int, active5=None) -> np.ndarray:
    """Rows of the 13 pruner inputs: alpha at iterations 1..5, step distance at 1..5, n, log T,
    and Upsilon(alpha_5) minus the largest Upsilon(alpha_5) among the rows marked active5 (the
    restarts still running at iteration 5; all rows when None)."""
    a = np.asarray(alpha_traj, dtype=np.float64)
    d = np.asarray(step_traj, dtype=np.float64)
    rows = a.shape[0]
    u5 = upsilon_clamped(a[:, 4])
    mask = np.ones(rows, dtype=bool) if active5 is None else np.asarray(active5, dtype=bool)
    ref = u5[mask].max() if mask.any() else 0.0
    return np.concatenate([a, d, np.full((rows, 1), float(n)), np.full((rows, 1), np.log(float(T))),
                           (u5 - ref)[:, None]], axis=1)


def standardisation(F: np.ndarray, eps: float = 1e-6):
    """Column means and reciprocal standard deviations (population form) of the features."""
    F = np.asarray(F, dtype=np.float64)
    mean = F.mean(axis=0)
    std = np.sqrt(((F - mean) ** 2).mean(axis=0))
    return mean, 1.0 / np.maximum(std, eps)


def forward(params: np.ndarray, F: np.ndarray, keep: bool = False):
    """Keep-probabilities p (rows,), and the intermediate activations when keep=True."""
    P = unpack(params)
    x = (np.asarray(F, dtype=np.float64) - P["mean"]) * P["scale"]
    a1 = x @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ P["w3"] + P["b3"][0]
    p = 1.0 / (1.0 + np.exp(-z))
    if keep:
        return p, {"x": x, "a1": a1, "h1": h1, "a2": a2, "h2": h2, "z": z}
    return p


def loss(params: np.ndarray, F: np.ndarray, y: np.ndarray, pos_weight: float = 1.0) -> float:
    p = forward(params, F)
    y = np.asarray(y, dtype=np.float64)
    eps = 1e-300
    return float(-np.mean(pos_weight * y * np.log(p + eps) + (1.0 - y) * np.log(1.0 - p + eps)))


def loss_grad(params: np.ndarray, F: np.ndarray, y: np.ndarray, pos_weight: float = 1.0):
    """Loss and its gradient with respect to every parameter (mean and scale get zero
    gradient: they are fixed by the training set, not learned), by back-propagation."""
    P = unpack(params)
    p, act = forward(params, F, keep=True)
    y = np.asarray(y, dtype=np.float64)
    B = F.shape[0]
    dz = (p * (pos_weight * y + 1.0 - y) - pos_weight * y) / B          # dL/dlogit
    g = {name: np.zeros(shape) for name, shape in SIZES}
    g["w3"] = act["h2"].T @ dz
    g["b3"] = np.array([dz.sum()])
    d2 = np.outer(dz, P["w3"]) * (act["a2"] > 0)
    g["W2"] = d2.T @ act["h1"]
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (act["a1"] > 0)
    g["W1"] = d1.T @ act["x"]
    g["b1"] = d1.sum(axis=0)
    return loss(params, F, y, pos_weight), pack(g)


def adam_step(params, m, v, grad, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015) of every parameter; returns new (params, m, v).
    The standardisation block (first 2 * N_IN entries) is left unchanged."""
    params = np.array(params, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    upd = lr * mh / (np.sqrt(vh) + eps)
    upd[:2 * N_IN] = 0.0
    return params - upd, m, v


def numeric_grad(params: np.ndarray, F: np.ndarray, y: np.ndarray, pos_weight: float = 1.0,
                 h: float = 1e-6, idx=None) -> np.ndarray:
    """Central finite differences of the loss (selected parameter indices, or all)."""
    idx = range(len(params)) if idx is None else idx
    out = np.zeros(len(params))
    for i in idx:
        e = np.zeros(len(params))
        e[i] = h
        out[i] = (loss(params + e, F, y, pos_weight) - loss(params - e, F, y, pos_weight)) / (2 * h)
    return out
