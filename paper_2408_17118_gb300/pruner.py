"""Training driver of the learned restart pruner (not part of the paper's method).

The network and its kernels live in the library (ica_mlp_* in include/ica.h); this module only
orders the calls: record the method's own restart trajectories with ica_order_fit(record=True),
standardise the inputs, run full-batch Adam steps with ica_mlp_train_step, and pick the keep
threshold from the positives' predicted probabilities. Every arithmetic step runs on the GPU in
the library's kernels.
"""
from __future__ import annotations

import time

import torch

from . import ica


def collect(ctx: ica.Context, datasets, M: int, iters: int, tol: float, seed: int, opts=None):
    """Record (features, labels) of every restart of every component of each whitened data set
    (a list of N x T float32 CUDA tensors). Returns (F rows x ICA_MLP_IN, y rows) on the device."""
    Fs, ys = [], []
    for k, Xw in enumerate(datasets):
        N = Xw.shape[0]
        o = ica.ica_default_opts() if opts is None else opts
        _, _, (F, y) = ica.ica_order_fit(ctx, Xw, M, N, iters, tol, seed + k, o, record=True)
        Fs.append(F.reshape(-1, ica.ICA_MLP_IN))
        ys.append(y.reshape(-1))
    return torch.cat(Fs).contiguous(), torch.cat(ys).contiguous()


def collect_sets(ctx: ica.Context, sets, iters: int, tol: float, seed: int, opts=None):
    """As collect, for data sets with their own restart counts: sets = [(Xw, M), ...]."""
    Fs, ys = [], []
    for k, (Xw, M) in enumerate(sets):
        F, y = collect(ctx, [Xw], M, iters, tol, seed + k, opts)
        Fs.append(F)
        ys.append(y)
    return torch.cat(Fs).contiguous(), torch.cat(ys).contiguous()


def train(ctx: ica.Context, F: torch.Tensor, y: torch.Tensor, steps: int = 300, lr: float = 3e-3, seed: int = 7,
          fp16: bool = True, recall: float = 0.999, tau_cap: float = 0.5):
    """Train from scratch; returns (params, tau, report). tau keeps at least `recall` of the
    positive training rows (capped at tau_cap)."""
    t0 = time.perf_counter()
    params = ica.ica_mlp_init(ctx, seed)
    ica.ica_mlp_standardize(ctx, F, params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    n_pos = float(y.sum().item())
    n_neg = float(y.numel()) - n_pos
    pos_weight = max(1.0, min(50.0, n_neg / max(n_pos, 1.0)))
    scratch = None
    losses = []
    for step in range(1, steps + 1):
        loss, _, scratch = ica.ica_mlp_train_step(ctx, params, m, v, step, F, y, lr, pos_weight, fp16, scratch)
        if step == 1 or step == steps:
            losses.append(float(loss.item()))
    p = ica.ica_mlp_forward(ctx, params, F, fp16=True)
    pos = p[y > 0.5]
    if pos.numel():
        q = torch.quantile(pos.double(), 1.0 - recall).item()
        tau = float(min(tau_cap, q))
    else:
        tau = tau_cap
    keep_neg = float(((p >= tau) & (y < 0.5)).sum().item()) / max(n_neg, 1.0)
    report = {"rows": int(y.numel()), "positives": int(n_pos), "pos_weight": pos_weight, "loss_first": losses[0],
              "loss_last": losses[-1], "tau": tau, "train_recall": float((pos >= tau).double().mean().item()) if pos.numel() else None,
              "negatives_kept": keep_neg, "train_seconds": time.perf_counter() - t0, "steps": steps}
    return params, tau, report
