"""Python binding of the ordering-ICA C ABI: the same entry points as include/ica.h.

Argument marshalling only. Device buffers are torch CUDA tensors (torch provides device memory
and the stream); every computation runs in libica.so's kernels. Each function raises
``IcaError`` when the library returns a non-zero status.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import ICA_BF16, ICA_FP8, ICA_FP32, ICA_MLP_IN, ICA_MLP_PARAMS, ICA_PLAIN_FP32, ica_dataset, ica_opts  # noqa: F401


class IcaError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _lib.load()
        msg = lib.ica_status_string(status).decode()
        detail = lib.ica_last_error().decode() if status == 2 else ""
        super().__init__(f"{where}: {msg} (status {status})" + (f": {detail}" if detail else ""))
        self.status = status


def _check(status: int, where: str):
    if status != 0:
        raise IcaError(status, where)


def _ptr(t: torch.Tensor | None, dtype=None, name: str = "tensor") -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


class Context:
    """An ica_ctx bound to one device, torch's current stream and a torch-allocated workspace."""

    def __init__(self, device: int = 0):
        self.lib = _lib.load()
        self.device = device
        h = C.c_void_p()
        _check(self.lib.ica_create(C.byref(h), device), "ica_create")
        self.handle = h
        self.workspace = None
        self.set_stream(torch.cuda.current_stream(device))

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        _check(self.lib.ica_set_stream(self.handle, C.c_void_p(stream.cuda_stream)), "ica_set_stream")

    def ensure_workspace(self, N: int, T: int, M: int, opts: ica_opts | None = None):
        need = self.lib.ica_workspace_bytes(N, T, M, C.byref(opts) if opts is not None else None)
        if need == 0:
            raise ValueError(f"invalid sizes N={N} T={T} M={M}")
        if self.workspace is None or self.workspace.numel() < need:
            self.workspace = torch.empty(need, dtype=torch.uint8, device=f"cuda:{self.device}")
        _check(self.lib.ica_set_workspace(self.handle, C.c_void_p(self.workspace.data_ptr()), self.workspace.numel()),
               "ica_set_workspace")

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.lib.ica_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ica_default_opts(**overrides) -> ica_opts:
    o = ica_opts()
    _lib.load().ica_default_opts(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def ica_status_string(status: int) -> str:
    return _lib.load().ica_status_string(status).decode()


def ica_workspace_bytes(N: int, T: int, M: int, opts: ica_opts | None = None) -> int:
    return int(_lib.load().ica_workspace_bytes(N, T, M, C.byref(opts) if opts is not None else None))


def ica_whiten(ctx: Context, X: torch.Tensor, Xw: torch.Tensor | None = None):
    """X: N x T float32 (CUDA). Returns (Xw float32 N x T, V float64 N x N, mean float64 N)."""
    N, T = X.shape
    Xw = torch.empty_like(X) if Xw is None else Xw
    V = torch.empty((N, N), dtype=torch.float64, device=X.device)
    mean = torch.empty(N, dtype=torch.float64, device=X.device)
    ctx.ensure_workspace(N, T, 1, ica_default_opts(precision=ICA_FP32))
    _check(ctx.lib.ica_whiten(ctx.handle, _ptr(X, torch.float32, "X"), N, T, _ptr(Xw, torch.float32, "Xw"),
                              _ptr(V), _ptr(mean)), "ica_whiten")
    return Xw, V, mean


def ica_order_fit(ctx: Context, Xw: torch.Tensor, M: int, n_components: int, iters: int, tol: float, seed: int,
                  opts: ica_opts | None = None, B0: torch.Tensor | None = None,
                  prune_params: torch.Tensor | None = None, record: bool = False,
                  record_cands: torch.Tensor | None = None):
    """Fast ordering ICA on whitened Xw (N x T float32). Returns (W float64 n_found x N,
    kurtosis float64 n_found); with record=True also (features n_components x M x ICA_MLP_IN,
    labels n_components x M) for training the restart pruner. record_cands (optional, float64
    n_components x refine_topk x N, BF16 precision) receives each component's refined distinct
    candidates in the whitened space."""
    N, T = Xw.shape
    opts = ica_default_opts() if opts is None else opts
    if B0 is not None:
        if B0.shape != (n_components, M, N):
            raise ValueError("B0 must be n_components x M x N")
        opts.B0 = _ptr(B0, torch.float32, "B0")
    if prune_params is not None:
        if prune_params.numel() != ICA_MLP_PARAMS:
            raise ValueError(f"prune_params must hold {ICA_MLP_PARAMS} floats")
        opts.prune_params = _ptr(prune_params, torch.float32, "prune_params")
    rec = None
    if record:
        rec = (torch.zeros((n_components, M, ICA_MLP_IN), dtype=torch.float32, device=Xw.device),
               torch.zeros((n_components, M), dtype=torch.float32, device=Xw.device))
        opts.record_features = rec[0].data_ptr()
        opts.record_labels = rec[1].data_ptr()
    if record_cands is not None:
        if tuple(record_cands.shape) != (n_components, opts.refine_topk, N):
            raise ValueError("record_cands must be n_components x refine_topk x N")
        opts.record_cands = _ptr(record_cands, torch.float64, "record_cands")
    ctx.ensure_workspace(N, T, M, opts)
    W = torch.zeros((n_components, N), dtype=torch.float64, device=Xw.device)
    kurt = torch.zeros(n_components, dtype=torch.float64, device=Xw.device)
    nf = C.c_int(0)
    _check(ctx.lib.ica_order_fit(ctx.handle, _ptr(Xw, torch.float32, "Xw"), N, T, M, n_components, iters, float(tol),
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, C.byref(opts), _ptr(W), _ptr(kurt), C.byref(nf)),
           "ica_order_fit")
    if record:
        return W[: nf.value], kurt[: nf.value], rec
    return W[: nf.value], kurt[: nf.value]


def ica_order_fit_batched(ctx: Context, Xws: list, M: int, iters: int, tol: float, seed: int,
                          opts: ica_opts | None = None, n_components: list | None = None, workers: int = 0):
    """Fits every whitened data set of the list (N_k x T_k float32 CUDA tensors) concurrently.
    Returns a list of (W float64 n_found x N_k, kurtosis float64 n_found)."""
    opts = ica_default_opts() if opts is None else opts
    count = len(Xws)
    sets = (ica_dataset * count)()
    outs, founds = [], [C.c_int(0) for _ in range(count)]
    for k, Xw in enumerate(Xws):
        N, T = Xw.shape
        nc = N if n_components is None else int(n_components[k])
        W = torch.zeros((nc, N), dtype=torch.float64, device=Xw.device)
        kurt = torch.zeros(nc, dtype=torch.float64, device=Xw.device)
        outs.append((W, kurt))
        sets[k].Xw = _ptr(Xw, torch.float32, "Xw")
        sets[k].N, sets[k].T, sets[k].n_components = N, T, nc
        sets[k].W_out, sets[k].kurt_out = W.data_ptr(), kurt.data_ptr()
        sets[k].n_found = C.pointer(founds[k])
    need = ctx.lib.ica_batched_workspace_bytes(sets, count, M, C.byref(opts), workers)
    if need == 0:
        raise ValueError("invalid batch sizes")
    if ctx.workspace is None or ctx.workspace.numel() < need:
        ctx.workspace = torch.empty(need, dtype=torch.uint8, device=f"cuda:{ctx.device}")
    _check(ctx.lib.ica_set_workspace(ctx.handle, C.c_void_p(ctx.workspace.data_ptr()), ctx.workspace.numel()),
           "ica_set_workspace")
    _check(ctx.lib.ica_order_fit_batched(ctx.handle, sets, count, M, iters, float(tol), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                         C.byref(opts), workers), "ica_order_fit_batched")
    return [(W[: f.value], k[: f.value]) for (W, k), f in zip(outs, founds)]


def ica_last_stats(ctx: Context) -> str:
    buf = C.create_string_buffer(1 << 20)
    _check(ctx.lib.ica_last_stats(ctx.handle, buf, len(buf)), "ica_last_stats")
    return buf.value.decode()


def ica_init_restarts(ctx: Context, seed: int, component: int, M: int, n: int, ldb: int | None = None,
                      device: int = 0) -> torch.Tensor:
    ldb = n if ldb is None else ldb
    B = torch.empty((M, ldb), dtype=torch.float32, device=f"cuda:{device}")
    _check(ctx.lib.ica_init_restarts(ctx.handle, int(seed) & 0xFFFFFFFFFFFFFFFF, component, M, n, _ptr(B), ldb),
           "ica_init_restarts")
    return B


def ica_deflation_basis(ctx: Context, W: torch.Tensor, N: int) -> torch.Tensor:
    k = W.shape[0]
    G = torch.empty((N - k, N), dtype=torch.float64, device=W.device)
    ctx.ensure_workspace(N, 8, 1, ica_default_opts(precision=ICA_FP32))
    _check(ctx.lib.ica_deflation_basis(ctx.handle, _ptr(W, torch.float64, "W") if k else None, k, N, _ptr(G)),
           "ica_deflation_basis")
    return G


def _ld(T: int) -> int:
    return (T + 7) // 8 * 8


def ica_reduce(ctx: Context, G: torch.Tensor, Xw: torch.Tensor, want32: bool = True, want16: bool = True):
    """X~ = G Xw. Returns (Xt32 n_pad x ld float32 or None, Xt16 n_pad x ld bfloat16 or None)."""
    n, N = G.shape
    T = Xw.shape[1]
    n_pad = (n + 15) // 16 * 16
    ld = _ld(T)
    Xt32 = torch.empty((n_pad, ld), dtype=torch.float32, device=Xw.device) if want32 else None
    Xt16 = torch.empty((n_pad, ld), dtype=torch.bfloat16, device=Xw.device) if want16 else None
    _check(ctx.lib.ica_reduce(ctx.handle, _ptr(G, torch.float64, "G"), n, N, _ptr(Xw, torch.float32, "Xw"), T,
                              _ptr(Xt32), ld, _ptr(Xt16), ld), "ica_reduce")
    return Xt32, Xt16


def ica_quantize_e4m3(ctx: Context, Xt32: torch.Tensor, n: int, T: int):
    """E4M3 copy of the FP32 reduced data (rows 0..n-1 of Xt32, row stride Xt32.shape[1]).
    Returns (X8 uint8 n8 x ld8 raw E4M3 bytes, scales float32 3 n8 + 1)."""
    n8 = (n + 31) // 32 * 32
    ld8 = (T + 15) // 16 * 16
    o = ica_default_opts()
    o.precision = ICA_FP8
    ctx.ensure_workspace(n, T, 1, o)
    X8 = torch.empty((n8, ld8), dtype=torch.uint8, device=Xt32.device)
    sc = torch.empty(3 * n8 + 1, dtype=torch.float32, device=Xt32.device)
    _check(ctx.lib.ica_quantize_e4m3(ctx.handle, _ptr(Xt32, torch.float32, "Xt32"), n, T, Xt32.shape[1], _ptr(X8),
                                     ld8, _ptr(sc)), "ica_quantize_e4m3")
    return X8, sc


def _xt_args(Xt: torch.Tensor, precision: int):
    want = torch.float32 if precision == ICA_FP32 else torch.bfloat16
    if Xt.dtype != want:
        raise ValueError(f"Xt must be {want} for precision {precision}")
    return _ptr(Xt, want, "Xt"), Xt.shape[1]


def ica_fp_step(ctx: Context, precision: int, B: torch.Tensor, n: int, Xt: torch.Tensor, T: int):
    """One un-normalised matrix-form update of the M rows of B (M x n_pad float32).
    Returns (Bnew M x n_pad float32, moments M x 4 float32)."""
    M, n_pad = B.shape
    xp, ldx = _xt_args(Xt, precision)
    ctx.ensure_workspace(n, T, M, ica_default_opts(precision=precision))
    Bnew = torch.empty_like(B)
    mom = torch.empty((M, 4), dtype=torch.float32, device=B.device)
    _check(ctx.lib.ica_fp_step(ctx.handle, precision, _ptr(B, torch.float32, "B"), M, n, xp, T, ldx, _ptr(Bnew),
                               _ptr(mom)), "ica_fp_step")
    return Bnew, mom


def ica_kurtosis(ctx: Context, precision: int, B: torch.Tensor, n: int, Xt: torch.Tensor, T: int):
    """alpha and Upsilon (float64, M each) of the rows of B on reduced data Xt."""
    M, n_pad = B.shape
    xp, ldx = _xt_args(Xt, precision)
    ctx.ensure_workspace(n, T, M, ica_default_opts(precision=precision))
    a = torch.empty(M, dtype=torch.float64, device=B.device)
    u = torch.empty(M, dtype=torch.float64, device=B.device)
    _check(ctx.lib.ica_kurtosis(ctx.handle, precision, _ptr(B, torch.float32, "B"), M, n, xp, T, ldx, _ptr(a),
                                _ptr(u)), "ica_kurtosis")
    return a, u


def ica_fp_step_noalloc(precision: int, B: torch.Tensor, n: int, Xt: torch.Tensor, T: int,
                        stream: torch.cuda.Stream | None = None):
    """ica_fp_step without a context or workspace: for callers that cannot allocate device
    memory (the library keeps its scratch in a fixed 16 MiB array per GPU). Returns
    (Bnew, moments); the output tensors here are allocated by torch only for this binding's
    convenience - a C caller passes its own."""
    M, n_pad = B.shape
    xp, ldx = _xt_args(Xt, precision)
    if Xt.device != B.device:
        raise ValueError("B and Xt must be on the same device")
    stream = torch.cuda.current_stream(B.device) if stream is None else stream
    Bnew = torch.empty_like(B)
    mom = torch.empty((M, 4), dtype=torch.float32, device=B.device)
    with torch.cuda.device(B.device):  # the C call works on the current device
        _check(_lib.load().ica_fp_step_noalloc(precision, _ptr(B, torch.float32, "B"), M, n, xp, T, ldx, _ptr(Bnew),
                                               _ptr(mom), C.c_void_p(stream.cuda_stream)), "ica_fp_step_noalloc")
    return Bnew, mom


def fluctuation(Ws) -> "np.ndarray":
    """Run-to-run fluctuation of the components of several fits (Section 4.3, an analysis of the
    outputs, no device work): for component i, the mean over ordered pairs of runs (t != u) of
    1 - |cos(w_i^t, w_i^u)|. Ws: list of (n x N) arrays or tensors; the shortest fit bounds i."""
    import numpy as np

    Ws = [np.asarray(w.cpu() if hasattr(w, "cpu") else w, dtype=np.float64) for w in Ws]
    R = len(Ws)
    if R < 2:
        raise ValueError("fluctuation needs at least two runs")
    n = min(w.shape[0] for w in Ws)
    unit = [w[:n] / np.linalg.norm(w[:n], axis=1, keepdims=True) for w in Ws]
    acc = np.zeros(n)
    for t in range(R):
        for u in range(R):
            if t != u:
                acc += 1.0 - np.abs(np.sum(unit[t] * unit[u], axis=1))
    return acc / (R * (R - 1))


# ------------------------------------------------------------------ learned restart pruner
def ica_mlp_init(ctx: Context, seed: int, params: torch.Tensor | None = None) -> torch.Tensor:
    params = torch.empty(ICA_MLP_PARAMS, dtype=torch.float32, device=f"cuda:{ctx.device}") if params is None else params
    _check(ctx.lib.ica_mlp_init(ctx.handle, int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(params, torch.float32, "params")),
           "ica_mlp_init")
    return params


def ica_mlp_standardize(ctx: Context, F: torch.Tensor, params: torch.Tensor):
    rows = F.shape[0]
    _check(ctx.lib.ica_mlp_standardize(ctx.handle, _ptr(F, torch.float32, "F"), rows,
                                       _ptr(params, torch.float32, "params")), "ica_mlp_standardize")


def ica_mlp_forward(ctx: Context, params: torch.Tensor, F: torch.Tensor, fp16: bool = True) -> torch.Tensor:
    rows = F.shape[0]
    prob = torch.empty(rows, dtype=torch.float32, device=F.device)
    _check(ctx.lib.ica_mlp_forward(ctx.handle, _ptr(params, torch.float32, "params"), _ptr(F, torch.float32, "F"),
                                   rows, int(fp16), _ptr(prob)), "ica_mlp_forward")
    return prob


def ica_mlp_scratch_bytes(rows: int) -> int:
    return int(_lib.load().ica_mlp_scratch_bytes(rows))


def ica_mlp_train_step(ctx: Context, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int,
                       F: torch.Tensor, y: torch.Tensor, lr: float, pos_weight: float = 1.0, fp16: bool = True,
                       scratch: torch.Tensor | None = None, want_grad: bool = False):
    """One training step; returns (loss tensor [1], grad tensor or None, scratch)."""
    rows = F.shape[0]
    need = ica_mlp_scratch_bytes(rows)
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(need, dtype=torch.uint8, device=F.device)
    loss = torch.empty(1, dtype=torch.float32, device=F.device)
    grad = torch.empty(ICA_MLP_PARAMS, dtype=torch.float32, device=F.device) if want_grad else None
    _check(ctx.lib.ica_mlp_train_step(ctx.handle, _ptr(params, torch.float32, "params"), _ptr(m), _ptr(v), int(step),
                                      _ptr(F, torch.float32, "F"), _ptr(y, torch.float32, "y"), rows, float(lr),
                                      float(pos_weight), int(fp16), C.c_void_p(scratch.data_ptr()), scratch.numel(),
                                      _ptr(loss), _ptr(grad)), "ica_mlp_train_step")
    return loss, grad, scratch
