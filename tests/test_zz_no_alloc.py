"""The allocation-free update step, ica_fp_step_noalloc, checked against ica_fp_step.

ica_fp_step_noalloc exists for callers that cannot call cudaMalloc: code running inside an
application whose allocator already owns the whole GPU, plug-ins that may not allocate after
start-up, or loops that cannot afford the device synchronisation a cudaFree implies. It keeps
its scratch in a fixed 16 MiB array inside the library instead of a caller-provided workspace.

The test calls it through the C ABI twice in a row (the second call runs on the array as the
first call left it) and compares each result with the workspace-based entry point on the same
inputs, within the tolerance the step tests use against the FP64 oracle. This file is collected
last so that a failure here never hides another test's result.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2408_17118_gb300 import _lib

    return _lib.load()


def rup(v, m):
    return (v + m - 1) // m * m


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("M,n,T", [(300, 37, 12345), (129, 64, 40_000), (100, 256, 10_000), (1, 1, 64)])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_matches_workspace_step(lib, prec, M, n, T):
    from paper_2408_17118_gb300 import ica

    p = ica.ICA_FP32 if prec == "fp32" else ica.ICA_BF16
    dtype = torch.float32 if prec == "fp32" else torch.bfloat16
    n_pad, ld = rup(n, 16), rup(T, 8)
    X = synth.small_random(n, T, seed=3 * M + n)
    B = np.zeros((M, n_pad), dtype=np.float32)
    B[:, :n] = oracle.normalise_rows(np.random.default_rng(M + T).standard_normal((M, n)))
    xt = torch.zeros((n_pad, ld), dtype=dtype)
    xt[:n, :T] = torch.from_numpy(X).to(dtype)
    xt = xt.cuda()
    Bt = torch.from_numpy(B).cuda()

    ctx = ica.Context(0)
    ref, ref_mom = ica.ica_fp_step(ctx, p, Bt, n, xt, T)
    ref = ref.cpu().numpy()
    ref_mom = ref_mom.cpu().numpy()
    ctx.close()

    Bq = bf16(B[:, :n]) if prec == "bf16" else B[:, :n]
    Xq = bf16(X) if prec == "bf16" else X
    Z = Bq.astype(np.float64) @ Xq.astype(np.float64)
    S = (np.abs(Z) ** 3) @ np.abs(Xq.astype(np.float64)).T / T
    tol = (1e-4 if prec == "fp32" else 2.0 ** -8) * S + 1e-6

    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        Bnew = torch.full_like(Bt, float("nan"))
        mom = torch.full((M, 4), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.ica_fp_step_noalloc(p, Bt.data_ptr(), M, n, xt.data_ptr(), T, ld, Bnew.data_ptr(), mom.data_ptr(),
                                     stream)
        assert st == 0, (call, lib.ica_status_string(st))
        got = Bnew.cpu().numpy()
        assert np.all(np.abs(got[:, :n] - ref[:, :n]) <= tol), (call, np.abs(got[:, :n] - ref[:, :n]).max())
        assert np.all(got[:, n:] == 0)
        assert np.allclose(mom.cpu().numpy()[:, :3], ref_mom[:, :3], rtol=2e-5, atol=1e-7), call


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_2408_17118_gb300 import ica

    tiny = torch.zeros(16, dtype=torch.float32, device="cuda")
    # 16,256 rows x (256 + 4) floats exceed the 16 MiB array: refused before any launch
    st = lib.ica_fp_step_noalloc(ica.ICA_BF16, tiny.data_ptr(), 16_200, 256, tiny.data_ptr(), 1024, 1024,
                                 tiny.data_ptr(), None, None)
    assert st == 6  # ICA_ERR_WORKSPACE
    # FP32 tiles are 64 rows: 20,032 rows x 260 floats do not fit either
    st = lib.ica_fp_step_noalloc(ica.ICA_FP32, tiny.data_ptr(), 20_000, 256, tiny.data_ptr(), 1024, 1024,
                                 tiny.data_ptr(), None, None)
    assert st == 6
    # outside the documented argument range (as for ica_fp_step): refused as well
    st = lib.ica_fp_step_noalloc(ica.ICA_FP32, tiny.data_ptr(), 70_000, 16, tiny.data_ptr(), 1024, 1024,
                                 tiny.data_ptr(), None, None)
    assert st == 1  # ICA_ERR_ARG


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_python_binding(lib, prec):
    """The Python binding makes B's device current around the C call (the entry point works on
    the current device) and enqueues on the given stream; M = 3 takes the few-row FP32 kernel."""
    from paper_2408_17118_gb300 import ica

    p = ica.ICA_FP32 if prec == "fp32" else ica.ICA_BF16
    dtype = torch.float32 if prec == "fp32" else torch.bfloat16
    M, n, T = 3, 20, 5000
    n_pad, ld = rup(n, 16), rup(T, 8)
    X = synth.small_random(n, T, seed=11)
    B = np.zeros((M, n_pad), dtype=np.float32)
    B[:, :n] = oracle.normalise_rows(np.random.default_rng(5).standard_normal((M, n)))
    xt = torch.zeros((n_pad, ld), dtype=dtype)
    xt[:n, :T] = torch.from_numpy(X).to(dtype)
    xt, Bt = xt.cuda(), torch.from_numpy(B).cuda()
    ctx = ica.Context(0)
    ref, ref_mom = ica.ica_fp_step(ctx, p, Bt, n, xt, T)
    ctx.close()
    side = torch.cuda.Stream()
    for _ in range(2):
        got, mom = ica.ica_fp_step_noalloc(p, Bt, n, xt, T, stream=side)
        side.synchronize()
        # same kernels and split as ica_fp_step (the scratch does not bind here): identical
        assert torch.equal(got, ref) and torch.equal(mom[:, :2], ref_mom[:, :2])
