"""Failure paths of the C ABI, provoked on the host's request without faulting the GPU.

* NaN or Inf in the raw data: ica_whiten reports ICA_ERR_NONFINITE (its row-mean pass sees the
  non-finite sum).
* A rank-deficient data matrix: the covariance has a zero eigenvalue, ICA_ERR_ILLCOND
  (Section 2.2: whitening needs a full-rank covariance).
* A deflation basis whose F~F~^T is singular (Section 3.3, Eq. 7: span(W) meets span(e_1..e_n)):
  ICA_ERR_ILLCOND.
* A bounded device wait that runs out: the persistent BF16 stage is asked (opts.stall_test) to
  wait at its first grid barrier for one arrival more than it has CTAs, with a 50 ms limit
  (opts.wait_ns). Every CTA gives up, frees TMEM and returns; the call reports ICA_ERR_TIMEOUT.

After each error the same context runs a normal fit and gets the result it got before.
"""
import time

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ica():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2408_17118_gb300 import ica as m

    return m


@pytest.fixture(scope="module")
def ctx(ica):
    c = ica.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def good(ica, ctx):
    """A normal fit of a small EEG-like mixture (the reference result after each error)."""
    w = synth.eeg_like(24, 20_000, 200, seed=3, n_components=6)
    X = torch.from_numpy(w.X).cuda()
    Xw, _, _ = ica.ica_whiten(ctx, X)
    W, k = ica.ica_order_fit(ctx, Xw, w.M, w.n_components, w.iters, w.tol, 5)
    return w, X, W.cpu().numpy(), k.cpu().numpy()


def refit_matches(ica, ctx, good):
    w, X, W0, k0 = good
    Xw, _, _ = ica.ica_whiten(ctx, X)
    W, k = ica.ica_order_fit(ctx, Xw, w.M, w.n_components, w.iters, w.tol, 5)
    assert np.array_equal(W.cpu().numpy(), W0) and np.array_equal(k.cpu().numpy(), k0)


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_nonfinite_input(ica, ctx, good, bad):
    w, X, _, _ = good
    Xb = X.clone()
    Xb[5, 1234] = bad
    with pytest.raises(ica.IcaError) as e:
        ica.ica_whiten(ctx, Xb)
    assert e.value.status == 3  # ICA_ERR_NONFINITE
    refit_matches(ica, ctx, good)


def test_rank_deficient_input(ica, ctx, good):
    w, X, _, _ = good
    Xb = X.clone()
    Xb[7] = Xb[2]  # two identical channels: the covariance is singular
    with pytest.raises(ica.IcaError) as e:
        ica.ica_whiten(ctx, Xb)
    assert e.value.status == 4  # ICA_ERR_ILLCOND
    refit_matches(ica, ctx, good)


@pytest.mark.parametrize("N,k", [(4, 1), (16, 3)])
def test_singular_reduction_basis(ica, ctx, good, N, k):
    """W = the first k unit vectors: F = I - W^T W has zero rows 0..k-1, so F~ (its first
    N - k rows, Eq. 7) has k zero rows and F~F~^T is singular."""
    W = torch.zeros((k, N), dtype=torch.float64, device="cuda")
    W[torch.arange(k), torch.arange(k)] = 1.0
    with pytest.raises(ica.IcaError) as e:
        ica.ica_deflation_basis(ctx, W, N)
    assert e.value.status == 4  # ICA_ERR_ILLCOND
    refit_matches(ica, ctx, good)


def test_bounded_wait_runs_out(ica, ctx, good):
    w, X, _, _ = good
    Xw, _, _ = ica.ica_whiten(ctx, X)
    opts = ica.ica_default_opts(precision=ica.ICA_BF16, wait_ns=50_000_000, stall_test=1)
    t0 = time.perf_counter()
    with pytest.raises(ica.IcaError) as e:
        ica.ica_order_fit(ctx, Xw, w.M, w.n_components, w.iters, w.tol, 5, opts)
    dt = time.perf_counter() - t0
    assert e.value.status == 5  # ICA_ERR_TIMEOUT
    assert dt < 1.5, dt  # gave up after the 50 ms limit, not the 2 s default
    refit_matches(ica, ctx, good)
    # the short limit alone (nothing stalls) changes nothing
    W, k = ica.ica_order_fit(ctx, Xw, w.M, w.n_components, w.iters, w.tol, 5,
                             ica.ica_default_opts(precision=ica.ICA_BF16, wait_ns=50_000_000))
    assert np.array_equal(W.cpu().numpy(), good[2])
