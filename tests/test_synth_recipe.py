"""CPU checks of the seeded input recipe (synth/): the workload shapes and source mixes the
benchmarks and parity tests stand on, sources standardised, noise level, reproducibility."""
import numpy as np

import synth

NON_GAUSS_SUPER = {"laplace", "t4", "t6", "t10"}
NON_GAUSS_SUB = {"uniform", "binary", "sinusoid"}


def test_small_mixture_recipe():
    w = synth.small_mixture(0)
    assert (w.N, w.T, w.M, w.n_components) == (8, 10_000, 64, 8)
    assert w.kinds == ["laplace", "uniform", "t5", "binary", "exp", "laplace2", "uniform", "gauss"]
    assert w.iters == 200 and w.tol == 1e-10
    S = w.S.astype(np.float64)
    assert np.abs(S.mean(axis=1)).max() < 1e-6
    assert np.abs((S * S).mean(axis=1) - 1.0).max() < 1e-5
    # no noise: X is the mixture itself
    assert np.allclose(w.X, (w.A.astype(np.float32) @ w.S), atol=1e-5)


def test_eeg_like_recipe():
    w = synth.eeg_like(64, 20_000, 16, seed=3, keep_sources=True)
    assert (w.N, w.T, w.M, w.n_components, w.iters, w.tol) == (64, 20_000, 16, 64, 30, 1e-6)
    sup = [k for k in w.kinds if k in NON_GAUSS_SUPER]
    sub = [k for k in w.kinds if k in NON_GAUSS_SUB]
    gauss = [k for k in w.kinds if k == "gauss"]
    assert len(sup) == 24 and len(sub) == 24 and len(gauss) == 16
    S = w.S.astype(np.float64)
    assert np.abs(S.mean(axis=1)).max() < 1e-6
    assert np.abs((S * S).mean(axis=1) - 1.0).max() < 1e-5
    # sensor noise sigma = 0.05 on every channel
    resid = w.X.astype(np.float64) - w.A @ S
    assert abs(resid.std() - 0.05) < 2e-3


def test_eeg64_is_the_benchmark_shape():
    w = synth.eeg64(0)
    assert (w.N, w.T, w.M, w.n_components) == (64, 200_000, 1024, 64)
    assert w.X.dtype == np.float32 and w.X.flags["C_CONTIGUOUS"]


def test_batch_recipe_shapes():
    ws = synth.batch_of_datasets(count=32, seed=1, T_lo=200, T_hi=4000)
    assert len(ws) == 32
    assert {w.N for w in ws} <= {16, 32, 48, 64, 96, 128}
    assert len({w.N for w in ws}) >= 4  # uneven N
    assert all(200 <= w.T <= 4000 for w in ws)
    assert all(w.M == 512 for w in ws)


def test_reproducible_and_seeded():
    a = synth.small_mixture(5, T=2000)
    b = synth.small_mixture(5, T=2000)
    c = synth.small_mixture(6, T=2000)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.A, b.A)
    assert not np.array_equal(a.X, c.X)
    B0 = synth.restart_inits(64, 8, 8, 1000)
    assert B0.shape == (8, 64, 8) and B0.dtype == np.float32
    assert np.array_equal(B0, synth.restart_inits(64, 8, 8, 1000))
