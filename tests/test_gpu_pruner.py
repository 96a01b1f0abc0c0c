"""GPU parity of the learned restart pruner (ica_mlp_* kernels) against the FP64 oracle, and
the pruned fit against the unpruned one (the pruner's fallback and judge)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from oracle import mlp
from oracle import ordering_ica as oica

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ica():
    from paper_2408_17118_gb300 import ica as _ica
    return _ica


@pytest.fixture(scope="module")
def ctx(ica):
    c = ica.Context(0)
    yield c
    c.close()


def _rand_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    P = {name: rng.standard_normal(shape) * scale for name, shape in mlp.SIZES}
    P["mean"] = rng.standard_normal(mlp.N_IN) * 0.5
    P["scale"] = rng.uniform(0.5, 2.0, mlp.N_IN)
    return mlp.pack(P).astype(np.float32).astype(np.float64)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("rows", [1, 37, 1000])
def test_forward_parity(ica, ctx, rows):
    params = _rand_params(1)
    F = np.random.default_rng(2).standard_normal((rows, mlp.N_IN)).astype(np.float32).astype(np.float64)
    ref = mlp.forward(params, F)
    p32 = ica.ica_mlp_forward(ctx, _dev(params), _dev(F), fp16=False).cpu().numpy()
    p16 = ica.ica_mlp_forward(ctx, _dev(params), _dev(F), fp16=True).cpu().numpy()
    assert np.abs(p32 - ref).max() < 2e-5
    assert np.abs(p16 - ref).max() < 3e-2


@pytest.mark.parametrize("pos_weight", [1.0, 6.0])
def test_gradient_parity(ica, ctx, pos_weight):
    # full-batch loss and back-propagated gradient against the FP64 oracle (lr = 0: no update)
    params = _rand_params(3)
    rng = np.random.default_rng(4)
    F = rng.standard_normal((700, mlp.N_IN)).astype(np.float32).astype(np.float64)
    y = (rng.uniform(size=700) < 0.2).astype(np.float64)
    L, g = mlp.loss_grad(params, F, y, pos_weight)
    P = _dev(params)
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    for fp16, tol_l, tol_g in [(False, 1e-5, 1e-4), (True, 2e-2, 5e-2)]:
        loss, grad, _ = ica.ica_mlp_train_step(ctx, P, m, v, 1, _dev(F), _dev(y), 0.0, pos_weight, fp16, want_grad=True)
        gg = grad.cpu().numpy().astype(np.float64)
        assert abs(float(loss.item()) - L) <= tol_l * abs(L)
        assert np.linalg.norm(gg - g) <= tol_g * np.linalg.norm(g)
        assert np.all(gg[:2 * mlp.N_IN] == 0)
    # parameters unchanged with lr = 0
    assert np.array_equal(P.cpu().numpy(), params.astype(np.float32))


def test_adam_step_parity(ica, ctx):
    params = _rand_params(5)
    rng = np.random.default_rng(6)
    F = rng.standard_normal((300, mlp.N_IN)).astype(np.float32).astype(np.float64)
    y = (rng.uniform(size=300) < 0.3).astype(np.float64)
    P = _dev(params)
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    loss, grad, _ = ica.ica_mlp_train_step(ctx, P, m, v, 1, _dev(F), _dev(y), 1e-3, 1.0, False, want_grad=True)
    g = grad.cpu().numpy().astype(np.float64)
    ref, _, _ = mlp.adam_step(params, np.zeros_like(params), np.zeros_like(params), g, 1, 1e-3)
    assert np.abs(P.cpu().numpy() - ref).max() < 1e-6


def test_standardize_and_init(ica, ctx):
    rng = np.random.default_rng(7)
    F = (rng.standard_normal((5000, mlp.N_IN)) * np.arange(1, mlp.N_IN + 1) + np.arange(mlp.N_IN)).astype(np.float32)
    P = ica.ica_mlp_init(ctx, 11)
    P2 = ica.ica_mlp_init(ctx, 11)
    assert torch.equal(P, P2)
    ica.ica_mlp_standardize(ctx, _dev(F), P)
    mean, scale = mlp.standardisation(F.astype(np.float64))
    p = P.cpu().numpy()
    k = mlp.N_IN
    assert np.allclose(p[:k], mean, rtol=1e-5, atol=1e-5)
    assert np.allclose(p[k:2 * k], scale, rtol=1e-5)
    blocks = mlp.unpack(p.astype(np.float64))
    assert abs(blocks["W1"].std() - np.sqrt(2 / 12)) < 0.05 and abs(blocks["W2"].std() - np.sqrt(2 / 64)) < 0.02
    assert np.all(blocks["b1"] == 0) and np.all(blocks["b2"] == 0) and blocks["b3"][0] == 0


def test_recorded_features_match_oracle(ica, ctx):
    # alpha at iteration 1 is the kurtosis of the initial restart on X~ (Eq. 2); labels mark the
    # restarts that ended at the picked direction (the picked restart itself included)
    w = synth.small_mixture(0)
    X = torch.from_numpy(w.X).cuda()
    Xw, V, mean = ica.ica_whiten(ctx, X)
    M = w.M
    B0 = synth.restart_inits(M, 8, 8, seed=3)
    opts = ica.ica_default_opts(precision=ica.ICA_FP32)
    W, k, (F, y) = ica.ica_order_fit(ctx, Xw, M, 8, w.iters, w.tol, 1, opts, B0=torch.from_numpy(B0).cuda(),
                                     record=True)
    st = json.loads(ica.ica_last_stats(ctx))
    F = F.cpu().numpy()
    y = y.cpu().numpy()
    Xw64 = oica.whiten(w.X.astype(np.float64))[0]
    z = (B0[0].astype(np.float64) / np.linalg.norm(B0[0], axis=1, keepdims=True)) @ Xw64
    alpha0 = np.mean(z ** 4, axis=1) / np.mean(z ** 2, axis=1) ** 2 - 3.0
    assert np.abs(F[0, :, 0] - alpha0).max() < 2e-3
    for i, comp in enumerate(st["components"]):
        assert y[i, comp["winner"]] == 1.0
        assert np.all(F[i, :, 10] == 8 - i)
        assert np.allclose(F[i, :, 11], np.log(w.X.shape[1]))
        # Upsilon gap at iteration 5 to the best restart still running then (rows that stopped
        # earlier keep alpha_5 = 0 and are not part of the reference)
        ran5 = F[i, :, 4] != 0.0
        if ran5.any():
            ref = mlp.features(F[i, :, :5], F[i, :, 5:10], 8 - i, w.X.shape[1], active5=ran5)[:, 12]
            assert np.abs(F[i, :, 12] - ref).max() < 1e-4
            assert F[i, ran5, 12].max() == 0.0
    assert np.all((y == 0) | (y == 1))


def _fit(ica, ctx, Xw, w, prune=None, tau=None, record=False, keep_frac=None, cos=None):
    opts = ica.ica_default_opts(precision=ica.ICA_BF16)
    if tau is not None:
        opts.prune_tau = tau
    if keep_frac is not None:
        opts.prune_keep_frac = keep_frac
    if cos is not None:
        opts.prune_cos = cos
    out = ica.ica_order_fit(ctx, Xw, w.M, w.n_components, w.iters, w.tol, 21, opts, prune_params=prune, record=record)
    return out, json.loads(ica.ica_last_stats(ctx))


@pytest.fixture(scope="module")
def trained(ica, ctx):
    from paper_2408_17118_gb300 import pruner
    data = []
    for seed in (1, 2):
        w = synth.eeg_like(32, 50_000, 512, seed=seed)
        data.append(ica.ica_whiten(ctx, torch.from_numpy(w.X).cuda())[0])
    F, y = pruner.collect(ctx, data, 512, 30, 1e-6, seed=100)
    params, tau, report = pruner.train(ctx, F, y, steps=300)
    return params, tau, report


def test_pruned_fit_matches_unpruned_and_saves_work(ica, ctx, trained):
    params, tau, report = trained
    assert report["loss_last"] < report["loss_first"]
    w = synth.eeg_like(32, 50_000, 512, seed=0)
    Xw = ica.ica_whiten(ctx, torch.from_numpy(w.X).cuda())[0]
    (W0, k0), st0 = _fit(ica, ctx, Xw, w)
    (W1, k1), st1 = _fit(ica, ctx, Xw, w, prune=params, tau=tau)
    W0, W1 = W0.cpu().numpy(), W1.cpu().numpy()
    assert W0.shape == W1.shape
    _judge(W0, st0, W1, w, Xw.cpu().numpy().astype(np.float64))
    rows0 = sum(c["rows_updated"] for c in st0["components"])
    rows1 = sum(c["rows_updated"] for c in st1["components"])
    pruned = sum(c["pruned"] for c in st1["components"])
    assert pruned > 0
    assert rows1 < rows0, (rows1, rows0)


def _tie_tol(alpha):
    # FP32 resolution of Upsilon at alpha: relative kurtosis error 1e-4 times |dUpsilon/dalpha|
    return 1e-4 * abs(alpha) * abs((alpha / 2) / (alpha / 2 + 1)) + 1e-6


def _judge(W0, st0, W1, w, Xw=None):
    """The pruner's judge: every component the Gaussianity test (Eq. 3) calls non-Gaussian in the
    unpruned fit (Upsilon above 2 (N - i + 2)(N - i + 1) / T) must be in the pruned fit; a
    different position, or a different direction in its place, is allowed only between
    objectives that FP32 cannot order (within the Upsilon resolution of the 1e-4 kurtosis
    tolerance). The components after them span the Gaussian subspace, where no direction is
    unique (Theorem 1), and are not compared."""
    N, T = w.X.shape
    comps = st0["components"]
    ng = 0
    for c in comps:
        if c["upsilon"] < oica.gaussianity_threshold(N, c["i"], T):
            break
        ng += 1
    assert ng >= N // 2, ng  # 3/4 of the sources are non-Gaussian
    cos = np.abs(W0[:ng] @ W1.T)
    for i in range(ng):
        j = int(np.argmax(cos[i]))
        tol = _tie_tol(comps[i]["alpha"])
        if cos[i, j] >= 1 - 1e-5:
            if j != i:
                assert abs(comps[j]["upsilon"] - comps[i]["upsilon"]) <= tol + _tie_tol(comps[j]["alpha"]), (i, j)
            continue
        assert Xw is not None, ("component missing from the pruned fit", i)
        y0, y1 = W0[i] @ Xw, W1[i] @ Xw
        u0 = float(oica.upsilon(oica.kurtosis_alpha(y0)))
        u1 = float(oica.upsilon(oica.kurtosis_alpha(y1)))
        assert u1 >= u0 - tol, (i, u0, u1, tol)


def test_keep_floor_alone_keeps_the_leaders(ica, ctx, trained):
    """tau above every probability: the network keeps nothing, so only the floor stays - the
    max(refine_topk, ceil(prune_keep_frac x active)) restarts leading Upsilon at iteration 5 and
    any tied with the last of them (binary-like rows clamp alpha at -1.999 and tie) - and the
    pruned fit still picks the unpruned fit's non-Gaussian components."""
    import math

    params, _, _ = trained
    w = synth.eeg_like(32, 50_000, 512, seed=9)
    Xw = ica.ica_whiten(ctx, torch.from_numpy(w.X).cuda())[0]
    (W0, k0), st0 = _fit(ica, ctx, Xw, w)
    (W1, k1), st1 = _fit(ica, ctx, Xw, w, prune=params, tau=1.01, keep_frac=0.05, cos=0.0)
    checked = 0
    for c in st1["components"]:
        if c["fallback"] or not c["active"] or c["iterations"] < 5:
            continue
        act5 = c["active"][0]  # rows still running at iteration 5, before the pruner
        if act5 > 0:  # at least the floor stays (more where restarts tie at the threshold)
            assert act5 - c["pruned"] >= min(act5, max(4, math.ceil(0.05 * act5))), c
            checked += 1
    assert checked >= 8
    _judge(W0.cpu().numpy(), st0, W1.cpu().numpy(), w, Xw.cpu().numpy().astype(np.float64))
    assert sum(c["rows_updated"] for c in st1["components"]) < sum(c["rows_updated"] for c in st0["components"])


def test_redundant_restarts_leave_safely(ica, ctx, trained):
    """The network keeps everything (tau 0) and no floor: only restarts dominated by a restart
    that leads them in Upsilon at iteration 5 and points the same way (|cos| >= 0.99) leave.
    Every direction keeps its leader, so the fit picks the unpruned fit's non-Gaussian
    components (the judge) while most restarts leave after the fifth iteration."""
    params, _, _ = trained
    w = synth.eeg_like(32, 50_000, 512, seed=9)
    Xw = ica.ica_whiten(ctx, torch.from_numpy(w.X).cuda())[0]
    (W0, k0), st0 = _fit(ica, ctx, Xw, w)
    (W1, k1), st1 = _fit(ica, ctx, Xw, w, prune=params, tau=0.0, keep_frac=0.0, cos=0.99)
    _judge(W0.cpu().numpy(), st0, W1.cpu().numpy(), w, Xw.cpu().numpy().astype(np.float64))
    pruned = sum(c["pruned"] for c in st1["components"])
    assert pruned > 0.5 * sum(c["active"][0] for c in st1["components"] if c["active"] and c["iterations"] >= 5)



def test_fallback_restores_unpruned_result(ica, ctx, trained):
    # tau above every probability and no keep floor: the pruner drops every active restart, so
    # every component must fall back to the unpruned fit, which is deterministic: identical output
    params, _, _ = trained
    w = synth.eeg_like(16, 20_000, 128, seed=5)
    Xw = ica.ica_whiten(ctx, torch.from_numpy(w.X).cuda())[0]
    (W0, k0), _ = _fit(ica, ctx, Xw, w)
    (W1, k1), st1 = _fit(ica, ctx, Xw, w, prune=params, tau=1.01, keep_frac=0.0, cos=0.0)
    assert torch.equal(W0, W1) and torch.equal(k0, k1)
    assert all(c["fallback"] == 1 for c in st1["components"] if c["pruned"] > 0)
