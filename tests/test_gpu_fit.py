"""End-to-end parity of ica_whiten + ica_order_fit against the FP64 oracle (Algorithm 2).

Bar (FP32 path and the BF16 path after its FP32 refinement): the same ordered components as
the oracle, |w_gpu . w_oracle| >= 1 - 1e-5 per component, relative kurtosis error <= 1e-4, and
W W^T = I to 1e-12 (the append runs in FP64 on an orthonormal basis). Where the oracle's own
Upsilon margin between two components is tiny the comparison would be decided by rounding;
such near-ties are reported by the assertion message instead of being silently passed.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2408_17118_gb300 import ica

    c = ica.Context(0)
    yield c
    c.close()


def gpu_fit(ctx, w, prec, B0=None, seed=0, gauss=False, iters=None, tol=None, **kw):
    from paper_2408_17118_gb300 import ica

    X = torch.from_numpy(w.X).cuda()
    Xw, V, mean = ica.ica_whiten(ctx, X)
    opts = ica.ica_default_opts(precision=prec, gauss_test=int(gauss), **kw)
    W, kurt = ica.ica_order_fit(ctx, Xw, w.M, w.n_components, iters or w.iters, tol or w.tol, seed, opts,
                                B0=None if B0 is None else torch.from_numpy(B0).cuda())
    torch.cuda.synchronize()
    return W.cpu().numpy(), kurt.cpu().numpy(), Xw, V.cpu().numpy()


def sign_near_tie(w, rel=1e-4):
    """The two largest magnitudes of w agree to `rel`: the canonical sign (largest-magnitude
    entry positive) is then decided by rounding and may differ between two correct fits."""
    a = np.sort(np.abs(w))[::-1]
    return len(a) > 1 and a[0] - a[1] <= rel * a[0]


def check_parity(W, kurt, ref, label):
    assert W.shape == ref.W.shape, (label, W.shape, ref.W.shape)
    assert np.abs(W @ W.T - np.eye(W.shape[0])).max() < 1e-12, label
    cos = np.sum(W * ref.W, axis=1)  # signed: both sides make the largest-magnitude entry positive
    ups = oracle.upsilon(ref.alpha)
    margin = np.abs(np.diff(ups)) if len(ups) > 1 else np.array([np.inf])
    assert np.all(np.abs(cos) >= 1 - 1e-5), (label, "cos", cos, "oracle Upsilon margins", margin)
    flipped = [i for i in range(len(cos)) if cos[i] < 0]
    assert all(sign_near_tie(ref.W[i]) for i in flipped), (label, "sign differs", flipped)
    rel = np.abs(kurt - ref.alpha) / np.abs(ref.alpha)
    assert np.all(rel <= 1e-4), (label, "rel kurtosis error", rel)


@pytest.fixture(scope="module")
def c1_ref():
    w = synth.small_mixture(0)
    B0 = synth.restart_inits(w.M, w.N, w.N, 1000)
    ref, Xw, V, mean = oracle.order_fit(w.X, w.M, w.N, w.iters, w.tol, B0)
    return w, B0, ref


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8", "plain"])
def test_c1_parity_explicit_restarts(ctx, c1_ref, prec):
    from paper_2408_17118_gb300 import ica

    p = {"fp32": ica.ICA_FP32, "bf16": ica.ICA_BF16, "fp8": ica.ICA_FP8, "plain": ica.ICA_PLAIN_FP32}[prec]
    w, B0, ref = c1_ref
    W, kurt, Xw, V = gpu_fit(ctx, w, p, B0=B0)
    check_parity(W, kurt, ref, prec)


def test_c1_parity_seeded_restarts(ctx):
    """No B0: the GPU draws restarts from Philox4x32-10 + Box-Muller; the oracle draws the same
    ones from its own implementation of that generator."""
    from paper_2408_17118_gb300 import ica

    w = synth.small_mixture(1)
    seed = 0x1234_5678_9ABC
    B0 = oracle.seeded_B0(seed, w.M, w.N, w.N)
    ref, _, _, _ = oracle.order_fit(w.X, w.M, w.N, w.iters, w.tol, B0)
    W, kurt, _, _ = gpu_fit(ctx, w, ica.ICA_BF16, seed=seed)
    check_parity(W, kurt, ref, "seeded bf16")


@pytest.mark.parametrize("N,T,M,ncomp", [(16, 3000, 100, 16), (33, 5000, 1, 5), (20, 4097, 300, 20),
                                         (40, 2000, 129, 12)])
def test_ragged_shapes(ctx, N, T, M, ncomp):
    from paper_2408_17118_gb300 import ica

    kinds = [synth.SMALL_SOURCES[i % 8] for i in range(N)]
    w = synth.generators._mix(f"r{N}", kinds, T, N + T, M, 100, 1e-8, n_components=ncomp)
    B0 = synth.restart_inits(M, N, ncomp, 7)
    ref, _, _, _ = oracle.order_fit(w.X, M, ncomp, 100, 1e-8, B0)
    for p in (ica.ICA_FP32, ica.ICA_BF16):
        W, kurt, _, _ = gpu_fit(ctx, w, p, B0=B0)
        check_parity(W, kurt, ref, f"N{N} T{T} M{M} p{p}")


def test_gaussianity_test(ctx):
    """Eq. 3 stop on the Section 4.2 N=30 data (20 GGD + 10 Gaussian sources)."""
    from paper_2408_17118_gb300 import ica

    w = synth.ggd_paper(0, with_gaussians=True, M=100)
    B0 = synth.restart_inits(100, 30, 30, 5)
    ref, _, _, _ = oracle.order_fit(w.X, 100, 30, 30, 1e-6, B0, gauss_test=True)
    W, kurt, _, _ = gpu_fit(ctx, w, ica.ICA_BF16, B0=B0, gauss=True, iters=30, tol=1e-6)
    assert W.shape[0] == ref.W.shape[0] == 20
    check_parity(W, kurt, ref, "gauss-test")


def test_determinism(ctx, c1_ref):
    from paper_2408_17118_gb300 import ica

    w, B0, ref = c1_ref
    a = gpu_fit(ctx, w, ica.ICA_BF16, B0=B0)
    b = gpu_fit(ctx, w, ica.ICA_BF16, B0=B0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_full_size_eeg_like_sampled(ctx):
    """The N=64, T=200,000, M=1024 fit (the bench configuration, BF16): properties that hold at
    any size, plus sampled FP64 checks of individual components:
    orthonormal W; each sampled w a fixed point of the Algorithm 1 update (projected onto the
    complement of the earlier components); its kurtosis equal to the oracle's FP64 kurtosis of
    y = w Xw; and no FP64 FastICA run from 16 fresh restarts on component 1 beating it."""
    from paper_2408_17118_gb300 import ica

    w = synth.eeg64(0)
    W, kurt, Xw, V = gpu_fit(ctx, w, ica.ICA_BF16, seed=11)
    assert W.shape == (64, 64)
    assert np.abs(W @ W.T - np.eye(64)).max() < 1e-12
    Xw = Xw.cpu().numpy().astype(np.float64)
    T = w.T
    for i in (0, 1, 17, 40, 63):
        wi = W[i]
        y = wi @ Xw
        a = oracle.kurtosis_alpha(y)
        assert abs(kurt[i] - a) <= 1e-4 * abs(a) + 1e-6, (i, kurt[i], a)
        if i < 63:
            E = W[:i].T @ W[:i]
            v = Xw @ (y * y * y) / T - 3.0 * wi
            v = v - E @ v
            v /= np.linalg.norm(v)
            assert abs(v @ wi) >= 1 - 1e-8, (i, 1 - abs(v @ wi))
    ups0 = oracle.upsilon(kurt[0])
    rng = np.random.default_rng(3)
    for l in range(16):
        w0 = rng.standard_normal(64)
        wl, yl, _, _ = oracle.fastica_run(w0, Xw, np.zeros((64, 64)), 30, 1e-6)
        assert oracle.upsilon(oracle.kurtosis_alpha(yl)) <= ups0 + 1e-6, l


@pytest.mark.parametrize("N,T,M,ncomp,seed", [(80, 12_003, 300, 5, 85), (128, 16_001, 300, 6, 129),
                                              (136, 12_345, 130, 6, 136), (256, 12_007, 130, 5, 256)])
def test_wide_stage_parity(ctx, N, T, M, ncomp, seed):
    """Reduced dimensions above 64: the persistent BF16 stage takes its 128-sample-chunk form
    (n_pad 80 and 128) and its 64-sample-chunk form with a 256-column accumulator (n_pad 144 and
    256); whitening runs the FP64 Jacobi at m = N. EEG-like mixtures (the workload's source mix
    and noise), ragged T and restart tiles. Same bar as the small case against the FP64 oracle."""
    import json

    from paper_2408_17118_gb300 import ica

    # seeds whose oracle winners are each reached by many restarts (at these small T a winner
    # reached by a single restart is common, and its trajectory may leave the basin under BF16
    # rounding: a different, equally valid pick rather than an error of the kernels)
    w = synth.eeg_like(N, T, M, seed=seed, iters=100, tol=1e-8, n_components=ncomp)
    B0 = synth.restart_inits(M, N, ncomp, 13 + seed)
    ref, _, _, _ = oracle.order_fit(w.X, M, ncomp, 100, 1e-8, B0)
    W, kurt, _, _ = gpu_fit(ctx, w, ica.ICA_BF16, B0=B0)
    st = json.loads(ica.ica_last_stats(ctx))
    assert st["stage_persistent_launches"] >= ncomp, st["stage_persistent_note"]
    check_parity(W, kurt, ref, f"N{N} T{T} M{M} bf16")
    W, kurt, _, _ = gpu_fit(ctx, w, ica.ICA_FP32, B0=B0)
    check_parity(W, kurt, ref, f"N{N} T{T} M{M} fp32")
    # FP8 form: iterations 1..3 of each stage on E4M3 operands (n rounded up to 32: the padded K
    # of the 8-bit products), then BF16 and the FP32 refinement
    W, kurt, _, _ = gpu_fit(ctx, w, ica.ICA_FP8, B0=B0)
    st = json.loads(ica.ica_last_stats(ctx))
    assert st["stage_fp8_launches"] >= ncomp, st
    check_parity(W, kurt, ref, f"N{N} T{T} M{M} fp8")


@pytest.mark.parametrize("case", ["small", "eeg32", "ragged", "wide100", "wide200"])
def test_persistent_stage_equals_per_launch(ctx, case):
    """The persistent cooperative BF16 stage (one launch per component: update, grid barrier,
    row completion, grid barrier, removal of converged rows) runs the same arithmetic as the
    per-launch update + finalize path: identical W, kurtoses and restart updates. The persistent
    stage reports the exact iteration count; the per-launch loop learns the active count only
    every fourth iteration and counts the empty launches before that read. At 64-sample chunks
    (n_pad > 128, case wide200) the persistent stage issues the first product's two BF16 terms
    into two accumulators and adds them in the epilogue, where the per-launch kernel accumulates
    both in one: the same fixed points up to FP32 rounding there."""
    import json

    from paper_2408_17118_gb300 import ica

    if case == "small":
        w = synth.small_mixture(0)
    elif case == "eeg32":
        w = synth.eeg_like(32, 50_000, 512, seed=4)
    elif case == "ragged":
        w = synth.eeg_like(21, 9_999, 300, seed=5)  # ragged n, T and M
    elif case == "wide100":  # n_pad 112 .. 96: 128-sample chunks, two second-product issuers
        w = synth.eeg_like(100, 20_000, 300, seed=6, n_components=8)
    else:  # n_pad 208: 64-sample chunks, one issuer, 256-column accumulator
        w = synth.eeg_like(200, 12_000, 200, seed=7, n_components=4)
    out = []
    for persistent in (1, 0):  # (equal work shares off: the per-launch path's split of the samples)
        W, kurt, _, _ = gpu_fit(ctx, w, ica.ICA_BF16, seed=7, stage_persistent=persistent, stage_streamk=0)
        st = json.loads(ica.ica_last_stats(ctx))
        out.append((W, kurt, st))
    (W0, k0, s0), (W1, k1, s1) = out
    assert s0["stage_persistent_launches"] >= 1 and s1["stage_persistent_launches"] == 0
    if case == "wide200":
        assert np.all(np.sum(W0 * W1, axis=1) >= 1 - 1e-6)
        assert np.all(np.abs(k0 - k1) <= 1e-5 * np.abs(k1))
        for c0, c1 in zip(s0["components"], s1["components"]):
            assert abs(c0["rows_updated"] - c1["rows_updated"]) <= 0.02 * c1["rows_updated"]
        return
    assert np.array_equal(W0, W1) and np.array_equal(k0, k1)
    for c0, c1 in zip(s0["components"], s1["components"]):
        assert c0["rows_updated"] == c1["rows_updated"] and c0["refine_rows"] == c1["refine_rows"]
        assert c0["iterations"] <= c1["iterations"] < c0["iterations"] + 4


def test_certify_full_size_eeg_like(ctx):
    """The bench configuration (EEG-like N=64, T=200,000, M=1024, BF16 with FP32 refinement) is
    too large for the full FP64 oracle; its picks are certified in FP64 instead: for each of the
    48 non-Gaussian components the library records its refined distinct candidates
    (opts.record_cands), and oracle.certify_picks refines the pick and every candidate with the
    FP64 FastICA run of Algorithm 1 (projected onto the complement of the fit's earlier
    components) and compares their objectives as Algorithm 2's argmax does. Each pick must be
    an FP64 fixed point (|cos| >= 1 - 1e-5 with its refinement) and no distinct candidate may
    beat it by more than the FP32 error of Upsilon."""
    from paper_2408_17118_gb300 import ica

    w = synth.eeg64(0)
    X = torch.from_numpy(w.X).cuda()
    Xw, V, mean = ica.ica_whiten(ctx, X)
    opts = ica.ica_default_opts(precision=ica.ICA_BF16)
    cands = torch.zeros((w.n_components, opts.refine_topk, w.N), dtype=torch.float64, device="cuda")
    W, kurt = ica.ica_order_fit(ctx, Xw, w.M, w.n_components, w.iters, w.tol, 11, opts, record_cands=cands)
    W, kurt, cands = W.cpu().numpy(), kurt.cpu().numpy(), cands.cpu().numpy()
    Xw64 = Xw.cpu().numpy().astype(np.float64)
    assert np.abs(W @ W.T - np.eye(64)).max() < 1e-12
    n_ng = 48  # 3/4 of the sources are non-Gaussian
    for i in range(n_ng):  # the pick is one of the recorded candidates
        assert np.max(np.abs(cands[i] @ W[i])) >= 1 - 1e-12, i
    checks = oracle.certify_picks(Xw64, W, cands, K=30, eps=1e-9, components=range(n_ng))
    for c in checks:
        assert c.pick_cos >= 1 - 1e-5, c
        assert c.margin >= -1e-4 * max(1.0, abs(c.ups_pick)), c
        assert abs(kurt[c.i] - c.alpha_pick) <= 1e-4 * abs(c.alpha_pick), (c, kurt[c.i])
    assert sum(c.candidates > 1 for c in checks) >= n_ng // 2  # most components compare >1 candidate


@pytest.mark.parametrize("L", [1, 3, 10, 30, 100])
def test_gaussianity_count_sweep(ctx, L):
    """Section 4.2, second experiment (Fig. 2a): the number of non-Gaussian sources the
    Gaussianity test (Eq. 3) estimates on the N = 30 data (20 generalised-Gaussian + 10
    Gaussian sources, T = 10,000) as a function of the number of restarts L. For each L and
    two random initialisations the GPU fit (BF16 stage + FP32 refinement) must estimate the
    same count as the FP64 oracle from the same initial restarts; from L = 10 on (each optimum
    then reached by several restarts) also the same components. With one or three restarts a
    component is whatever optimum its single trajectory reaches, and the BF16 stage's first
    iterations (one BF16 term) may send it into a neighbouring basin: there only the count,
    the quantity the experiment measures, is compared."""
    from paper_2408_17118_gb300 import ica

    w = synth.ggd_paper(0, with_gaussians=True, M=L)
    for run in range(2):
        B0 = synth.restart_inits(L, 30, 30, 1000 + 17 * run + L)
        ref, _, _, _ = oracle.order_fit(w.X, L, 30, 30, 1e-6, B0, gauss_test=True)
        W, kurt, _, _ = gpu_fit(ctx, w, ica.ICA_BF16, B0=B0, gauss=True, iters=30, tol=1e-6)
        assert W.shape[0] == ref.W.shape[0], (L, run, W.shape[0], ref.W.shape[0])
        if L >= 10:
            check_parity(W, kurt, ref, f"L{L} run{run}")


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("case", ["small", "ragged"])
def test_algorithm1_parity(ctx, prec, case):
    """Algorithm 1's form on the GPU (opts.algorithm = 1: every iteration on the full whitened
    data, the found components projected out of each update and of the N-dimensional initial
    restarts) against the FP64 oracle's Algorithm 1 from the same initial vectors."""
    from paper_2408_17118_gb300 import ica

    p = {"fp32": ica.ICA_FP32, "bf16": ica.ICA_BF16, "fp8": ica.ICA_FP8}[prec]
    if case == "small":
        w = synth.small_mixture(0)
        iters, tol = w.iters, w.tol
    else:
        kinds = [synth.SMALL_SOURCES[i % 8] for i in range(20)]
        w = synth.generators._mix("r20", kinds, 4097, 24, 300, 100, 1e-8, n_components=12)
        iters, tol = 100, 1e-8
    B0 = synth.restart_inits(w.M, w.N, w.n_components, 1000 + w.N)
    ref, _, _, _ = oracle.order_fit(w.X, w.M, w.n_components, iters, tol, B0, algorithm=1, full_init=True)
    W, kurt, _, _ = gpu_fit(ctx, w, p, B0=B0, iters=iters, tol=tol, algorithm=1)
    check_parity(W, kurt, ref, f"alg1 {case} {prec}")


def test_fluctuation_of_algorithms_1_and_2(ctx):
    """Section 4.3's run-to-run fluctuation (1 - |cos| between runs from different random
    restarts, averaged over run pairs) on an EEG-like mixture, for both algorithms on the GPU:
    the strongly non-Gaussian leading components are unique, so both algorithms reproduce them
    across runs (fluctuation near 0), and both find the same ones."""
    from paper_2408_17118_gb300 import ica

    w = synth.eeg_like(32, 50_000, 256, seed=12, n_components=12)
    runs = {1: [], 2: []}
    for alg in (1, 2):
        for seed in (101, 202, 303):
            W, _, _, _ = gpu_fit(ctx, w, ica.ICA_BF16, seed=seed, algorithm=alg)
            runs[alg].append(W)
    f1, f2 = ica.fluctuation(runs[1]), ica.fluctuation(runs[2])
    assert f1.shape == f2.shape == (12,)
    # (two sources whose objectives tie within FP32 may trade places between runs)
    assert np.sum(f1[:8] < 1e-5) >= 6 and np.sum(f2[:8] < 1e-5) >= 6, (f1, f2)
    cross = np.max(np.abs(runs[1][0][:8] @ runs[2][0][:8].T), axis=1)  # same directions, any order
    assert np.all(cross >= 1 - 1e-5), cross


@pytest.mark.parametrize("N,M", [(48, 2560), (200, 8192)])
def test_stage_equal_work_shares(ctx, N, M):
    """M restarts = 20 or 64 restart tiles: the one-wave shape (2 sample splits per tile at 64
    tiles, 7 at 20) leaves 24 and 12 of the 152 SMs idle, so the persistent stage hands every CTA
    an equal share of the (tile x chunk) work instead. Same fixed points as the one-wave shape:
    the same components (|cos| >= 1 - 1e-5) and kurtoses (relative 1e-5), summation order aside."""
    import json

    from paper_2408_17118_gb300 import ica

    w = synth.eeg_like(N, 20_000, M, seed=N + 1, n_components=4)
    res = []
    for sk in (1, 0):
        W, kurt, _, _ = gpu_fit(ctx, w, ica.ICA_BF16, seed=3, stage_streamk=sk)
        st = json.loads(ica.ica_last_stats(ctx))
        res.append((W, kurt, st))
    (W1, k1, s1), (W0, k0, s0) = res
    assert s1["stage_streamk_first_iteration"] == 1 and s0["stage_streamk_first_iteration"] == 0
    assert np.all(np.abs(np.sum(W1 * W0, axis=1)) >= 1 - 1e-5)
    assert np.all(np.abs(k1 - k0) <= 1e-5 * np.abs(k0))
