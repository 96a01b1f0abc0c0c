"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: known-answer vectors,
closed forms, invariants the paper states, a brute-force search, or an independent numerical
derivative. Together they are chosen so that a dropped term, a wrong sign, a wrong index or a
transposed operand anywhere in ``oracle/`` fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from conftest import GOLDEN


# ------------------------------------------------------------------ random initial restarts
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        ctr, key, want = v[0:4], v[4:6], tuple(v[6:10])
        assert oracle.philox4x32_10(ctr, key) == want
        got = oracle.philox4x32_10_np(*[np.array([c], dtype=np.uint64) for c in ctr], key[0], key[1])
        assert tuple(int(g[0]) for g in got) == want


def test_restart_normals_are_standard_normal():
    from scipy import stats
    z = oracle.restart_normals(seed=12345, component=3, M=4000, n=50).ravel()
    assert abs(z.mean()) < 5.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # odd n takes the cosine half of the last pair; rows differ, components differ
    a = oracle.restart_normals(7, 0, 3, 5)
    b = oracle.restart_normals(7, 1, 3, 5)
    assert a.shape == (3, 5) and not np.allclose(a, b)
    assert np.array_equal(oracle.restart_normals(7, 0, 3, 6)[:, :5], a)


def test_uniform52_open_interval():
    u = oracle.uniform52(np.array([0, 0xFFFFFFFF], dtype=np.uint64), np.array([0, 0xFFFFFFFF], dtype=np.uint64))
    assert u[0] > 0.0 and u[1] < 1.0
    assert u[0] == 2.0 ** -53 and u[1] == 1.0 - 2.0 ** -53


# ------------------------------------------------------------------ Eq. 1 / Eq. 2 / Eq. 3
def test_upsilon_properties():
    a = np.linspace(-1.999, 50.0, 20001)
    u = oracle.upsilon(a)
    assert np.all(u >= -1e-15)
    assert oracle.upsilon(0.0) == 0.0
    # small-alpha series: -2 log(1 + a/2) = -a + a^2/4 - a^3/12 + a^4/32 - a^5/80 + ...
    for s in (1e-3, -1e-3, 2e-2, -3e-2):
        series = s * s / 4.0 - s ** 3 / 12.0 + s ** 4 / 32.0
        assert abs(oracle.upsilon(s) - series) < abs(s) ** 5 / 40.0 + 1e-15  # + rounding of log(1 + a/2)
    # increasing in |alpha| on each side of 0, diverging at alpha = -2
    assert np.all(np.diff(u[a > 0]) > 0) and np.all(np.diff(u[a < 0]) < 0)
    assert oracle.upsilon(-2.0) == math.inf and oracle.upsilon(-1.999999) > 20.0
    # Theorem 1 example: a uniform source (-1.2) ranks above a t_10 source (+1) by Upsilon
    assert oracle.upsilon(-1.2) > oracle.upsilon(1.0)


def test_kurtosis_of_known_distributions():
    tab = {l.split()[0]: float(l.split()[1]) for l in open(os.path.join(GOLDEN, "closed_form_kurtosis.txt"))
           if l.strip() and not l.startswith("#")}
    T = 2_000_000
    tol = {"laplace": 0.1, "uniform": 0.01, "t6": 1.0, "t10": 0.15, "gauss": 0.02, "exp": 0.4,
           "binary": 1e-9, "sinusoid": 2e-2, "laplace2": 15.0}  # sinusoid: non-integer cycle count
    for kind, want in tab.items():
        raw = synth.make_source(kind, synth.rng_for(5, 99), T)
        y = synth.standardise(raw)
        if kind == "binary":  # exact for the sample: two-point law with P(+1) = p
            p = np.mean(raw > 0); q = 1 - p
            assert abs(want - (1 - 6 * 0.25) / 0.25) < 1e-15
            want = (1 - 6 * p * q) / (p * q)
        assert abs(oracle.kurtosis_alpha(y) - want) < tol[kind], kind
    # generalised Gaussian closed form (Section 4.2 sources)
    for rho in (2 * 2 ** (-10 / 4), 2 * 2 ** (-1 / 4), 2 * 2 ** (1 / 4), 2 * 2 ** (10 / 4)):
        g = math.gamma
        want = g(5 / rho) * g(1 / rho) / g(3 / rho) ** 2 - 3
        y = synth.standardise(synth.ggd_source(synth.rng_for(6, 1), rho, T))
        assert abs(oracle.kurtosis_alpha(y) - want) < max(0.02, 0.15 * abs(want)), rho


def test_gaussianity_threshold_formula_shape():
    # Eq. 3 is zero-free and shrinks as 1/T and as the remaining dimension falls
    assert oracle.gaussianity_threshold(30, 1, 10_000) == 2 * 31 * 30 / 10_000
    assert oracle.gaussianity_threshold(30, 30, 10_000) == 2 * 2 * 1 / 10_000


# ------------------------------------------------------------------ whitening
def test_whitening_invariants():
    w = synth.small_mixture(3, T=5000)
    Xw, V, mean = oracle.whiten(w.X)
    T = w.T
    assert np.abs(Xw.mean(axis=1)).max() < 1e-12
    assert np.abs(Xw @ Xw.T / T - np.eye(w.N)).max() < 1e-12
    assert np.abs(V - V.T).max() < 1e-12 * np.abs(V).max()
    assert np.linalg.eigvalsh(V).min() > 0  # symmetric positive definite: the unique ZCA matrix
    Xc = w.X.astype(np.float64) - w.X.astype(np.float64).mean(axis=1, keepdims=True)
    assert np.abs(mean - w.X.astype(np.float64).mean(axis=1)).max() < 1e-12
    assert np.abs(V @ Xc - Xw).max() < 1e-10


# ------------------------------------------------------------------ Section 3.3 deflation basis
@pytest.mark.parametrize("N,k", [(8, 1), (8, 4), (8, 7), (20, 13), (33, 5)])
def test_deflation_basis_invariants(N, k):
    rng = np.random.default_rng(N * 100 + k)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    W = Q[:k]
    G = oracle.deflation_basis(W, N)
    n = N - k
    assert G.shape == (n, N)
    assert np.abs(G @ G.T - np.eye(n)).max() < 1e-10            # orthonormal rows
    assert np.abs(W @ G.T).max() < 1e-10                        # orthogonal to found rows
    assert np.abs(G.T @ G - (np.eye(N) - W.T @ W)).max() < 1e-10  # spans the whole complement
    Ft = (np.eye(N) - W.T @ W)[:n]
    R = G @ Ft.T                                                # polar factor: F~ G^T = (F~F~^T)^(1/2)
    assert np.abs(R - R.T).max() < 1e-10 and np.linalg.eigvalsh((R + R.T) / 2).min() > 0
    assert np.abs(R @ R - Ft @ Ft.T).max() < 1e-10


@pytest.mark.parametrize("delta", [1e-5, 1e-6])
def test_deflation_basis_near_singular(delta):
    """Eq. 7 with found rows that nearly contain e_0 (a unit vector of the first n coordinates):
    w_0 = (e_0 + delta e_{N-1}) / norm, so F~F~^T has an eigenvalue of at most about delta^2
    (1e-10, 1e-12). The basis is still accepted and correct to the accuracy FP64 eigenpairs allow: length
    along the bad eigenvector within about eps / delta^2, direction within eps / delta."""
    N, k = 12, 3
    rng = np.random.default_rng(5)
    w0 = np.zeros(N)
    w0[0], w0[N - 1] = 1.0, delta
    w0 /= np.linalg.norm(w0)
    rest = rng.standard_normal((k - 1, N))
    rest -= np.outer(rest @ w0, w0)
    q, _ = np.linalg.qr(rest.T)
    W = np.vstack([w0, q.T[: k - 1]])
    assert np.abs(W @ W.T - np.eye(k)).max() < 1e-14
    n = N - k
    Ft = (np.eye(N) - W.T @ W)[:n]
    lam = np.linalg.eigvalsh(Ft @ Ft.T)
    assert 0.0 < lam.min() <= 1.01 * delta * delta
    G = oracle.deflation_basis(W, N)
    eps = np.finfo(np.float64).eps
    assert np.abs(G @ G.T - np.eye(n)).max() < 100 * eps / lam.min()
    assert np.abs(W @ G.T).max() < 100 * eps / np.sqrt(lam.min())


def test_deflation_basis_refuses_singular():
    """An exactly singular F~F~^T (a found row equal to e_0) is refused."""
    N = 6
    W = np.zeros((1, N))
    W[0, 0] = 1.0
    with pytest.raises(np.linalg.LinAlgError):
        oracle.deflation_basis(W, N)


# ------------------------------------------------------------------ Section 3.1 matrix update
def test_matrix_update_is_kurtosis_gradient():
    """B' + 3B must equal the gradient of J(b) = mean((b X~)^4)/4, checked row by row by
    central finite differences (independent of the closed-form update)."""
    Xt = synth.small_random(6, 3000, seed=4).astype(np.float64)
    rng = np.random.default_rng(0)
    B = rng.standard_normal((5, 6))
    U = oracle.matrix_update(B, Xt)
    J = lambda b: np.mean((b @ Xt) ** 4) / 4.0
    h = 1e-5
    for r in range(B.shape[0]):
        g = np.empty(6)
        for k in range(6):
            e = np.zeros(6); e[k] = h
            g[k] = (J(B[r] + e) - J(B[r] - e)) / (2 * h)
        assert np.allclose(U[r] + 3.0 * B[r], g, rtol=1e-7, atol=1e-8), r


def test_step_distance_sign_tolerant():
    b = oracle.normalise_rows(np.array([[1.0, 2.0, 2.0], [3.0, 0.0, 4.0]]))
    assert np.allclose(oracle.step_distance(b, -b), 0.0)
    assert np.allclose(oracle.step_distance(b, b), 0.0)
    assert np.allclose(np.sum(b * b, axis=1), 1.0)
    c = b.copy(); c[0] = [0.0, 0.0, 1.0]
    assert oracle.step_distance(c, b)[0] == pytest.approx(min(np.linalg.norm(c[0] - b[0]), np.linalg.norm(c[0] + b[0])))


# ------------------------------------------------------------------ end-to-end on the N=8 workload
def test_orthonormal_output(small_oracle):
    w, B0, res, Xw, V, mean = small_oracle
    assert res.W.shape == (8, 8)
    assert np.abs(res.W @ res.W.T - np.eye(8)).max() < 1e-12


def test_recovery_and_order(small_oracle):
    """Theorem 1: W V A is a signed permutation (Amari index) and the components come out in
    descending Upsilon of the sources' kurtosis (here the sample kurtosis of each true source)."""
    w, B0, res, Xw, V, mean = small_oracle
    P = res.W @ V @ w.A
    assert oracle.amari_index(P) < 3e-2  # T = 1e4: finite-sample error ~ T^-1/2
    src = np.argmax(np.abs(P), axis=1)
    assert sorted(src) == list(range(8))
    S = w.S.astype(np.float64)
    alpha_true = oracle.kurtosis_alpha(S)
    ups_true = oracle.upsilon(alpha_true)
    # standard error of each source's sample Upsilon: delta method on alpha = mean(y^4) - 3,
    # se(alpha) = std(y^4) / sqrt(T), dUpsilon/dalpha = (alpha/2) / (alpha/2 + 1)
    se_alpha = np.std(S ** 4, axis=1) / math.sqrt(w.T)
    se_ups = np.abs((alpha_true / 2.0) / (alpha_true / 2.0 + 1.0)) * se_alpha
    seq, se = ups_true[src], se_ups[src]
    for k in range(len(seq) - 1):
        # a swap of neighbours is allowed only where the sample Upsilon values are within three
        # standard errors of each other (the finite-sample order is then not resolved)
        assert seq[k] >= seq[k + 1] or abs(seq[k] - seq[k + 1]) < 3.0 * math.hypot(se[k], se[k + 1]), k
    assert np.all(np.diff(oracle.upsilon(res.alpha)) <= 1e-9)


@pytest.mark.slow
def test_recovery_large_T():
    w = synth.small_mixture(1, T=100_000)
    B0 = synth.restart_inits(w.M, w.N, w.N, 1001)
    res, Xw, V, mean = oracle.order_fit(w.X, w.M, w.N, w.iters, w.tol, B0)
    assert oracle.amari_index(res.W @ V @ w.A) < 1e-2


def test_gaussian_component(small_oracle):
    w, B0, res, Xw, V, mean = small_oracle
    assert abs(res.alpha[-1]) <= 3.0 * math.sqrt(24.0 / w.T)


def test_fixed_point_residual(small_oracle):
    """At convergence the update maps each found w to +-w (Algorithm 1 form, full space)."""
    w, B0, res, Xw, V, mean = small_oracle
    T = w.T
    for i in range(7):
        wi = res.W[i]
        E = res.W[:i].T @ res.W[:i]
        y = wi @ Xw
        v = Xw @ (y * y * y) / T - 3.0 * wi
        v = v - E @ v
        v = v / np.linalg.norm(v)
        tol = 1e-9 if res.iterations[i].min() < w.iters else 1e-5
        assert min(np.linalg.norm(v - wi), np.linalg.norm(v + wi)) < tol, i


def test_last_component_is_the_remaining_direction(small_oracle):
    w, B0, res, Xw, V, mean = small_oracle
    _, _, vt = np.linalg.svd(res.W[:7])
    null = vt[-1]
    assert abs(abs(null @ res.W[7]) - 1.0) < 1e-12
    assert res.iterations[7].max() == 1


def test_algorithm1_equals_algorithm2():
    """Reduction of signals (Section 3.3) changes no trajectory: the batched reduced iteration
    with w = G^T b equals the per-initialisation projected iteration."""
    w = synth.small_mixture(2, T=4000, M=16)
    B0 = synth.restart_inits(16, 8, 8, 77)
    Xw, V, mean = oracle.whiten(w.X)
    r2 = oracle.fast_ordering_ica(Xw, 16, 60, 1e-10, B0)
    r1 = oracle.ordering_ica_original(Xw, 16, 60, 1e-10, B0)
    for u1, u2 in zip(r1.upsilon_all, r2.upsilon_all):  # every restart, not only the winner
        assert np.abs(u1 - u2).max() < 1e-9 * max(1.0, np.abs(u1).max())
    assert np.abs(r1.W - r2.W).max() < 1e-8
    assert np.abs(r1.alpha - r2.alpha).max() < 1e-10
    for a, b in zip(r1.iterations, r2.iterations):
        assert np.array_equal(a, b)


def test_two_dimensional_brute_force():
    """N = 2: the first component must sit at the global maximum of Upsilon over all unit
    vectors (cos t, sin t), found by a dense angle grid plus golden-section refinement."""
    T = 20_000
    S = np.vstack([synth.standardise(synth.make_source("laplace", synth.rng_for(3, 0), T)),
                   synth.standardise(synth.make_source("uniform", synth.rng_for(3, 1), T))])
    A = np.array([[1.0, 0.6], [-0.4, 1.3]])
    X = (A @ S).astype(np.float32)
    B0 = synth.restart_inits(8, 2, 2, 5)
    res, Xw, V, mean = oracle.order_fit(X, 8, 2, 200, 1e-12, B0)
    f = lambda t: float(oracle.upsilon(oracle.kurtosis_alpha(np.cos(t) * Xw[0] + np.sin(t) * Xw[1])))
    th = np.linspace(0, math.pi, 100_000, endpoint=False)
    Y = np.outer(np.cos(th[::10]), Xw[0]) + np.outer(np.sin(th[::10]), Xw[1])  # coarse pass
    vals = oracle.upsilon(oracle.kurtosis_alpha(Y))
    t0 = th[::10][int(np.argmax(vals))]
    lo, hi = t0 - 2e-4 * 10, t0 + 2e-4 * 10
    g = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        a, b = hi - g * (hi - lo), lo + g * (hi - lo)
        if f(a) > f(b):
            hi = b
        else:
            lo = a
    tbest = (lo + hi) / 2
    w1 = res.W[0]
    t_or = math.atan2(w1[1], w1[0]) % math.pi
    d = abs(t_or - tbest) % math.pi
    assert min(d, math.pi - d) < 1e-6
    assert abs(res.W[1] @ w1) < 1e-12


def test_invariance_to_invertible_transform(small_oracle):
    """Separated signals y = W V (X - mean) do not depend on an invertible transform of X."""
    w, B0, res, Xw, V, mean = small_oracle
    Q = np.random.default_rng(3).standard_normal((8, 8))
    X2 = (Q @ w.X.astype(np.float64))
    res2, Xw2, V2, mean2 = oracle.order_fit(X2, w.M, w.N, w.iters, w.tol, B0)
    Y1 = res.W @ Xw
    Y2 = res2.W @ Xw2
    for i in range(7):
        c = abs(Y1[i] @ Y2[i]) / w.T
        assert c > 1 - 1e-6, (i, c)


def test_gaussianity_test_counts_non_gaussian_sources():
    """Eq. 3 stopping rule on the Section 4.2 second experiment: 20 generalised-Gaussian sources
    plus 10 Gaussian ones (N = 30, T = 10,000, L = 100). The test must stop after exactly the
    20 non-Gaussian components."""
    w = synth.ggd_paper(0, with_gaussians=True, M=100)
    B0 = synth.restart_inits(100, 30, 30, 5)
    res, Xw, V, mean = oracle.order_fit(w.X, 100, 30, 30, 1e-6, B0, gauss_test=True)
    assert res.W.shape[0] == 20
    P = np.abs(res.W @ V @ w.A)
    assert set(np.argmax(P, axis=1)) == set(range(20))  # all non-Gaussian sources, no Gaussian one


def test_canonical_sign():
    """Q7 reading of the sign of w (Algorithm 2 leaves it free): the largest-magnitude entry is
    made positive, the first one on ties."""
    assert np.array_equal(oracle.canonical_sign(np.array([0.3, -0.8, 0.5])), [-0.3, 0.8, -0.5])
    assert np.array_equal(oracle.canonical_sign(np.array([0.3, 0.8, -0.5])), [0.3, 0.8, -0.5])
    assert np.array_equal(oracle.canonical_sign(np.array([-0.6, 0.6, 0.1])), [0.6, -0.6, -0.1])  # tie: index 0
    assert np.array_equal(oracle.canonical_sign(np.array([0.6, -0.6, 0.1])), [0.6, -0.6, 0.1])
    assert np.array_equal(oracle.canonical_sign(np.array([0.0, -1e-300])), [0.0, 1e-300])
    w = np.array([0.1, -0.2, 0.3, -0.9])
    assert np.array_equal(oracle.canonical_sign(-w), oracle.canonical_sign(w))  # sign-invariant


def test_fit_rows_have_canonical_sign(small_oracle):
    w, B0, res, Xw, V, mean = small_oracle
    for row in res.W:
        k = int(np.argmax(np.abs(row)))
        assert row[k] > 0 and np.all(np.abs(row[:k]) < abs(row[k]))


def test_amari_index_values():
    assert oracle.amari_index(np.eye(4)) == 0.0
    P = np.array([[0, 2.0, 0], [0, 0, -1.0], [3.0, 0, 0]])
    assert oracle.amari_index(P) == 0.0
    assert oracle.amari_index(np.array([[1.0, 0.5], [0.5, 1.0]])) == pytest.approx(0.5)


def test_fluctuation_metric():
    a = np.eye(3)
    assert np.allclose(oracle.fluctuation([a, -a, a]), 0.0)
    b = np.array([[0, 1.0, 0], [1.0, 0, 0], [0, 0, 1.0]])
    f = oracle.fluctuation([a, b])
    assert np.allclose(f, [1.0, 1.0, 0.0])


# ------------------------------------------------------------------ FP64 certification of picks
def _distinct_top(trace, k, thresh=1.0 - 1e-3):
    """The k best restarts of one oracle component by Upsilon, distinct directions only, mapped
    to the whitened space (w = b G, Section 3.3)."""
    order = np.argsort(-trace.upsilon, kind="stable")
    picked = []
    for r in order:
        b = trace.B_final[r] / np.linalg.norm(trace.B_final[r])
        if all(abs(b @ q) < thresh for q in picked):
            picked.append(b)
        if len(picked) == k:
            break
    rows = [b @ trace.G for b in picked]
    return np.array([r / np.linalg.norm(r) for r in rows])


def _cands_of(res, k):
    N = res.W.shape[1]
    C = np.zeros((len(res.traces), k, N))
    for i, tr in enumerate(res.traces):
        top = _distinct_top(tr, k)
        C[i, : len(top)] = top
    return C


def test_certify_accepts_the_oracle_picks(small_oracle):
    """Algorithm 2's own picks pass: each is an FP64 fixed point and no distinct candidate among
    its component's best restarts has a larger Upsilon."""
    w, B0, res, Xw, V, mean = small_oracle
    checks = oracle.certify_picks(Xw, res.W, _cands_of(res, 4), K=200, eps=1e-12)
    assert len(checks) == 8
    for c in checks:
        assert c.pick_cos >= 1 - 1e-12, c
        assert c.margin >= -1e-9, c
        assert c.ups_pick == pytest.approx(float(oracle.upsilon(res.alpha[c.i])), rel=1e-9, abs=1e-12)
    assert sum(c.candidates > 1 for c in checks) >= 5  # the comparison is not vacuous


def test_certify_flags_a_wrong_pick(small_oracle):
    """A planted mistake: component 0's pick replaced by its runner-up (a distinct direction with
    a smaller Upsilon). The check must report a negative margin for that component."""
    w, B0, res, Xw, V, mean = small_oracle
    C = _cands_of(res, 4)
    W = res.W.copy()
    W[0] = C[0, 1]
    c = oracle.certify_picks(Xw, W, C, K=200, eps=1e-12, components=[0])[0]
    assert c.margin < -1e-3, c


def test_certify_two_dimensional_brute_force():
    """N = 2: the pick at the brute-force maximum of Upsilon over the unit circle passes, its
    refined objective equals the brute-force value, and a pick 0.3 rad away is flagged."""
    T = 20_000
    S = np.vstack([synth.standardise(synth.make_source("laplace", synth.rng_for(3, 0), T)),
                   synth.standardise(synth.make_source("uniform", synth.rng_for(3, 1), T))])
    X = (np.array([[1.0, 0.6], [-0.4, 1.3]]) @ S).astype(np.float32)
    Xw, V, mean = oracle.whiten(X)
    f = lambda t: float(oracle.upsilon(oracle.kurtosis_alpha(np.cos(t) * Xw[0] + np.sin(t) * Xw[1])))
    th = np.linspace(0, math.pi, 20_000, endpoint=False)
    vals = oracle.upsilon(oracle.kurtosis_alpha(np.outer(np.cos(th), Xw[0]) + np.outer(np.sin(th), Xw[1])))
    t0 = th[int(np.argmax(vals))]
    lo, hi = t0 - 2e-4, t0 + 2e-4
    g = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        a, b = hi - g * (hi - lo), lo + g * (hi - lo)
        if f(a) > f(b):
            hi = b
        else:
            lo = a
    tb = (lo + hi) / 2
    W = np.array([[math.cos(tb), math.sin(tb)], [-math.sin(tb), math.cos(tb)]])
    ang = np.linspace(0, math.pi, 16, endpoint=False)
    C = np.zeros((2, 16, 2))
    C[0] = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    c = oracle.certify_picks(Xw, W, C, K=500, eps=1e-13, components=[0])[0]
    assert c.pick_cos >= 1 - 1e-10 and c.margin >= -1e-9
    assert c.ups_pick == pytest.approx(f(tb), rel=1e-9)
    Wbad = np.array([[math.cos(tb + 0.3), math.sin(tb + 0.3)], [0.0, 0.0]])
    bad = oracle.certify_picks(Xw, Wbad, C, K=500, eps=1e-13, components=[0])[0]
    # refined, the bad pick either moves away (not a fixed point) or lands on a worse optimum
    assert bad.pick_cos < 1 - 1e-5 or bad.margin < -1e-6


def test_algorithm1_full_init_reaches_the_same_components(small_oracle):
    """Algorithm 1 from N-dimensional random initial vectors (projected by FastICA itself) finds
    the same ordered components as Algorithm 2 on the N=8 mixture (each non-Gaussian optimum is
    reached by many of the 64 restarts either way)."""
    w, B0, res, Xw, V, mean = small_oracle
    r1 = oracle.ordering_ica_original(Xw, w.M, 60, 1e-10, B0, full_init=True)
    cos = np.abs(np.sum(r1.W * res.W, axis=1))
    assert np.all(cos[:7] >= 1 - 1e-8), cos
    assert np.allclose(r1.alpha[:7], res.alpha[:7], rtol=1e-8)


def test_package_fluctuation_matches_the_oracle():
    from paper_2408_17118_gb300 import ica

    rng = np.random.default_rng(4)
    Ws = [rng.standard_normal((6, 9)) for _ in range(4)]
    assert np.allclose(ica.fluctuation(Ws), oracle.fluctuation(Ws), atol=1e-15)
    a = np.eye(3)
    assert np.allclose(ica.fluctuation([a, -a, 2 * a]), 0.0)
