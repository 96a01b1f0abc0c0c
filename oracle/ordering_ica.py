"""FP64 CPU oracle of the ordering ICA (Matsuda & Yamaguchi, arXiv 2408.17118).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct reference that the
CUDA path is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference legs may import it; the library in ``paper_2408_17118_gb300`` never
does, and this package imports nothing from the library. All arithmetic is float64 numpy;
library primitives (matrix product, symmetric eigendecomposition) serve as single steps.

Every function follows a passage of the paper, cited by section, equation or algorithm. The
paper writes samples as M and restarts as L; this file uses T for samples and M (or L inside
the algorithm functions) for restarts, matching the library's argument names.

Readings where the paper is silent or self-contradictory:

* convergence: a run has converged when min(||w - w_prev||, ||w + w_prev||) <= eps. The
  printed test in Algorithm 1 ("||w+w_prev|| > eps or ||w-w_prev|| > eps") can never fail for
  unit vectors, and Algorithm 2 prints the same test as the removal condition.
* restarts still unconverged after K iterations stay candidates (Algorithm 1 returns w after K
  iterations; Algorithm 2 would otherwise drop them).
* the matrix update is B <- (Z o Z o Z) X~^T / T - 3B (the form printed in Algorithm 2; the
  display in Section 3.1 writes the transposed product).
* whitening: centre each row, C = Xc Xc^T / T, V = C^(-1/2) (symmetric, ZCA), Xw = V Xc.
* ties in argmax go to the lowest restart index; the sign of each output row is made canonical
  (largest-magnitude entry positive, first such entry on ties).
* initial restarts: i.i.d. N(0,1) entries from Philox4x32-10 and Box-Muller (see
  ``philox4x32_10`` and ``restart_normals``), or an explicit B0 passed in.
* Upsilon(alpha) = +inf when alpha <= -2 (the log argument leaves its domain there).
* the deflation basis keeps the first n rows of F (Eq. 7) and is refused only when
  F~ F~^T has an eigenvalue <= 1e-14 (eigenvalues of 1e-11 occur in generic data where the
  found components and the kept coordinates have about equal dimension).

Parity status: every function here is pinned by tests in ``tests/test_oracle_pins.py``
(closed forms, invariants, brute force on N=2, known-answer vectors); none is unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

F64 = np.float64


# --------------------------------------------------------------------------------------------
# Objective (Section 2.2, Eq. 1 and Eq. 2)
# --------------------------------------------------------------------------------------------

def kurtosis_alpha(y: np.ndarray) -> np.ndarray:
    """Eq. 2: alpha = sum_m y_m^4 / T - 3 along the last axis (y has unit variance)."""
    y = np.asarray(y, dtype=F64)
    y2 = y * y
    return np.mean(y2 * y2, axis=-1) - 3.0


def upsilon(alpha) -> np.ndarray:
    """Eq. 1: Upsilon(alpha) = alpha - 2 log(alpha/2 + 1); +inf where alpha <= -2."""
    a = np.asarray(alpha, dtype=F64)
    out = np.full(a.shape, np.inf)
    ok = a > -2.0
    out[ok] = a[ok] - 2.0 * np.log(a[ok] / 2.0 + 1.0)
    return out if out.shape else float(out)


def gaussianity_threshold(N: int, i: int, T: int) -> float:
    """Eq. 3 / Algorithm 1 and 2 stopping rule: stop at component i (1-based) when
    Upsilon(alpha_i) < 2 (N - i + 2)(N - i + 1) / T."""
    return 2.0 * (N - i + 2) * (N - i + 1) / T


# --------------------------------------------------------------------------------------------
# Whitening (Section 2.2: X is whitened in advance; Theorem 1 assumes zero-mean rows)
# --------------------------------------------------------------------------------------------

def whiten(X: np.ndarray):
    """Centre the rows, then apply V = C^(-1/2) with C = Xc Xc^T / T (symmetric whitening).

    Returns (Xw, V, mean) with Xw = V (X - mean) so that Xw Xw^T / T = I.
    """
    X = np.asarray(X, dtype=F64)
    T = X.shape[1]
    mean = X.mean(axis=1)
    Xc = X - mean[:, None]
    C = (Xc @ Xc.T) / T
    lam, E = np.linalg.eigh(C)
    V = (E * (1.0 / np.sqrt(lam))) @ E.T
    return V @ Xc, V, mean


# --------------------------------------------------------------------------------------------
# Algorithm 1: original ordering ICA, one FastICA run per initialisation
# --------------------------------------------------------------------------------------------

def converged(w: np.ndarray, w_prev: np.ndarray, eps: float) -> bool:
    """Sign-tolerant convergence: min(||w - w_prev||, ||w + w_prev||) <= eps."""
    return min(np.linalg.norm(w - w_prev), np.linalg.norm(w + w_prev)) <= eps


def fastica_run(w: np.ndarray, X: np.ndarray, E: np.ndarray, K: int, eps: float):
    """Algorithm 1, function FastICA: kurtosis fixed point with projection deflation.

    w <- w - E w; normalise; repeat { y = w^T X; w <- X (y o y o y)^T / T - 3 w; w <- w - E w;
    normalise } while fewer than K iterations and not converged.
    Returns (w, y, iterations, converged).
    """
    T = X.shape[1]
    w = np.asarray(w, dtype=F64).copy()
    w = w - E @ w
    w = w / math.sqrt(w @ w)
    t = 0
    while True:
        w_prev = w
        y = w @ X
        w = X @ (y * y * y) / T - 3.0 * w
        w = w - E @ w
        w = w / math.sqrt(w @ w)
        t += 1
        done = converged(w, w_prev, eps)
        if not (t < K and not done):
            break
    return w, w @ X, t, done


@dataclass
class FitResult:
    W: np.ndarray            # n_found x N, rows orthonormal, ordered by descending Upsilon
    alpha: np.ndarray        # n_found excess kurtoses of the extracted components
    winners: list            # restart index chosen for each component
    iterations: list         # per component: iterations used by each restart (array of M)
    n_converged: list        # per component: restarts that met the tolerance
    upsilon_all: list        # per component: Upsilon of every restart's final vector
    G: list                  # per component: reduction basis used (Algorithm 2 only)


def canonical_sign(w: np.ndarray) -> np.ndarray:
    """Flip w so that its largest-magnitude entry (first on ties) is positive."""
    k = int(np.argmax(np.abs(w)))
    return w if w[k] >= 0 else -w


def ordering_ica_original(Xw: np.ndarray, L: int, K: int, eps: float, B0: np.ndarray,
                          n_components: int | None = None, gauss_test: bool = False,
                          full_init: bool = False) -> FitResult:
    """Algorithm 1 on whitened Xw with explicit initial restarts.

    B0[i] holds the initialisations for component i. For comparison with Algorithm 2 the
    initial vector of restart l is w = G^T b0 where b0 = B0[i, l, :N-i] and G is the reduction
    basis of Section 3.3 (at i = 0, G = I); that w lies in the complement of the found
    components, so the projection in FastICA leaves it unchanged. With full_init the initial
    vector is the N-dimensional b0 = B0[i, l, :N] itself (Algorithm 1's random w), which the
    FastICA run first projects onto the complement of the found components.
    """
    Xw = np.asarray(Xw, dtype=F64)
    N, T = Xw.shape
    n_comp = N if n_components is None else n_components
    W = np.zeros((0, N))
    res = FitResult(W, np.zeros(0), [], [], [], [], [])
    alphas = []
    for i in range(1, n_comp + 1):
        n = N - i + 1
        E = W.T @ W if i > 1 else np.zeros((N, N))
        G = deflation_basis(W, N) if i > 1 else np.eye(N)
        ws, alpha, its = [], np.empty(L), np.empty(L, dtype=np.int64)
        n_conv = 0
        for l in range(L):
            w0 = np.asarray(B0[i - 1, l, :N], dtype=F64) if full_init else G.T @ np.asarray(B0[i - 1, l, :n], dtype=F64)
            w, y, t, done = fastica_run(w0, Xw, E, K, eps)
            ws.append(w)
            alpha[l] = kurtosis_alpha(y)
            its[l] = t
            n_conv += int(done)
        ups = upsilon(alpha)
        p = int(np.argmax(ups))
        if gauss_test and ups[p] < gaussianity_threshold(N, i, T):
            break
        W = np.vstack([W, canonical_sign(ws[p])])
        alphas.append(alpha[p])
        res.winners.append(p)
        res.iterations.append(its)
        res.n_converged.append(n_conv)
        res.upsilon_all.append(ups)
    res.W = W
    res.alpha = np.asarray(alphas)
    return res


# --------------------------------------------------------------------------------------------
# Section 3.3: reduction of signals under the orthonormality constraints
# --------------------------------------------------------------------------------------------

def deflation_basis(W: np.ndarray, N: int) -> np.ndarray:
    """Eq. 6 and Eq. 7: F = I_N - W^T W; F~ = first N-i+1 rows of F;
    G = (F~ F~^T)^(-1/2) F~ (rows orthonormal, orthogonal to the rows of W)."""
    W = np.asarray(W, dtype=F64)
    k = W.shape[0]
    n = N - k
    F = np.eye(N) - W.T @ W
    Ft = F[:n, :]
    S = Ft @ Ft.T
    lam, U = np.linalg.eigh(S)
    # Eq. 7 keeps the first n rows of F; F~ F~^T is then nearly singular when the found rows nearly
    # contain a unit vector of the first n coordinates (eigenvalues of 1e-11 occur near n = k = N/2
    # in generic data). FP64 eigenpairs keep G accurate to about 1 % in length and 1e-9 in
    # direction down to 1e-14; below that the basis is refused.
    if lam.min() <= 1e-14:
        raise np.linalg.LinAlgError(f"F~ F~^T is singular (lambda_min = {lam.min():.3e})")
    S_inv_half = (U * (1.0 / np.sqrt(lam))) @ U.T
    return S_inv_half @ Ft


def reduce_signals(G: np.ndarray, Xw: np.ndarray) -> np.ndarray:
    """Eq. 8: X~ = G X."""
    return np.asarray(G, dtype=F64) @ np.asarray(Xw, dtype=F64)


# --------------------------------------------------------------------------------------------
# Section 3.1 / Algorithm 2: matrix form of all runs at once
# --------------------------------------------------------------------------------------------

def matrix_update(B: np.ndarray, Xt: np.ndarray) -> np.ndarray:
    """Eq. 4 and the update of Algorithm 2: Z = B X~; B' = (Z o Z o Z) X~^T / T - 3 B.

    B is (restarts x n), X~ is (n x T). Returns the un-normalised update.
    """
    B = np.asarray(B, dtype=F64)
    Xt = np.asarray(Xt, dtype=F64)
    T = Xt.shape[1]
    Z = B @ Xt
    return (Z * Z * Z) @ Xt.T / T - 3.0 * B


def normalise_rows(B: np.ndarray) -> np.ndarray:
    """Algorithm 2: every row b <- b / sqrt(b b^T)."""
    B = np.asarray(B, dtype=F64)
    return B / np.sqrt(np.sum(B * B, axis=1, keepdims=True))


def step_distance(B: np.ndarray, Bprev: np.ndarray) -> np.ndarray:
    """Per row min(||b - b_prev||, ||b + b_prev||) (the convergence reading above)."""
    dm = np.sqrt(np.sum((B - Bprev) ** 2, axis=1))
    dp = np.sqrt(np.sum((B + Bprev) ** 2, axis=1))
    return np.minimum(dm, dp)


@dataclass
class ComponentTrace:
    G: np.ndarray
    Xt_shape: tuple
    B_final: np.ndarray      # M x n final restart rows (converged and not)
    iterations: np.ndarray   # M: iterations each restart ran
    converged: np.ndarray    # M bools
    alpha: np.ndarray        # M
    upsilon: np.ndarray      # M
    winner: int
    step_norms: list         # per iteration: (active restart ids, distances)
    alpha_traj: list         # per iteration: (active restart ids, alpha of the pre-update rows)


def fast_ordering_component(Xt: np.ndarray, B0: np.ndarray, K: int, eps: float,
                            record: bool = False):
    """Inner part of Algorithm 2 for one component on reduced data X~ (n x T).

    B0 (M x n) are the raw initial rows; they are normalised first. Rows whose step distance
    falls to eps or below move to B_conv and are never updated again (Section 3.2). Returns the
    final rows of every restart, the iterations each ran, which converged, and optionally the
    per-iteration step norms and pre-update kurtoses of the active rows.
    """
    Xt = np.asarray(Xt, dtype=F64)
    B = normalise_rows(B0)
    M = B.shape[0]
    active = np.arange(M)
    its = np.zeros(M, dtype=np.int64)
    conv = np.zeros(M, dtype=bool)
    steps, atraj = [], []
    t = 0
    while True:
        Bprev = B[active]
        if record:
            atraj.append((active.copy(), kurtosis_alpha(Bprev @ Xt)))
        Bnew = normalise_rows(matrix_update(Bprev, Xt))
        d = step_distance(Bnew, Bprev)
        B[active] = Bnew
        its[active] += 1
        done = d <= eps
        if record:
            steps.append((active.copy(), d))
        conv[active[done]] = True
        active = active[~done]
        t += 1
        if not (t < K and active.size > 0):
            break
    return B, its, conv, steps, atraj


def fast_ordering_ica(Xw: np.ndarray, L: int, K: int, eps: float, B0: np.ndarray,
                      n_components: int | None = None, gauss_test: bool = False,
                      record: bool = False) -> FitResult:
    """Algorithm 2 (Fast Ordering ICA) on whitened Xw, with explicit initial restarts B0.

    For each component i: reduce X (Eq. 6-8), iterate all L restarts in matrix form with
    removal of converged rows, take alpha of every candidate (converged rows plus rows still
    running after K iterations), pick p = argmax Upsilon (lowest index on ties), optionally
    stop by the Gaussianity test, and append w = b_p G.
    """
    Xw = np.asarray(Xw, dtype=F64)
    N, T = Xw.shape
    n_comp = N if n_components is None else n_components
    W = np.zeros((0, N))
    res = FitResult(W, np.zeros(0), [], [], [], [], [])
    res.traces = []
    alphas = []
    for i in range(1, n_comp + 1):
        n = N - i + 1
        if i > 1:
            G = deflation_basis(W, N)
            Xt = reduce_signals(G, Xw)
        else:
            G = np.eye(N)
            Xt = Xw
        B, its, conv, steps, atraj = fast_ordering_component(Xt, B0[i - 1, :, :n], K, eps, record)
        alpha = kurtosis_alpha(B @ Xt)
        ups = upsilon(alpha)
        p = int(np.argmax(ups))
        if gauss_test and ups[p] < gaussianity_threshold(N, i, T):
            break
        w = B[p] @ G
        W = np.vstack([W, canonical_sign(w)])
        alphas.append(alpha[p])
        res.winners.append(p)
        res.iterations.append(its)
        res.n_converged.append(int(conv.sum()))
        res.upsilon_all.append(ups)
        res.G.append(G)
        res.traces.append(ComponentTrace(G, Xt.shape, B, its, conv, alpha, ups, p, steps, atraj))
    res.W = W
    res.alpha = np.asarray(alphas)
    return res


def order_fit(X: np.ndarray, M: int, n_components: int, iters: int, tol: float, B0: np.ndarray,
              gauss_test: bool = False, algorithm: int = 2, record: bool = False, full_init: bool = False):
    """Whiten raw X, then run Algorithm 2 (default) or Algorithm 1 (full_init: N-dimensional
    initial vectors). Returns (result, Xw, V, mean)."""
    Xw, V, mean = whiten(X)
    fit = fast_ordering_ica if algorithm == 2 else ordering_ica_original
    kw = {"record": record} if algorithm == 2 else {"full_init": full_init}
    return fit(Xw, M, iters, tol, B0, n_components=n_components, gauss_test=gauss_test, **kw), Xw, V, mean


# --------------------------------------------------------------------------------------------
# Certification of a fit's picks in FP64 (for fits too large for the full oracle)
# --------------------------------------------------------------------------------------------

@dataclass
class PickCheck:
    i: int                   # component (0-based)
    ups_pick: float          # Upsilon (Eq. 1) of the refined pick
    ups_best_other: float    # largest Upsilon among refined candidates distinct from the pick (-inf if none)
    margin: float            # ups_pick - ups_best_other
    pick_cos: float          # |cos| between the submitted pick and its FP64 refinement
    alpha_pick: float        # Eq. 2 kurtosis of the refined pick
    candidates: int          # non-zero candidate rows checked


def certify_picks(Xw: np.ndarray, W: np.ndarray, cands: np.ndarray, K: int = 50, eps: float = 1e-10,
                  components=None, distinct: float = 1.0 - 1e-3) -> list:
    """FP64 re-check of the global pick of Algorithm 2 for each listed component i.

    W (n x N) is a fit's output, row i its pick w_i; cands (n x k x N) holds, per component,
    candidate directions in the whitened space from which that fit picked (zero rows unused).
    With E = W[:i]^T W[:i] (the components found before, taken from the fit itself), the pick
    and every candidate are refined by the FastICA run of Algorithm 1 (projected kurtosis fixed
    point, FP64, to eps or K iterations); their kurtoses (Eq. 2) and objectives (Eq. 1) are then
    compared as Algorithm 2's argmax compares them. Candidates within |cos| >= `distinct` of the
    refined pick are the same direction and are not compared. A correct pick is a fixed point
    (pick_cos ~ 1) with margin >= 0 up to the precision the fit ran in.
    """
    Xw = np.asarray(Xw, dtype=F64)
    W = np.asarray(W, dtype=F64)
    cands = np.asarray(cands, dtype=F64)
    N = Xw.shape[0]
    out = []
    for i in (range(W.shape[0]) if components is None else components):
        E = W[:i].T @ W[:i] if i > 0 else np.zeros((N, N))
        wp, yp, _, _ = fastica_run(W[i], Xw, E, K, eps)
        a_p = float(kurtosis_alpha(yp))
        u_p = float(upsilon(a_p))
        best, used = -np.inf, 0
        for c in cands[i]:
            if not np.any(c):
                continue
            used += 1
            wc, yc, _, _ = fastica_run(c, Xw, E, K, eps)
            if abs(wc @ wp) >= distinct:
                continue
            best = max(best, float(upsilon(kurtosis_alpha(yc))))
        out.append(PickCheck(i, u_p, best, u_p - best, float(abs(wp @ W[i])), a_p, used))
    return out


# --------------------------------------------------------------------------------------------
# Random initial restarts: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) + Box-Muller
# --------------------------------------------------------------------------------------------

_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_U32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on one 128-bit counter and a 64-bit key (pure Python ints).

    Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (32x32 -> 64-bit products);
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key advances by the Weyl constants
    (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (int(v) & _U32 for v in ctr)
    k0, k1 = (int(v) & _U32 for v in key)
    for r in range(10):
        if r:
            k0 = (k0 + _PHILOX_W0) & _U32
            k1 = (k1 + _PHILOX_W1) & _U32
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & _U32
        hi1, lo1 = p1 >> 32, p1 & _U32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def philox4x32_10_np(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 over uint32 numpy arrays (same definition as above)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & _U32)
    k1 = np.uint64(int(k1) & _U32)
    m32 = np.uint64(_U32)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(_PHILOX_W0)) & m32
            k1 = (k1 + np.uint64(_PHILOX_W1)) & m32
        p0 = np.uint64(_PHILOX_M0) * c0
        p1 = np.uint64(_PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & m32
        hi1, lo1 = p1 >> np.uint64(32), p1 & m32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform52(a, b):
    """Two 32-bit words -> a double strictly inside (0, 1): u = (k + 0.5) / 2^52 with the
    52-bit integer k = (a >> 6) * 2^26 + (b >> 6); k + 0.5 is exact in a double."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    k = (a >> np.uint64(6)) * np.uint64(67108864) + (b >> np.uint64(6))
    return (k.astype(F64) + 0.5) / 4503599627370496.0


def restart_normals(seed: int, component: int, M: int, n: int) -> np.ndarray:
    """Initial restart matrix (M x n) of i.i.d. N(0,1) entries, not yet normalised.

    Entry (l, 2j) and (l, 2j+1) come from one Philox4x32-10 call with counter (j, l, component,
    0) and key (seed low 32 bits, seed high 32 bits): u1 from words (0, 1), u2 from words
    (2, 3), then Box-Muller r = sqrt(-2 ln u1), theta = 2 pi u2, (r cos theta, r sin theta).
    """
    npair = (n + 1) // 2
    j, l = np.meshgrid(np.arange(npair, dtype=np.uint64), np.arange(M, dtype=np.uint64))
    c2 = np.full(j.shape, component, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10_np(j, l, c2, np.zeros_like(j), seed & _U32, (seed >> 32) & _U32)
    u1 = uniform52(x0, x1)
    u2 = uniform52(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * math.pi * u2
    out = np.empty((M, 2 * npair))
    out[:, 0::2] = r * np.cos(th)
    out[:, 1::2] = r * np.sin(th)
    return out[:, :n]


def seeded_B0(seed: int, M: int, N: int, n_components: int) -> np.ndarray:
    """B0 array (n_components x M x N) of the seeded initial restarts; row l of component i
    uses its first N-i entries."""
    B0 = np.zeros((n_components, M, N))
    for i in range(n_components):
        B0[i, :, : N - i] = restart_normals(seed, i, M, N - i)
    return B0


# --------------------------------------------------------------------------------------------
# Evaluation helpers (Section 4)
# --------------------------------------------------------------------------------------------

def amari_index(P: np.ndarray) -> float:
    """Amari performance index of P = W V A, scaled to [0, 1]; 0 iff P is a scaled permutation."""
    P = np.abs(np.asarray(P, dtype=F64))
    N = P.shape[0]
    r = np.sum(P / P.max(axis=1, keepdims=True), axis=1) - 1.0
    c = np.sum(P / P.max(axis=0, keepdims=True), axis=0) - 1.0
    return float((r.sum() + c.sum()) / (2.0 * N * (N - 1)))


def fluctuation(Ws: list) -> np.ndarray:
    """Section 4.3: mean over ordered run pairs (t != u) of 1 - |cos(w_i^t, w_i^u)| per component."""
    R = len(Ws)
    n = min(w.shape[0] for w in Ws)
    acc = np.zeros(n)
    for t in range(R):
        for u in range(R):
            if t == u:
                continue
            a, b = Ws[t][:n], Ws[u][:n]
            cos = np.sum(a * b, axis=1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
            acc += 1.0 - np.abs(cos)
    return acc / (R * (R - 1))
