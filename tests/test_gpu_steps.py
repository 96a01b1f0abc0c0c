"""Per-step parity of the CUDA path against the FP64 oracle, through the C ABI.

Sizes span several tiles and ragged tails (restart tiles of 64/128 rows, sample chunks of 64/128,
reduced dimension padded to 16). Tolerances are derived from the arithmetic of each step:

* FP32 products: |error| <= 1e-4 * S + 1e-6, with S = sum_t |z_t^3 x_kt| / T the magnitude
  scale of the element (FP32 accumulation, random-walk growth with wide margin).
* BF16 tensor-core update: the operands are rounded to BF16 on both sides (the oracle takes the
  same rounded inputs); the GPU additionally rounds z^3 to BF16 (relative error <= 2^-9) and
  accumulates in FP32, so |error| <= 2^-8 * S + 1e-6 (a factor 2 of slack on the rounding
  bound).
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


def rup(v, m):
    return (v + m - 1) // m * m


def bf16(a: np.ndarray) -> np.ndarray:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def padded_xt(X: np.ndarray, n_pad: int, dtype) -> torch.Tensor:
    n, T = X.shape
    ld = rup(T, 8)
    out = torch.zeros((n_pad, ld), dtype=dtype)
    out[:n, :T] = torch.from_numpy(X.astype(np.float32)).to(dtype)
    return out.cuda()


def random_rows(M, n, n_pad, seed):
    B = oracle.normalise_rows(np.random.default_rng(seed).standard_normal((M, n))).astype(np.float32)
    Bp = np.zeros((M, n_pad), dtype=np.float32)
    Bp[:, :n] = B
    return Bp


# ------------------------------------------------------------------------------ initial restarts
@pytest.mark.parametrize("seed,comp,M,n", [(0, 0, 64, 8), (12345678901, 3, 130, 37), (2 ** 63 + 5, 7, 7, 256),
                                           (1, 0, 1, 1), (99, 200, 300, 255)])
def test_init_restarts(ctx, seed, comp, M, n):
    from paper_2408_17118_gb300 import ica

    ldb = rup(n, 16)
    B = ica.ica_init_restarts(ctx, seed, comp, M, n, ldb).cpu().numpy()
    ref = oracle.normalise_rows(oracle.restart_normals(seed, comp, M, n))
    assert np.abs(B[:, :n] - ref).max() < 2e-7
    assert np.all(B[:, n:] == 0)


# ------------------------------------------------------------------------------ deflation basis
@pytest.mark.parametrize("N,k", [(8, 1), (8, 4), (8, 7), (33, 10), (33, 20), (64, 32), (64, 63), (130, 65),
                                 (256, 1), (256, 128), (256, 200)])
def test_deflation_basis(ctx, N, k):
    from paper_2408_17118_gb300 import ica

    Q, _ = np.linalg.qr(np.random.default_rng(N * 7 + k).standard_normal((N, N)))
    W = np.ascontiguousarray(Q[:k])
    G = ica.ica_deflation_basis(ctx, torch.from_numpy(W).cuda(), N).cpu().numpy()
    ref = oracle.deflation_basis(W, N)
    assert G.shape == ref.shape
    # both sides evaluate (F~F~^T)^(-1/2) F~ in FP64; their rounding errors are amplified by
    # 1 / lambda_min(F~F~^T), which reaches ~1e5 for N = 256
    Ft = (np.eye(N) - W.T @ W)[: N - k]
    lam_min = np.linalg.eigvalsh(Ft @ Ft.T).min()
    tol = max(1e-12, 100 * np.finfo(np.float64).eps / lam_min)
    assert np.abs(G - ref).max() < tol, (np.abs(G - ref).max(), tol)
    assert np.abs(G @ G.T - np.eye(N - k)).max() < tol
    assert np.abs(W @ G.T).max() < tol


def _e4m3_scale_exponent(m):
    """Largest e with m 2^e <= 448 (m > 0), exactly (powers of two scale exactly)."""
    if not m > 0:
        return 0
    e = int(np.floor(np.log2(448.0 / m)))
    while np.ldexp(m, e) > 448.0:
        e -= 1
    while np.ldexp(m, e + 1) <= 448.0:
        e += 1
    return e


@pytest.mark.parametrize("n,T", [(5, 1000), (40, 4_099), (130, 3_000), (256, 2_053)])
def test_quantize_e4m3(ctx, n, T):
    """The E4M3 operand of the FP8 iterations: every byte equals torch's float32 -> float8_e4m3fn
    conversion (round to nearest even) of x 2^e_k, e_k the largest exponent with
    max |x_k| 2^e_k <= 448; padding rows and samples zero; the scale table as documented. Rows
    of very different magnitudes (2^-20 .. 2^12) and an all-zero row."""
    from paper_2408_17118_gb300 import ica

    rng = np.random.default_rng(n + T)
    ld = (T + 7) // 8 * 8
    X = np.zeros((n, ld), dtype=np.float32)
    X[:, :T] = rng.standard_t(4, size=(n, T)).astype(np.float32)
    X[:, :T] *= np.ldexp(1.0, (np.arange(n) % 33) - 20)[:, None].astype(np.float32)
    X[n // 2, :] = 0.0
    X8, sc = ica.ica_quantize_e4m3(ctx, torch.from_numpy(X).cuda(), n, T)
    X8, sc = X8.cpu().numpy(), sc.cpu().numpy()
    n8 = (n + 31) // 32 * 32
    assert X8.shape == (n8, (T + 15) // 16 * 16)
    e = np.array([_e4m3_scale_exponent(float(np.abs(X[k, :T]).max())) for k in range(n)])
    scaled = (X[:, :T].astype(np.float64) * np.ldexp(1.0, e)[:, None]).astype(np.float32)
    ref = torch.from_numpy(scaled).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(X8[:n, :T], ref), np.argwhere(X8[:n, :T] != ref)[:5]
    assert not X8[n:].any() and not X8[:, T:].any()
    c = 8 + e.min()
    assert np.array_equal(sc[:n], np.ldexp(1.0, e).astype(np.float32))
    assert np.array_equal(sc[n8:n8 + n], np.ldexp(1.0, c - e).astype(np.float32))
    assert np.array_equal(sc[2 * n8:2 * n8 + n], np.ldexp(1.0, -e).astype(np.float32))
    assert sc[3 * n8] == np.float32(np.ldexp(1.0, -c))


@pytest.mark.parametrize("delta", [1e-4, 1e-5])
def test_deflation_basis_near_singular(ctx, delta):
    """Found rows that nearly contain e_0 (here F~F~^T has an eigenvalue of about 0.007 delta^2:
    7e-11 and 7e-13, between the refusal threshold 1e-14 and 1e-10): the GPU basis is accepted
    and matches the oracle's within the FP64 eigenpair accuracy at that eigenvalue."""
    from paper_2408_17118_gb300 import ica

    N, k = 64, 30
    rng = np.random.default_rng(9)
    w0 = np.zeros(N)
    w0[0], w0[N - 1] = 1.0, delta
    w0 /= np.linalg.norm(w0)
    rest = rng.standard_normal((k - 1, N))
    rest -= np.outer(rest @ w0, w0)
    q, _ = np.linalg.qr(rest.T)
    W = np.ascontiguousarray(np.vstack([w0, q.T[: k - 1]]))
    G = ica.ica_deflation_basis(ctx, torch.from_numpy(W).cuda(), N).cpu().numpy()
    ref = oracle.deflation_basis(W, N)
    Ft = (np.eye(N) - W.T @ W)[: N - k]
    lam_min = np.linalg.eigvalsh(Ft @ Ft.T).min()
    assert 1e-14 < lam_min < 1e-10
    tol = 100 * np.finfo(np.float64).eps / lam_min
    assert np.abs(G @ G.T - np.eye(N - k)).max() < tol
    assert np.abs(W @ G.T).max() < 100 * np.finfo(np.float64).eps / np.sqrt(lam_min)
    assert np.abs(G - ref).max() < tol


@pytest.mark.parametrize("N,k", [(64, 24), (64, 40), (40, 20)])
def test_deflation_basis_repeated_eigenvalues(ctx, N, k):
    # W = Q W0 with W0 rows cos(th) e_a + sin(th) e_b (a among the first n coordinates, b among
    # the last k) and th from two values: the Gram matrix of the Jacobi solve has two clusters of
    # exactly repeated eigenvalues and is not diagonal; G = (F~F~^T)^(-1/2) F~ is still unique
    from paper_2408_17118_gb300 import ica

    n = N - k
    rng = np.random.default_rng(N + 3 * k)
    W0 = np.zeros((k, N))
    for i in range(k):
        th = 0.4 if i % 2 == 0 else 1.1
        W0[i, i % n] = np.cos(th) if i < n else 0.0
        W0[i, n + i] = np.sin(th) if i < n else 1.0
    W0 /= np.linalg.norm(W0, axis=1, keepdims=True)
    # rows with the same first coordinate must stay orthogonal: use distinct first coordinates
    assert np.abs(W0 @ W0.T - np.eye(k)).max() < 1e-12
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    W = np.ascontiguousarray(Q @ W0)
    G = ica.ica_deflation_basis(ctx, torch.from_numpy(W).cuda(), N).cpu().numpy()
    ref = oracle.deflation_basis(W, N)
    Ft = (np.eye(N) - W.T @ W)[:n]
    tol = max(1e-12, 100 * np.finfo(np.float64).eps / np.linalg.eigvalsh(Ft @ Ft.T).min())
    assert np.abs(G - ref).max() < tol, (np.abs(G - ref).max(), tol)
    assert np.abs(G @ G.T - np.eye(n)).max() < tol
    assert np.abs(W @ G.T).max() < tol


def test_whiten_repeated_eigenvalues(ctx):
    # X = A S with S S^T / T = I exactly and A = Q diag(d), d with repeated values: the covariance
    # A A^T has clusters of exactly repeated eigenvalues; V = C^(-1/2) is unique
    from paper_2408_17118_gb300 import ica

    N, T = 48, 6000
    rng = np.random.default_rng(11)
    S, _ = np.linalg.qr(rng.standard_normal((T, N)))
    S = S.T * np.sqrt(T)
    S -= S.mean(axis=1, keepdims=True)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    d = np.repeat([0.5, 2.0, 7.0], N // 3)
    X = (Q * d) @ S + 3.0
    Xw, V, mean = ica.ica_whiten(ctx, torch.from_numpy(X.astype(np.float32)).cuda())
    Xw_o, V_o, mean_o = oracle.whiten(X.astype(np.float32).astype(np.float64))
    assert np.abs(V.cpu().numpy() - V_o).max() < 1e-8 * np.abs(V_o).max()


def test_deflation_basis_identity(ctx):
    from paper_2408_17118_gb300 import ica

    G = ica.ica_deflation_basis(ctx, torch.zeros((0, 12), dtype=torch.float64).cuda(), 12).cpu().numpy()
    assert np.array_equal(G, np.eye(12))


# ------------------------------------------------------------------------------ whitening
@pytest.mark.parametrize("kind", ["small", "eeg64", "n256"])
def test_whiten(ctx, kind):
    from paper_2408_17118_gb300 import ica

    if kind == "small":
        X = synth.small_mixture(0).X
    elif kind == "eeg64":
        X = synth.eeg_like(64, 20_000, 8, seed=1).X
    else:
        X = synth.eeg_like(256, 6000, 8, seed=2).X
    Xw, V, mean = ica.ica_whiten(ctx, torch.from_numpy(X).cuda())
    Xw_o, V_o, mean_o = oracle.whiten(X)
    assert np.abs(mean.cpu().numpy() - mean_o).max() < 1e-12 * (1 + np.abs(mean_o).max())
    assert np.abs(V.cpu().numpy() - V_o).max() < 1e-8 * np.abs(V_o).max()
    # FP32 apply: N-term FP32 dot products of O(1) values
    assert np.abs(Xw.cpu().numpy() - Xw_o).max() < 5e-5 * max(1.0, np.abs(Xw_o).max())


# ------------------------------------------------------------------------------ reduction
@pytest.mark.parametrize("N,k,T", [(8, 0, 1000), (20, 7, 4099), (64, 30, 20_000), (130, 3, 3000)])
def test_reduce(ctx, N, k, T):
    from paper_2408_17118_gb300 import ica

    Xw = synth.small_random(N, T, seed=N + k).astype(np.float32)
    if k:
        Q, _ = np.linalg.qr(np.random.default_rng(k).standard_normal((N, N)))
        G = oracle.deflation_basis(Q[:k], N)
    else:
        G = np.eye(N)
    n = N - k
    Xt32, Xt16 = ica.ica_reduce(ctx, torch.from_numpy(np.ascontiguousarray(G)).cuda(), torch.from_numpy(Xw).cuda())
    Xt32 = Xt32.cpu()
    Xt16 = Xt16.cpu()
    ref = G @ Xw.astype(np.float64)
    got = Xt32.numpy()[:n, :T]
    assert np.abs(got - ref).max() < 2e-6 * N * max(1.0, np.abs(Xw).max())
    assert torch.equal(Xt16[:, :T], Xt32[:, :T].to(torch.bfloat16))  # BF16 copy = rounding of the FP32 result
    assert torch.all(Xt32[n:, :T] == 0) and torch.all(Xt16[n:, :T].float() == 0)


# ------------------------------------------------------------------------------ fused update
STEP_SHAPES = [(1, 1, 64), (63, 5, 1000), (64, 16, 4097), (65, 17, 12345), (129, 37, 2000), (200, 64, 40_000),
               (300, 100, 5000), (128, 128, 8192), (130, 129, 3000), (257, 200, 6000), (100, 256, 10_000)]


def b_operand(B, n_pad):
    """The restart rows as the BF16 kernel feeds them to the tensor cores: two BF16 terms
    hi = bf16(b), lo = bf16(b - hi) (lo from shared memory for n_pad <= 64, from tensor memory
    above), both multiplied by the same BF16 X~ and accumulated in FP32."""
    B = np.asarray(B, dtype=np.float32)
    hi = bf16(B).astype(np.float32)
    lo = bf16((B - hi).astype(np.float32)).astype(np.float32)
    return hi.astype(np.float64) + lo.astype(np.float64)


def oracle_update(B, Xt, T, bf16_inputs, n_pad=None):
    Bq = b_operand(B, n_pad) if bf16_inputs else B.astype(np.float64)
    Xq = bf16(Xt) if bf16_inputs else Xt.astype(np.float64)
    Bq = Bq.astype(np.float64)
    Xq = Xq.astype(np.float64)
    Z = Bq @ Xq
    U = (Z ** 3) @ Xq.T / T - 3.0 * B.astype(np.float64)
    S = (np.abs(Z) ** 3) @ np.abs(Xq).T / T
    return U, S, Z


@pytest.mark.parametrize("M,n,T", STEP_SHAPES)
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fp_step(ctx, prec, M, n, T):
    from paper_2408_17118_gb300 import ica

    n_pad = rup(n, 16)
    Xt = synth.small_random(n, T, seed=M + n + T)
    B = random_rows(M, n, n_pad, seed=M * 31 + n)
    p = ica.ICA_FP32 if prec == "fp32" else ica.ICA_BF16
    xt = padded_xt(Xt, n_pad, torch.float32 if prec == "fp32" else torch.bfloat16)
    Bnew, mom = ica.ica_fp_step(ctx, p, torch.from_numpy(B).cuda(), n, xt, T)
    Bnew = Bnew.cpu().numpy()
    mom = mom.cpu().numpy()
    U, S, Z = oracle_update(B[:, :n], Xt, T, prec == "bf16", n_pad)
    tol = (1e-4 if prec == "fp32" else 2.0 ** -8) * S + 1e-6
    err = np.abs(Bnew[:, :n] - U)
    assert np.all(err <= tol), (err.max(), (err / tol).max())
    assert np.all(Bnew[:, n:] == 0)
    m2 = np.mean(Z ** 2, axis=1)
    m4 = np.mean(Z ** 4, axis=1)
    assert np.allclose(mom[:, 0], m2, rtol=2e-5, atol=1e-7)
    assert np.allclose(mom[:, 1], m4, rtol=2e-5, atol=1e-7)


@pytest.mark.parametrize("M,n,T", [(64, 8, 10_000), (300, 37, 4097), (129, 128, 20_000), (100, 200, 5000)])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_kurtosis(ctx, prec, M, n, T):
    from paper_2408_17118_gb300 import ica

    n_pad = rup(n, 16)
    Xt = synth.small_random(n, T, seed=n + T)  # includes binary rows (alpha close to -2)
    B = random_rows(M, n, n_pad, seed=n)
    # make some rows point exactly / almost exactly at single sources (binary, uniform, ...)
    for r in range(min(M, 2 * n)):
        j = r % n
        v = np.zeros(n_pad, dtype=np.float32)
        v[j] = 1.0
        if r >= n:
            v[(j + 1) % n] = 1e-3
            v /= np.linalg.norm(v)
        B[r] = v
    p = ica.ICA_FP32 if prec == "fp32" else ica.ICA_BF16
    xt = padded_xt(Xt, n_pad, torch.float32 if prec == "fp32" else torch.bfloat16)
    a, u = ica.ica_kurtosis(ctx, p, torch.from_numpy(B).cuda(), n, xt, T)
    a = a.cpu().numpy()
    u = u.cpu().numpy()
    Bq = b_operand(B[:, :n], n_pad) if prec == "bf16" else B[:, :n].astype(np.float64)
    Xq = bf16(Xt).astype(np.float64) if prec == "bf16" else Xt.astype(np.float64)
    Z = Bq @ Xq
    m2 = np.mean(Z ** 2, axis=1)
    ref_a2 = np.mean(Z ** 4, axis=1) / m2 ** 2 - 1.0  # alpha + 2 of the normalised row
    # alpha + 2 from FP32 sums of (z^2 - 1)^2: relative error ~1e-5 plus an absolute floor
    got_a2 = a + 2.0
    assert np.all(np.abs(got_a2 - ref_a2) <= 3e-5 * ref_a2 + 1e-8), np.abs(got_a2 - ref_a2).max()
    fin = ref_a2 > 1e-9
    ref_u = ref_a2[fin] - 2.0 - 2.0 * np.log(ref_a2[fin] / 2.0)
    assert np.allclose(u[fin], ref_u, rtol=1e-4, atol=1e-5)


def test_fp_step_full_size_sampled(ctx):
    """The launch configuration of the N=64, T=200,000, M=1024 fit (first iteration), BF16:
    sampled rows against the oracle on the same BF16 inputs."""
    from paper_2408_17118_gb300 import ica

    M, n, T = 1024, 64, 200_000
    w = synth.eeg64(0)
    Xw, V, mean = ica.ica_whiten(ctx, torch.from_numpy(w.X).cuda())
    Xt32, Xt16 = ica.ica_reduce(ctx, torch.eye(n, dtype=torch.float64).cuda(), Xw)
    B = ica.ica_init_restarts(ctx, 5, 0, M, n, n)
    Bnew, mom = ica.ica_fp_step(ctx, ica.ICA_BF16, B, n, Xt16, T)
    rows = np.random.default_rng(0).choice(M, 16, replace=False)
    Xq = Xt16[:n, :T].float().cpu().numpy().astype(np.float64)
    Bs = B.cpu().numpy()[rows]
    Zs = b_operand(Bs, 64) @ Xq
    U = (Zs ** 3) @ Xq.T / T - 3.0 * Bs
    S = (np.abs(Zs) ** 3) @ np.abs(Xq).T / T
    err = np.abs(Bnew.cpu().numpy()[rows] - U)
    assert np.all(err <= 2.0 ** -8 * S + 1e-6), (err / (2.0 ** -8 * S + 1e-6)).max()
