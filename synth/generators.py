"""Seeded synthetic inputs for the ordering ICA (Matsuda & Yamaguchi, arXiv 2408.17118).

This module draws random numbers and nothing else: source signals, mixing matrices, additive
noise and random initial restart matrices. It holds none of the method's arithmetic (no
whitening, no kurtosis, no fixed-point update). Both sides of every parity check take their
inputs from here: the FP64 CPU oracle (through the tests) and the CUDA path (through the tests
and bench.py). Every draw comes from numpy's PCG64 keyed by an explicit seed and a stream tag,
so a workload is reproducible bit for bit on x86 and Arm hosts.

Workload shapes follow the paper's experiments:

* ``small_mixture``: N=8 sources {Laplace, uniform, Student-t nu=5, binary +-1, centred exponential,
  Laplace^2, uniform, Gaussian}, T=10,000, A ~ N(0,1), M=64 restarts.
* ``eeg_like``: EEG-shaped data (the paper's EEG experiment uses N=61 channels and about
  160,000-190,000 samples, Section 4.3; the recordings are not available here, so this
  generator stands in for them): 3/4 of the channels carry non-Gaussian sources, half of them
  super-Gaussian (Laplace, Student-t nu in {4, 6, 10}) and half sub-Gaussian (uniform, binary,
  sinusoid with random frequency and phase); the rest are Gaussian; sigma=0.05 sensor noise.
  Used at N=64/T=2e5/M=1024 (``eeg64``), N=128/T=5e5/M=4096 (``eeg128``) and
  N=256/T=1e6/M=8192 (``eeg256``).
* ``batch_of_datasets``: 32 independent small-mixture-style datasets with N drawn from
  {16, 32, 48, 64, 96, 128} and T log-uniform in [2e4, 4e5].
* ``ggd_paper``: the artificial datasets of Section 4.2: generalised Gaussian sources with
  rho = 2 * 2^(i/4), i in {-10..-1, 1..10} (N=20), optionally plus 10 Gaussian sources (N=30).

Sources are standardised to zero sample mean and unit sample variance (1/T normalisation), as
Theorem 1 assumes normalised sources.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "rng_for",
    "standardise",
    "make_source",
    "small_mixture",
    "eeg_like",
    "eeg64",
    "eeg128",
    "eeg256",
    "batch_of_datasets",
    "ggd_paper",
    "ggd_source",
    "restart_inits",
    "small_random",
    "SMALL_SOURCES",
]


def rng_for(seed: int, *tags: int) -> np.random.Generator:
    """PCG64 generator keyed by (seed, tags...)."""
    return np.random.default_rng([int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF, *[int(t) for t in tags]])


def standardise(s: np.ndarray) -> np.ndarray:
    """Zero sample mean, unit sample variance (population, 1/T)."""
    s = np.asarray(s, dtype=np.float64)
    s = s - s.mean()
    return s / math.sqrt(float(np.mean(s * s)))


def ggd_source(rng: np.random.Generator, rho: float, T: int) -> np.ndarray:
    """Generalised Gaussian p(u) ~ exp(-(|u|/beta)^rho) with unit variance (Section 4.2).

    With v = (|u|/beta)^rho, v ~ Gamma(1/rho, 1); beta = sqrt(Gamma(1/rho)/Gamma(3/rho))
    makes the variance one. The sign is drawn independently.
    """
    beta = math.sqrt(math.gamma(1.0 / rho) / math.gamma(3.0 / rho))
    v = rng.gamma(1.0 / rho, 1.0, T)
    sign = rng.integers(0, 2, T) * 2 - 1
    return sign * beta * v ** (1.0 / rho)


def make_source(kind: str, rng: np.random.Generator, T: int) -> np.ndarray:
    """One raw (unstandardised) source signal of length T."""
    if kind == "laplace":
        return rng.laplace(0.0, 1.0, T)
    if kind == "uniform":
        return rng.uniform(-1.0, 1.0, T)
    if kind.startswith("t"):  # "t4", "t5", "t6", "t10": Student-t with nu degrees of freedom
        return rng.standard_t(int(kind[1:]), T)
    if kind == "binary":
        return (rng.integers(0, 2, T) * 2 - 1).astype(np.float64)
    if kind == "exp":  # centred exponential
        return rng.exponential(1.0, T) - 1.0
    if kind == "laplace2":
        return rng.laplace(0.0, 1.0, T) ** 2
    if kind == "gauss":
        return rng.standard_normal(T)
    if kind == "sinusoid":
        f = rng.uniform(5.0, 50.0)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        t = np.arange(T, dtype=np.float64)
        return np.sin(2.0 * math.pi * f * t / T + phi)
    if kind.startswith("ggd"):  # "ggd:<rho>"
        return ggd_source(rng, float(kind.split(":")[1]), T)
    raise ValueError(f"unknown source kind {kind!r}")


SMALL_SOURCES = ["laplace", "uniform", "t5", "binary", "exp", "laplace2", "uniform", "gauss"]


@dataclass
class Workload:
    """A mixed data set X = A S (+ noise) plus the truth that produced it."""

    name: str
    X: np.ndarray          # N x T float32, row-major, T contiguous (the library's input)
    A: np.ndarray          # N x N float64 mixing matrix
    S: np.ndarray | None   # N x T float32 standardised sources (None when not kept)
    kinds: list[str]
    M: int                 # restarts
    n_components: int
    iters: int
    tol: float
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def T(self) -> int:
        return int(self.X.shape[1])


def _mix(name, kinds, T, seed, M, iters, tol, noise=0.0, keep_sources=True, n_components=None):
    N = len(kinds)
    S = np.empty((N, T), dtype=np.float32)
    for i, kind in enumerate(kinds):
        S[i] = standardise(make_source(kind, rng_for(seed, 1, i), T)).astype(np.float32)
    A = rng_for(seed, 2).standard_normal((N, N))
    X = (A.astype(np.float32) @ S).astype(np.float32)
    if noise > 0.0:
        g = rng_for(seed, 3)
        for i in range(N):  # row by row keeps the peak memory at one row of noise
            X[i] += (noise * g.standard_normal(T)).astype(np.float32)
    return Workload(name=name, X=np.ascontiguousarray(X), A=A, S=S if keep_sources else None,
                    kinds=list(kinds), M=M, n_components=N if n_components is None else n_components,
                    iters=iters, tol=tol, seed=seed)


def small_mixture(seed: int = 0, T: int = 10_000, M: int = 64, iters: int = 200, tol: float = 1e-10) -> Workload:
    """N=8 plain ordering-ICA workload: eight distinct sources, no noise."""
    return _mix("small_mixture_N8", SMALL_SOURCES, T, seed, M, iters, tol)


def _eeg_kinds(N: int) -> list[str]:
    n_ng = (3 * N) // 4
    n_super = n_ng // 2
    n_sub = n_ng - n_super
    sup = ["laplace", "t4", "t6", "t10"]
    sub = ["uniform", "binary", "sinusoid"]
    kinds = [sup[i % len(sup)] for i in range(n_super)] + [sub[i % len(sub)] for i in range(n_sub)]
    return kinds + ["gauss"] * (N - n_ng)


def eeg_like(N: int, T: int, M: int, seed: int = 0, iters: int = 30, tol: float = 1e-6,
             noise: float = 0.05, keep_sources: bool = False, n_components: int | None = None) -> Workload:
    """EEG-shaped mixture: 3/4 non-Gaussian (half super-, half sub-Gaussian), 1/4 Gaussian, noise."""
    return _mix(f"eeg_like_N{N}_T{T}_M{M}", _eeg_kinds(N), T, seed, M, iters, tol, noise=noise,
                keep_sources=keep_sources, n_components=n_components)


def eeg64(seed: int = 0, **kw) -> Workload:
    """EEG-like N=64 channels, T=200,000 samples, M=1024 restarts, all 64 components."""
    return eeg_like(64, 200_000, 1024, seed=seed, **kw)


def eeg128(seed: int = 0, **kw) -> Workload:
    """Same generator at N=128, T=500,000, M=4096."""
    return eeg_like(128, 500_000, 4096, seed=seed, **kw)


def eeg256(seed: int = 0, **kw) -> Workload:
    """Same generator at N=256, T=1,000,000, M=8192."""
    return eeg_like(256, 1_000_000, 8192, seed=seed, **kw)


def batch_of_datasets(count: int = 32, seed: int = 0, M: int = 512, iters: int = 30, tol: float = 1e-6,
                      Ns=(16, 32, 48, 64, 96, 128), T_lo: int = 20_000, T_hi: int = 400_000,
                      keep_sources: bool = False) -> list[Workload]:
    """Independent datasets of uneven N and T (sources cycle through the small-mixture list)."""
    g = rng_for(seed, 7)
    out = []
    for k in range(count):
        N = int(g.choice(Ns))
        T = int(round(math.exp(g.uniform(math.log(T_lo), math.log(T_hi)))))
        kinds = [SMALL_SOURCES[i % len(SMALL_SOURCES)] for i in range(N)]
        out.append(_mix(f"batch{k}_N{N}_T{T}", kinds, T, seed * 1000 + 17 + k, M, iters, tol,
                        keep_sources=keep_sources))
    return out


def ggd_paper(seed: int = 0, T: int = 10_000, M: int = 100, with_gaussians: bool = False,
              iters: int = 30, tol: float = 1e-6) -> Workload:
    """Section 4.2 artificial data: rho = 2*2^(i/4), i in {-10..-1, 1..10}, optional 10 Gaussians."""
    rhos = [2.0 * 2.0 ** (i / 4.0) for i in list(range(-10, 0)) + list(range(1, 11))]
    kinds = [f"ggd:{r!r}" for r in rhos] + (["gauss"] * 10 if with_gaussians else [])
    w = _mix(f"ggd_N{len(kinds)}", kinds, T, seed, M, iters, tol)
    w.extra["rho"] = rhos
    return w


def restart_inits(M: int, N: int, n_components: int, seed: int) -> np.ndarray:
    """Explicit initial restart matrices B0: n_components x M x N float32, i.i.d. N(0,1).

    Component i (0-based) uses the first N-i columns of B0[i] (its reduced dimension); the
    method normalises each row itself. Passing the same B0 to the oracle and to the CUDA path
    removes the random-number generator from a parity comparison.
    """
    g = rng_for(seed, 11)
    return g.standard_normal((n_components, M, N)).astype(np.float32)


def small_random(n: int, T: int, seed: int, kind: str = "mixed") -> np.ndarray:
    """A small n x T float32 matrix with unit-variance non-Gaussian rows (kernel-level tests)."""
    g = rng_for(seed, 13)
    if kind == "gauss":
        return g.standard_normal((n, T)).astype(np.float32)
    rows = []
    kinds = ["laplace", "uniform", "t6", "binary", "exp", "gauss", "sinusoid"]
    for i in range(n):
        rows.append(standardise(make_source(kinds[i % len(kinds)], rng_for(seed, 14, i), T)))
    return np.asarray(rows, dtype=np.float32)
