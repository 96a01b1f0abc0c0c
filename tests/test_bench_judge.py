"""The pruner's judge in bench.py (CPU): the rules by which a pruned fit counts as picking the
unpruned fit's ordered components, checked on hand-built fits of independent sources.

Whitened data here are independent standardised sources themselves (the mixing is the
identity), so the unmixing rows are unit vectors e_k, and each component's objective is the
source's sample Upsilon (Eq. 1 of its kurtosis, Eq. 2)."""
import math

import numpy as np
import pytest

import bench


def _fit_of_sources(T=40_000, seed=3):
    rng = np.random.default_rng(seed)
    S = np.stack([rng.laplace(size=T), rng.uniform(-1, 1, size=T), rng.standard_t(5, size=T),
                  np.sign(rng.standard_normal(T)), rng.standard_normal(T)])
    S = (S - S.mean(axis=1, keepdims=True)) / S.std(axis=1, keepdims=True)
    N = S.shape[0]
    ups = np.array([bench.upsilon64(np.eye(N)[k], S) for k in range(N)])
    order = np.argsort(-ups)
    Wu = np.eye(N)[order]
    comps = []
    for i, k in enumerate(order):
        y = S[k]
        a = float(np.mean(y ** 4) - 3.0)
        comps.append({"i": i + 1, "upsilon": float(ups[k]), "alpha": a})
    return S, Wu, {"components": comps}


def test_upsilon64_matches_eq1():
    S, Wu, st = _fit_of_sources()
    for w, c in zip(Wu, st["components"]):
        a = c["alpha"]
        ref = a - 2.0 * math.log(a / 2.0 + 1.0) if a > -2.0 else math.inf
        assert bench.upsilon64(w, S) == pytest.approx(ref, rel=1e-9)


def test_tie_tolerance_grows_next_to_binary_sources():
    # |dUpsilon/dalpha| = |(alpha/2)/(alpha/2 + 1)|: zero at alpha = 0, unbounded as alpha -> -2
    assert bench.upsilon_tie_tol(0.0) == pytest.approx(1e-6)
    assert bench.upsilon_tie_tol(-1.999) > 100 * bench.upsilon_tie_tol(3.0)
    assert bench.upsilon_tie_tol(-2.0) == math.inf


def test_identical_fits_pass():
    S, Wu, st = _fit_of_sources()
    j = bench.judge_same_components(Wu, st, Wu.copy(), S)
    assert j["ok"] and j["same_position"] == j["non_gaussian"] == 4  # the Gaussian source is below Eq. 3


def test_sign_of_rows_is_free():
    S, Wu, st = _fit_of_sources()
    j = bench.judge_same_components(Wu, st, -Wu, S)
    assert j["ok"] and j["same_position"] == 4


def test_swap_of_distinct_objectives_fails():
    S, Wu, st = _fit_of_sources()
    Wp = Wu.copy()
    Wp[[0, 1]] = Wp[[1, 0]]
    j = bench.judge_same_components(Wu, st, Wp, S)
    assert not j["ok"] and {f[0] for f in j["failed"]} == {1, 2}


def test_swap_within_fp32_resolution_passes():
    S, Wu, st = _fit_of_sources()
    comps = st["components"]
    comps[2]["upsilon"] = comps[1]["upsilon"] + 0.1 * bench.upsilon_tie_tol(comps[1]["alpha"])
    Wp = Wu.copy()
    Wp[[1, 2]] = Wp[[2, 1]]
    j = bench.judge_same_components(Wu, st, Wp, S)
    assert j["ok"] and len(j["swapped_ties"]) == 2 and j["same_position"] == 2


def test_replacement_by_a_worse_direction_fails():
    S, Wu, st = _fit_of_sources()
    Wp = Wu.copy()
    Wp[0] = Wu[-1]  # the Gaussian source's direction in place of the first component
    j = bench.judge_same_components(Wu, st, Wp, S)
    assert not j["ok"] and j["failed"][0][0] == 1


def test_replacement_by_a_better_direction_passes():
    """The unpruned fit's first component is a slightly rotated direction (|cos| < 1 - 1e-5 with
    the source's); the pruned fit has the source's own direction, whose objective is higher: a
    replacement the judge accepts."""
    S, Wu, st = _fit_of_sources()
    k = int(np.argmax(np.abs(Wu[0])))
    v = Wu[0].copy()
    v[(k + 1) % S.shape[0]] += 1e-2
    v /= np.linalg.norm(v)
    Wu2 = Wu.copy()
    Wu2[0] = v
    assert abs(v @ Wu[0]) < 1 - 1e-5
    assert bench.upsilon64(Wu[0], S) > bench.upsilon64(v, S)
    j = bench.judge_same_components(Wu2, st, Wu, S)
    assert j["ok"] and len(j["replaced_ties"]) == 1 and j["replaced_ties"][0][0] == 1


def test_missing_component_fails():
    S, Wu, st = _fit_of_sources()
    j = bench.judge_same_components(Wu, st, Wu[:2], S)
    assert not j["ok"] and [f[0] for f in j["failed"]] == [3, 4]
