"""CPU pins of the pruner oracle (oracle/mlp.py): back-propagation against central finite
differences, closed forms of a zero network and of the first Adam step, standardisation."""
import numpy as np
import pytest

from oracle import mlp


def _rand_params(rng, scale=0.3):
    P = {name: rng.standard_normal(shape) * scale for name, shape in mlp.SIZES}
    P["mean"] = rng.standard_normal(mlp.N_IN)
    P["scale"] = rng.uniform(0.5, 2.0, mlp.N_IN)
    return mlp.pack(P)


def test_layout_size():
    assert mlp.N_PARAMS == 26 + 64 * 13 + 64 + 64 * 64 + 64 + 64 + 1


@pytest.mark.parametrize("pos_weight", [1.0, 4.0])
def test_backprop_matches_finite_differences(pos_weight):
    rng = np.random.default_rng(1)
    params = _rand_params(rng)
    F = rng.standard_normal((40, mlp.N_IN))
    y = (rng.uniform(size=40) < 0.3).astype(np.float64)
    L, g = mlp.loss_grad(params, F, y, pos_weight)
    assert np.isclose(L, mlp.loss(params, F, y, pos_weight))
    idx = list(range(2 * mlp.N_IN, mlp.N_PARAMS, 7)) + [mlp.N_PARAMS - 1]
    gn = mlp.numeric_grad(params, F, y, pos_weight, h=1e-6, idx=idx)
    err = np.abs(g[idx] - gn[idx]).max() / np.abs(gn[idx]).max()
    assert err < 1e-6
    assert np.all(g[:2 * mlp.N_IN] == 0.0)


def test_zero_network_closed_form():
    # every weight zero, b3 = c: p = sigmoid(c) on every row, only b3 has a gradient
    c = 0.7
    P = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    P["scale"] = np.ones(mlp.N_IN)
    P["b3"] = np.array([c])
    params = mlp.pack(P)
    rng = np.random.default_rng(2)
    F = rng.standard_normal((25, mlp.N_IN))
    y = (np.arange(25) % 3 == 0).astype(np.float64)
    p = 1.0 / (1.0 + np.exp(-c))
    assert np.allclose(mlp.forward(params, F), p)
    w = 2.5
    L_expected = -np.mean(w * y * np.log(p) + (1 - y) * np.log(1 - p))
    L, g = mlp.loss_grad(params, F, y, w)
    assert np.isclose(L, L_expected, rtol=1e-14)
    assert np.isclose(g[-1], np.mean(p * (w * y + 1 - y) - w * y), rtol=1e-13)
    assert np.all(g[:-1] == 0.0)


def test_first_adam_step_is_signed_learning_rate():
    # step 1: bias-corrected moments are g and g^2, so the update is lr * g / (|g| + eps)
    rng = np.random.default_rng(3)
    params = _rand_params(rng)
    g = rng.standard_normal(mlp.N_PARAMS)
    g[np.abs(g) < 1e-3] = 1e-3
    lr = 0.01
    new, m, v = mlp.adam_step(params, np.zeros_like(g), np.zeros_like(g), g, 1, lr)
    upd = params - new
    k = 2 * mlp.N_IN
    assert np.all(upd[:k] == 0)
    assert np.allclose(upd[k:], lr * np.sign(g[k:]), rtol=1e-4)


def test_standardisation():
    rng = np.random.default_rng(4)
    F = rng.standard_normal((1000, mlp.N_IN)) * np.arange(1, 14) + np.arange(13)
    mean, scale = mlp.standardisation(F)
    Z = (F - mean) * scale
    assert np.allclose(Z.mean(axis=0), 0, atol=1e-12)
    assert np.allclose(Z.std(axis=0), 1, atol=1e-12)


def test_features_layout():
    a = np.array([[0.1, 0.2, 0.3, 0.4, 0.5], [1.0, 1.5, 2.0, 2.5, 3.0], [-1.0, -2.5, -3.0, -2.0, -2.5]])
    d = -np.arange(15.0).reshape(3, 5)
    F = mlp.features(a, d, 17, 1000, active5=[True, True, False])
    assert F.shape == (3, 13)
    assert np.all(F[:, :5] == a) and np.all(F[:, 5:10] == d)
    assert np.all(F[:, 10] == 17) and np.allclose(F[:, 11], np.log(1000))
    # Upsilon gap at iteration 5 against the best active row (row 1: alpha 3 -> 3 - 2 log 2.5)
    u = lambda x: x - 2 * np.log(x / 2 + 1)
    assert F[1, 12] == 0.0 and np.isclose(F[0, 12], u(0.5) - u(3.0))
    # alpha below -2 is clamped: finite gap
    assert np.isclose(F[2, 12], u(mlp.ALPHA_CLAMP) - u(3.0))


def test_training_reduces_loss_on_separable_data():
    rng = np.random.default_rng(5)
    F = rng.standard_normal((256, mlp.N_IN))
    y = (F[:, 0] + 0.5 * F[:, 3] > 0).astype(np.float64)
    P = {name: rng.standard_normal(shape) * (np.sqrt(2.0 / shape[-1]) if len(shape) == 2 else 0.0)
         for name, shape in mlp.SIZES}
    P["w3"] = rng.standard_normal(mlp.N_HID) * np.sqrt(2.0 / mlp.N_HID)
    mean, scale = mlp.standardisation(F)
    P["mean"], P["scale"] = mean, scale
    params = mlp.pack(P)
    m = np.zeros_like(params)
    v = np.zeros_like(params)
    L0 = mlp.loss(params, F, y)
    for step in range(1, 201):
        _, g = mlp.loss_grad(params, F, y)
        params, m, v = mlp.adam_step(params, m, v, g, step, 0.01)
    L1 = mlp.loss(params, F, y)
    acc = np.mean((mlp.forward(params, F) > 0.5) == (y > 0.5))
    assert L1 < 0.25 * L0 and acc > 0.97
