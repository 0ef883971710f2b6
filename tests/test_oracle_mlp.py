"""Pins of the selector-network oracle: analytic gradients against central finite differences,
and the Adam step against its closed form on one coordinate."""
import numpy as np

from oracle import mlp


def _data(seed=0, n=11, nin=5, nh=7, nout=3):
    rng = np.random.default_rng(seed)
    params = [rng.normal(scale=0.5, size=s) for s in mlp.shapes(nin, nh, nout)]
    X = rng.normal(size=(n, nin))
    T = rng.normal(size=(n, nout))
    M = (rng.uniform(size=(n, nout)) < 0.8).astype(float)
    return params, X, T, M


def test_gradients_match_finite_differences():
    params, X, T, M = _data()
    loss, grads = mlp.loss_and_grads(params, X, T, M)
    flat = mlp.flatten(params)
    g = mlp.flatten(grads)
    h = 1e-6
    for i in range(0, flat.size, 3):
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp = mlp.loss_and_grads(mlp.unflatten(fp, 5, 7, 3), X, T, M)[0]
        lm = mlp.loss_and_grads(mlp.unflatten(fm, 5, 7, 3), X, T, M)[0]
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-7 * max(1.0, abs(g[i]))


def test_mask_removes_targets():
    params, X, T, M = _data(seed=1)
    M[:, 1] = 0.0
    T2 = T.copy()
    T2[:, 1] += 100.0
    assert mlp.loss_and_grads(params, X, T, M)[0] == mlp.loss_and_grads(params, X, T2, M)[0]


def test_adam_first_step_is_lr_times_sign():
    # after one step from m = v = 0 the bias-corrected update is lr * g / (|g| + eps)
    flat = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    new, m, v = mlp.adam_step(flat, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(new, flat - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
