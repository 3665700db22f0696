"""Pins of the FP64 network oracle: finite differences and closed forms (CPU only)."""

import math

import numpy as np
import pytest

from oracle import mlp


def _net(rng, sizes):
    Ws = [rng.normal(0, 1 / math.sqrt(a), (b, a)) for a, b in zip(sizes[:-1], sizes[1:])]
    bs = [rng.normal(0, 0.1, b) for b in sizes[1:]]
    return Ws, bs


def test_gelu_closed_form_values():
    # GELU(x) = x Phi(x): Phi(0) = 1/2, Phi(1) = 0.8413447460685429 (normal CDF table)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(np.array([-1.0]))[0] + 1 - 0.8413447460685429) < 1e-15


@pytest.mark.parametrize("act", ["gelu", "elu"])
def test_activation_derivative_by_finite_differences(act):
    f, fp = mlp.ACT[act]
    x = np.linspace(-4, 4, 81) + 0.013
    h = 1e-6
    np.testing.assert_allclose(fp(x), (f(x + h) - f(x - h)) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("act", ["gelu", "elu"])
def test_backward_by_finite_differences(act):
    rng = np.random.default_rng(0)
    sizes = [5, 7, 6, 4]
    Ws, bs = _net(rng, sizes)
    x = rng.normal(size=(3, 5))
    dy = rng.normal(size=(3, 4))
    zs, y = mlp.forward(Ws, bs, x, act)
    dW, db = mlp.backward(Ws, bs, x, zs, dy, act)
    h = 1e-6
    for l in range(3):
        for (i, j) in [(0, 0), (1, 2), (sizes[l + 1] - 1, sizes[l] - 1)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            num = (np.sum(dy * mlp.forward(Wp, bs, x, act)[1]) - np.sum(dy * mlp.forward(Wm, bs, x, act)[1])) / (2 * h)
            assert abs(num - dW[l][i, j]) < 1e-7 * max(1, abs(num))
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][1] += h
        bm[l][1] -= h
        num = (np.sum(dy * mlp.forward(Ws, bp, x, act)[1]) - np.sum(dy * mlp.forward(Ws, bm, x, act)[1])) / (2 * h)
        assert abs(num - db[l][1]) < 1e-7 * max(1, abs(num))


def test_single_layer_is_linear_regression():
    """N_l = 1: the network is the affine map x A^T + b (no activation on the output layer)."""
    rng = np.random.default_rng(1)
    Ws, bs = _net(rng, [4, 3])
    x = rng.normal(size=(5, 4))
    np.testing.assert_allclose(mlp.forward(Ws, bs, x)[1], x @ Ws[0].T + bs[0], atol=1e-15)


def test_mae_and_gradient():
    y = np.array([[1.0, -2.0], [0.5, 3.0]])
    t = np.array([[0.0, 0.0], [1.0, 3.0]])
    loss, g = mlp.mae(y, t)
    assert loss == (1 + 2 + 0.5 + 0) / 4
    np.testing.assert_array_equal(g, np.array([[1, -1], [-1, 0]]) / 4)


def test_adam_first_step_is_signed_lr():
    """After one step from zero moments, the bias-corrected update is lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-8)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
