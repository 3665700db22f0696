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


def test_adam_constant_gradient_moves_by_lr_every_step():
    """With bias correction, a gradient that stays constant gives m_hat = g and v_hat = g^2 at every
    step (1 - beta^t cancels the zero start), so each of the steps moves the parameter by
    lr * g / (|g| + eps).  A wrong correction (e.g. 1 - beta * t, or none) breaks this from step 2."""
    g = np.array([0.3, -2.0, 5e-2])
    lr, eps = 0.01, 1e-8
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for step in range(1, 7):
        p_new, m, v = mlp.adam(p, g, m, v, step, lr=lr, eps=eps)
        np.testing.assert_allclose(p_new - p, -lr * g / (np.abs(g) + eps), rtol=1e-12)
        p = p_new


def test_adam_two_steps_by_hand():
    """Two steps worked by hand (beta1 = 0.9, beta2 = 0.999, lr = 0.1, eps = 0):
    step 1, g = 0.5:  m = 0.05, v = 2.5e-4, m_hat = 0.5, v_hat = 0.25, move = -0.1;
    step 2, g = -0.25: m = 0.045 - 0.025 = 0.02, v = 2.4975e-4 + 6.25e-5 = 3.1225e-4,
    m_hat = 0.02 / 0.19, v_hat = 3.1225e-4 / 1.999e-3, move = -0.1 m_hat / sqrt(v_hat)."""
    p, m, v = mlp.adam(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 1, lr=0.1, eps=0.0)
    assert abs(p[0] - 0.9) < 1e-15 and abs(m[0] - 0.05) < 1e-16 and abs(v[0] - 2.5e-4) < 1e-18
    p, m, v = mlp.adam(p, np.array([-0.25]), m, v, 2, lr=0.1, eps=0.0)
    assert abs(m[0] - 0.02) < 1e-16 and abs(v[0] - 3.1225e-4) < 1e-17
    m_hat, v_hat = 0.02 / 0.19, 3.1225e-4 / 1.999e-3
    assert abs(p[0] - (0.9 - 0.1 * m_hat / math.sqrt(v_hat))) < 1e-14
    assert abs(p[0] - 0.873366) < 1e-6      # 0.9 - 0.1 * 0.1052632 / 0.3952254
