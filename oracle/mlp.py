"""FP64 oracle of the element network.  TEST INFRASTRUCTURE ONLY.

Sec. 2.4.1: a fully connected network x_i = f_i(A_i x_{i-1} + b_i), i = 1..N_l,
with a nonlinear activation f_i on the hidden layers and the identity on the
output layer.  Sec. 3.1: the loss is the mean absolute error of the network
output and the optimiser is Adam.  The activation here is the exact GELU,
0.5 x (1 + erf(x / sqrt 2)) (the paper uses ELU; both are offered by the
library); erf is scipy's.

Row-major batches: x has shape [batch, width]; a weight A_i has shape
[out, in] so that a layer computes x @ A_i.T + b_i.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def elu(x):
    return np.where(x > 0, x, np.expm1(np.minimum(x, 0.0)))


def elu_grad(x):
    return np.where(x > 0, 1.0, np.exp(np.minimum(x, 0.0)))


ACT = {"gelu": (gelu, gelu_grad), "elu": (elu, elu_grad)}


def forward(weights, biases, x, act="gelu"):
    """Returns the list of pre-activations z_i and the output; z_i = x_{i-1} A_i^T + b_i."""
    f, _ = ACT[act]
    zs = []
    h = np.asarray(x, dtype=np.float64)
    for i, (A, b) in enumerate(zip(weights, biases)):
        z = h @ A.T + b
        zs.append(z)
        h = f(z) if i + 1 < len(weights) else z
    return zs, h


def backward(weights, biases, x, zs, dy, act="gelu"):
    """Gradients (dA_i, db_i) of sum(dy * output) by the chain rule through forward()."""
    f, fp = ACT[act]
    nl = len(weights)
    dA, db = [None] * nl, [None] * nl
    g = np.asarray(dy, dtype=np.float64)
    for i in range(nl - 1, -1, -1):
        if i + 1 < nl:
            g = g * fp(zs[i])
        h_prev = np.asarray(x, dtype=np.float64) if i == 0 else f(zs[i - 1])
        dA[i] = g.T @ h_prev
        db[i] = g.sum(axis=0)
        g = g @ weights[i]
    return dA, db


def mae(y, t):
    """Mean absolute error over every entry and its gradient with respect to y (sign(y - t)/count;
    the subgradient 0 is taken where y == t)."""
    d = y - t
    return float(np.mean(np.abs(d))), np.sign(d) / d.size


def adam(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; returns new (param, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v
