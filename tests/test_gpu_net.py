"""GPU parity of the element network (tcgen05 BF16 GEMMs) against the FP64 oracle network, and
the learned local stage (training, inference, energy-balance estimate, classical fallback)."""

import numpy as np
import pytest

import workloads as W
from oracle import hdg, mlp
from tests import _helpers as H

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round-to-nearest-even to bfloat16, returned as float64 (input preparation for the oracle)."""
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _set_random(net, rng, scale=1.0):
    Ws, bs = [], []
    for l in range(net.n_layers):
        out, inp = net.layer_shape(l)
        fan = net.n_feat if l == 0 else inp
        Wl = rng.uniform(-1, 1, (out, inp)) * scale / np.sqrt(fan)
        if l == 0:
            Wl[:, net.n_feat:] = 0.0
        bl = rng.uniform(-0.1, 0.1, out)
        net.elrt_net_params(l, "W", Wl)
        net.elrt_net_params(l, "b", bl)
        Ws.append(bf16_round(Wl))
        bs.append(np.asarray(bl, dtype=np.float32).astype(np.float64))
    return Ws, bs


@pytest.mark.parametrize("p,N,n", [(2, 4, 300), (6, 16, 130)])
def test_linear_network_is_an_exact_bf16_gemm(lib, p, N, n):
    """n_hidden = 0 (the paper's linear-regression case): y = x A^T + b.  BF16 x BF16 products are
    exact in FP32, so only FP32 accumulation separates the tensor-core result from FP64."""
    import torch
    net = lib.Net(p, N, n_hidden=0, width=64, seed=1)
    rng = np.random.default_rng(0)
    Ws, bs = _set_random(net, rng)
    x = rng.normal(size=(n, net.n_feat_pad))
    x[:, net.n_feat:] = 0.0
    y = torch.empty(n, net.n_out, device="cuda", dtype=torch.float32)
    net.elrt_net_forward(torch.tensor(x, dtype=torch.float32, device="cuda"), y)
    ref = bf16_round(x) @ Ws[0].T + bs[0]
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)
    net.close()


def test_mlp_forward_matches_oracle(lib):
    import torch
    net = lib.Net(2, 4, n_hidden=3, width=128, seed=2)
    rng = np.random.default_rng(1)
    Ws, bs = _set_random(net, rng)
    n = 200
    x = rng.normal(size=(n, net.n_feat_pad))
    x[:, net.n_feat:] = 0.0
    y = torch.empty(n, net.n_out, device="cuda", dtype=torch.float32)
    net.elrt_net_forward(torch.tensor(x, dtype=torch.float32, device="cuda"), y)
    _, ref = mlp.forward(Ws, bs, bf16_round(x), "gelu")
    got = y.cpu().numpy()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 1e-2, rel          # hidden activations are stored in BF16 between layers
    net.close()


@pytest.mark.parametrize("act,p,N,B", [("gelu", 2, 4, 128), ("elu", 2, 4, 128), ("gelu", 4, 8, 128),
                                       ("elu", 4, 8, 64)])
def test_gradients_match_oracle(lib, act, p, N, B):
    """Mean-absolute-error gradients of every layer (tcgen05 dgrad / wgrad GEMMs) against the
    FP64 backward pass of the oracle on the same BF16 weights, inputs and targets.  p = 4, N = 8
    (8400 outputs) takes the K-sliced input-gradient GEMM of the output layer and ragged
    256-column output tiles; B = 64 leaves every 128-row tile half empty."""
    import torch
    net = lib.Net(p, N, n_hidden=2, width=128, activation=act, seed=3)
    rng = np.random.default_rng(2)
    Ws, bs = _set_random(net, rng)
    x = rng.normal(size=(B, net.n_feat_pad))
    x[:, net.n_feat:] = 0.0
    t = rng.normal(size=(B, net.n_out))
    loss = net.elrt_net_train_step(torch.tensor(x, dtype=torch.float32, device="cuda"),
                                   torch.tensor(t, dtype=torch.float32, device="cuda"), lr=0.0)
    xb = bf16_round(x)
    zs, y = mlp.forward(Ws, bs, xb, act)
    l_ref, dy = mlp.mae(y, t)
    assert abs(loss - l_ref) < 1e-2 * l_ref
    dW, db = mlp.backward(Ws, bs, xb, zs, dy, act)
    for l in range(net.n_layers):
        gW = net.elrt_net_params(l, "dW")
        gb = net.elrt_net_params(l, "db")
        rW = np.linalg.norm(gW - dW[l]) / np.linalg.norm(dW[l])
        rb = np.linalg.norm(gb - db[l]) / np.linalg.norm(db[l])
        assert rW < 5e-2 and rb < 5e-2, (l, rW, rb)
    net.close()


def test_adam_first_step(lib):
    """One Adam step from zero moments moves every weight by lr * sign(g) (|g| >> eps)."""
    import torch
    net = lib.Net(2, 4, n_hidden=1, width=64, seed=4)
    rng = np.random.default_rng(3)
    Ws, bs = _set_random(net, rng)
    W_before = [net.elrt_net_params(l, "W") for l in range(net.n_layers)]
    B = 64
    x = rng.normal(size=(B, net.n_feat_pad))
    x[:, net.n_feat:] = 0.0
    t = rng.normal(size=(B, net.n_out)) * 3
    lr = 1e-3
    net.elrt_net_train_step(torch.tensor(x, dtype=torch.float32, device="cuda"),
                            torch.tensor(t, dtype=torch.float32, device="cuda"), lr=lr)
    xb = bf16_round(x)
    zs, y = mlp.forward(Ws, bs, xb)
    _, dy = mlp.mae(y, t)
    dW, _ = mlp.backward(Ws, bs, xb, zs, dy)
    for l in range(net.n_layers):
        step = net.elrt_net_params(l, "W") - W_before[l]
        live = np.abs(dW[l]) > 1e-6
        agree = np.isclose(step[live], -lr * np.sign(dW[l][live]), atol=lr * 1e-2)
        assert agree.mean() > 0.98, (l, agree.mean())
    net.close()


def test_adam_step_refreshes_the_bf16_weights(lib):
    """After an Adam step the forward pass (BF16 W) and the input-gradient GEMMs (BF16 W^T) use the
    updated weights: the gradients of a second batch match the oracle on the new FP32 masters."""
    import torch
    net = lib.Net(4, 8, n_hidden=2, width=128, seed=6)
    rng = np.random.default_rng(5)
    _set_random(net, rng)
    B = 128

    def data():
        x = rng.normal(size=(B, net.n_feat_pad))
        x[:, net.n_feat:] = 0.0
        return x, rng.normal(size=(B, net.n_out))

    def dev(a):
        return torch.tensor(a, dtype=torch.float32, device="cuda")

    x1, t1 = data()
    net.elrt_net_train_step(dev(x1), dev(t1), lr=3e-2)
    Ws = [bf16_round(net.elrt_net_params(l, "W")) for l in range(net.n_layers)]
    bs = [np.asarray(net.elrt_net_params(l, "b"), dtype=np.float64) for l in range(net.n_layers)]
    x2, t2 = data()
    loss = net.elrt_net_train_step(dev(x2), dev(t2), lr=0.0)
    xb = bf16_round(x2)
    zs, y = mlp.forward(Ws, bs, xb, "gelu")
    l_ref, dy = mlp.mae(y, t2)
    assert abs(loss - l_ref) < 1e-2 * l_ref
    dW, _ = mlp.backward(Ws, bs, xb, zs, dy, "gelu")
    for l in range(net.n_layers):
        gW = net.elrt_net_params(l, "dW")
        rW = np.linalg.norm(gW - dW[l]) / np.linalg.norm(dW[l])
        assert rW < 5e-2, (l, rW)
    net.close()


# ------------------------------------------------------------------ the learned local stage
P, NA = 2, 4


@pytest.fixture(scope="module")
def trained(lib):
    """A small element network (p = 2, N = 4) fitted to classical labels of 4096 elements."""
    import torch
    ctx = lib.Context(P, NA, 0.85, lib.ANG_FV0)
    xi, _ = lib.elrt_lgl(P)
    xx, zz = np.meshgrid(xi, xi)          # node i = a + (p+1) b: x index fastest
    def batch(n, hold):
        eb = W.element_batch(n, holdout=hold)
        kap = eb.kappa_at(xx.reshape(-1), zz.reshape(-1))
        return (torch.tensor(kap, device="cuda"), torch.tensor(eb.omega, device="cuda"),
                torch.tensor(eb.h, device="cuda"))
    def labels(k, o, h):
        n = o.numel()
        a = torch.empty(n, ctx.nin, ctx.nin, device="cuda", dtype=torch.float32)
        m = torch.empty(n, ctx.nm, ctx.nin, device="cuda", dtype=torch.float32)
        ctx.elrt_build_local(k, o, 1.0, a, m, mode=lib.LOCAL_FP32_IR, refine_steps=1, h_elem=h)
        return a, m
    tr = batch(4096, False)
    ho = batch(512, True)
    tr_l, ho_l = labels(*tr), labels(*ho)
    net = lib.Net(P, NA, n_hidden=3, width=256, seed=5)
    losses = net.elrt_net_fit(tr[0], tr[1], tr[2], tr_l[0], tr_l[1], epochs=60, batch=256, lr=1e-3, seed=1)
    yield dict(ctx=ctx, net=net, tr=tr, ho=ho, tr_l=tr_l, ho_l=ho_l, losses=losses)
    net.close()
    ctx.close()


def test_training_reduces_the_loss(trained):
    L = trained["losses"]
    assert np.all(np.isfinite(L))
    assert L[-1] < 0.2 * L[0], L


def test_trained_network_beats_the_mean_operator(lib, trained):
    """On held-out elements the network's in2out is far closer to the classical one than the
    best input-independent guess (the training-set mean operator)."""
    import torch
    net, ho, (a_ref, m_ref) = trained["net"], trained["ho"], trained["ho_l"]
    n = ho[1].numel()
    a = torch.empty_like(a_ref)
    m = torch.empty_like(m_ref)
    net.elrt_net_infer(ho[0], ho[1], 1.0, a, m, h_elem=ho[2])
    err = (torch.linalg.norm((a - a_ref).reshape(n, -1), dim=1) / torch.linalg.norm(a_ref.reshape(n, -1), dim=1))
    mean_op = trained["tr_l"][0].mean(dim=0, keepdim=True)
    err0 = (torch.linalg.norm((mean_op - a_ref).reshape(n, -1), dim=1) / torch.linalg.norm(a_ref.reshape(n, -1), dim=1))
    assert float(err.median()) < 0.25 * float(err0.median()), (float(err.median()), float(err0.median()))


def test_fallback_reproduces_the_classical_operators(lib, trained):
    import torch
    ctx, net, ho, (a_ref, m_ref) = trained["ctx"], trained["net"], trained["ho"], trained["ho_l"]
    n = ho[1].numel()
    a = torch.empty_like(a_ref)
    m = torch.empty_like(m_ref)
    est = torch.empty(n, device="cuda", dtype=torch.float32)
    # tolerance so small that every element falls back: the result is the classical solve
    nf = lib.elrt_build_local_learned(ctx, net, ho[0], ho[1], 1.0, a, m, tol=1e-30, h_elem=ho[2], estimate=est)
    assert nf == n
    np.testing.assert_allclose(a.cpu().numpy(), a_ref.cpu().numpy(), atol=1e-6)
    # no fallback: the network's own operators; the estimate of classical operators is ~0
    nf = lib.elrt_build_local_learned(ctx, net, ho[0], ho[1], 1.0, a, m, tol=1e30, h_elem=ho[2], estimate=est)
    assert nf == 0
    est_net = est.clone()
    nf = lib.elrt_build_local_learned(ctx, net, ho[0], ho[1], 1.0, a, m, tol=float(est_net.median()),
                                      h_elem=ho[2], estimate=est)
    assert 0 < nf < n
    assert float(est_net.median()) > 1e-5
