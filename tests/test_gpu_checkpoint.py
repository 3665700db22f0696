"""Network checkpoint round trip on the GPU: a reloaded network infers bit-identically and resumes
training where the saved one stands (same Adam moments and step counter: the next step gives the
same loss and weights, up to the summation order of the loss)."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_save_load_infers_identically_and_resumes(lib, tmp_path):
    import torch
    p, N = 2, 4
    ctx = lib.Context(p, N, 0.85, lib.ANG_FV0)
    xi, _ = lib.elrt_lgl(p)
    xx, zz = np.meshgrid(xi, xi)
    eb = W.element_batch(1024)
    k = torch.tensor(eb.kappa_at(xx.reshape(-1), zz.reshape(-1)), device="cuda")
    o = torch.tensor(eb.omega, device="cuda")
    h = torch.tensor(eb.h, device="cuda")
    n = len(eb)
    a = torch.empty(n, ctx.nin, ctx.nin, device="cuda", dtype=torch.float32)
    m = torch.empty(n, ctx.nm, ctx.nin, device="cuda", dtype=torch.float32)
    ctx.elrt_build_local(k, o, 1.0, a, m, mode=lib.LOCAL_FP32_IR, refine_steps=1, h_elem=h)
    net = lib.Net(p, N, n_hidden=2, width=128, activation="elu", seed=3)
    net.elrt_net_fit(k, o, h, a, m, epochs=3, batch=256, lr=1e-3, seed=1)
    path = str(tmp_path / "net.ckpt")
    net.elrt_net_save(path)
    info = lib.elrt_net_file_info(path)
    assert info["standardised"] == 1 and info["adam_step"] == 3 * (n // 256) and info["activation"] == 1
    net2 = lib.Net.elrt_net_load(path)
    assert (net2.n_out, net2.n_layers, net2.n_params) == (net.n_out, net.n_layers, net.n_params)
    a1, m1, a2, m2 = (torch.empty_like(t) for t in (a, m, a, m))
    net.elrt_net_infer(k, o, 1.0, a1, m1, h_elem=h)
    net2.elrt_net_infer(k, o, 1.0, a2, m2, h_elem=h)
    assert torch.equal(a1, a2) and torch.equal(m1, m2)
    # resume: one Adam step on the same batch from both networks
    rng = np.random.default_rng(5)
    x = torch.tensor(rng.normal(size=(128, net.n_feat_pad)), dtype=torch.float32, device="cuda")
    x[:, net.n_feat:] = 0
    t = torch.tensor(rng.normal(size=(128, net.n_out)), dtype=torch.float32, device="cuda")
    l1 = net.elrt_net_train_step(x, t, lr=1e-3)
    l2 = net2.elrt_net_train_step(x, t, lr=1e-3)
    assert abs(l1 - l2) <= 1e-6 * abs(l1)           # the loss is summed with atomics (order varies)
    for l in range(net.n_layers):
        np.testing.assert_allclose(net2.elrt_net_params(l, "W"), net.elrt_net_params(l, "W"), rtol=1e-6, atol=1e-9)
    # a damaged file is refused without creating a network
    b = bytearray(open(path, "rb").read())
    b[200] ^= 1
    open(path, "wb").write(bytes(b))
    with pytest.raises(lib.ElrtError):
        lib.Net.elrt_net_load(path)
    net.close()
    net2.close()
    ctx.close()
