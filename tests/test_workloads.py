"""The seeded input generators shared by the tests, the bench and the oracle runs: every input is
reproducible from its workload index, and the drawn quantities stay inside the stated recipes."""

import numpy as np
import pytest

import workloads as W


def test_same_workload_same_numbers():
    a, b = W.element_batch(300), W.element_batch(300)
    for f in ("h", "ell", "mu", "sd", "omega", "wavevectors", "phases"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    xi = np.array([-1.0, 0.0, 1.0])
    np.testing.assert_array_equal(a.kappa_at(xi, xi), b.kappa_at(xi, xi))
    fa, fb = W.problem_batch_fields(5), W.problem_batch_fields(5)
    for x, y in zip(fa, fb):
        assert (x.nx, x.nz, x.p) == (y.nx, y.nz, y.p)
        np.testing.assert_array_equal(x.omega, y.omega)
        np.testing.assert_array_equal(x.inflow, y.inflow)


def test_chunks_and_holdout_are_independent_streams():
    a = W.element_batch(256, chunk=128)
    # the second chunk is its own counter block, not a continuation of the first
    assert not np.array_equal(a.h[:128], a.h[128:])
    # a prefix of a batch is the same elements when the chunking agrees
    np.testing.assert_array_equal(W.element_batch(128, chunk=128).h, a.h[:128])
    ho = W.element_batch(256, holdout=True, chunk=128)
    assert not np.intersect1d(a.h, ho.h).size


def test_element_recipe_ranges():
    eb = W.element_batch(2000)
    assert eb.h.min() >= 0.05 and eb.h.max() <= 1.0
    r = eb.ell / eb.h
    assert r.min() >= 0.1 - 1e-12 and r.max() <= 2.0 + 1e-12
    assert eb.mu.min() >= -2.0 and eb.mu.max() <= 3.5
    assert eb.sd.min() >= 0.0 and eb.sd.max() <= 1.5
    assert eb.omega.min() >= 0.9 and eb.omega.max() <= 1.0
    xi = np.linspace(-1, 1, 5)
    kap = eb.kappa_at(xi, xi)
    assert np.all(kap > 0) and np.all(np.isfinite(kap))
    # log kappa is mu + sd f with f of unit variance: the standardised field has mean ~0, variance ~1
    f = (np.log(kap) - eb.mu[:, None]) / np.where(eb.sd > 0.05, eb.sd, np.nan)[:, None]
    f = f[np.isfinite(f)]
    assert abs(f.mean()) < 0.1 and 0.8 < f.var() < 1.2


def test_batch_fields_recipe():
    for pr in W.problem_batch_fields(40):
        assert 16 <= pr.nx <= 128 and 16 <= pr.nz <= 128
        assert pr.p in (4, 6, 8)
        assert pr.h == pytest.approx(10.0 / max(pr.nx, pr.nz))
        assert np.all(pr.omega >= 0.9) and np.all(pr.omega <= 1.0) and np.ptp(pr.omega) == 0.0
        _, total = W.inflow_layout(pr.nx, pr.nz, pr.p, pr.n_angles)
        assert pr.inflow.shape == (total,)
        assert np.all(pr.inflow >= 0.0)


def test_benchmark_slab():
    pr = W.problem_gaussian_slab(n=64)
    assert (pr.nx, pr.nz, pr.p, pr.n_angles, pr.hg_g) == (64, 64, 6, 16, 0.85)
    assert pr.h == pytest.approx(10.0 / 64) and np.all(pr.omega == 0.99)
    # the cloud: 0.1 km^-1 background plus a Gaussian of amplitude 20 at the slab centre
    k = pr.kappa(np.array([5.0, 0.0]), np.array([5.0, 0.0]))
    assert k[0] == pytest.approx(20.1) and k[1] == pytest.approx(0.1, abs=1e-3)
    _, total = W.inflow_layout(64, 64, 6, 16)
    assert pr.inflow.shape == (total,) and pr.inflow.max() > 0.0
    # the beam enters through the top only
    offs, _ = W.inflow_layout(64, 64, 6, 16)
    per_face = 7 * 8
    top = pr.inflow[offs[2]:offs[2] + 64 * per_face]
    assert top.max() > 0.0
    assert np.count_nonzero(pr.inflow) == np.count_nonzero(top)


def test_cloud_slab_torch_evaluation_matches_numpy():
    """The lognormal cloud slab's field evaluated with torch (used on the GPU for the 6.4 M nodes of
    the 512 x 256 slab) equals the numpy evaluation."""
    import torch
    prob = W.problem_cloud_slab()
    r = np.random.default_rng(3)
    x = np.concatenate([r.uniform(0, 50, 300), [5.0, 45.0, 25.0]])
    z = np.concatenate([r.uniform(0, 25, 300), [10.0, 10.0, 5.0]])
    ref = prob.kappa(x, z)
    got = prob.kappa.evaluate_torch(torch.tensor(x), torch.tensor(z), chunk=128).numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_modal_samples_follow_algorithm_2():
    """The paper's training distribution (Sec. 2.4.2): nodal values in [0, X_A] with the minimum 0 and
    the maximum X_A exactly; X_A uniform on [0, A_sigma]; the low-frequency bias makes the highest
    modes ~e^-4 of the lowest on average; reproducible; the held-out stream differs."""
    from oracle import hdg
    xi, _ = hdg.lgl(6)
    b = W.modal_sample_batch(400)
    s = b.sigma_at(xi)
    assert s.shape == (400, 49)
    np.testing.assert_allclose(s.min(axis=1), 0.0, atol=1e-15)
    np.testing.assert_allclose(s.max(axis=1), b.amplitude, rtol=1e-14)
    assert b.amplitude.min() >= 0 and b.amplitude.max() <= 10 and b.amplitude.mean() > 4
    ratio = np.abs(b.modal[:, 6, 6]).mean() / np.abs(b.modal[:, 0, 0]).mean()
    assert 0.5 * np.exp(-4) < ratio < 2 * np.exp(-4), ratio
    np.testing.assert_array_equal(W.modal_sample_batch(400).modal, b.modal)
    assert not np.allclose(W.modal_sample_batch(400, holdout=True).modal, b.modal)
