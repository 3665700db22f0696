"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the fact it checks; together they are chosen so that a dropped term, a sign
error, a transposed operand or a wrong DOF map in the oracle fails at least one of them.
"""

import dataclasses
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import hdg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------- LGL
def test_lgl_closed_forms():
    """LGL nodes/weights for p = 1..4 in closed form (Abramowitz & Stegun 25.4.32)."""
    xi, w = hdg.lgl(1)
    np.testing.assert_allclose(xi, [-1, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1, 1], atol=1e-15)
    xi, w = hdg.lgl(2)
    np.testing.assert_allclose(xi, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    xi, w = hdg.lgl(3)
    r = 1 / math.sqrt(5)
    np.testing.assert_allclose(xi, [-1, -r, r, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    xi, w = hdg.lgl(4)
    r = math.sqrt(3 / 7)
    np.testing.assert_allclose(xi, [-1, -r, 0, r, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 11))
def test_lgl_exact_to_degree_2p_minus_1(p):
    xi, w = hdg.lgl(p)
    for q in range(2 * p):
        exact = 0.0 if q % 2 else 2.0 / (q + 1)
        assert abs(np.dot(w, xi ** q) - exact) < 1e-13


@pytest.mark.parametrize("p", range(1, 9))
def test_derivative_matrix_exact_on_polynomials(p):
    xi, _ = hdg.lgl(p)
    D = hdg.lagrange_derivative(xi)
    for q in range(p + 1):
        want = q * xi ** (q - 1) if q else np.zeros_like(xi)
        np.testing.assert_allclose(D @ xi ** q, want, atol=1e-11)


# --------------------------------------------------------------------------------------- phase
def _phase_by_fourier(n_angles, g, angular):
    """Independent route to W: Fourier coefficients of the HG kernel by an FFT on a fine grid,
    then the exact cell integrals of each Fourier mode (Delta sinc^2(m Delta/2) for fv0)."""
    M = 1 << 16
    t = 2 * math.pi * np.arange(M) / M
    c_m = np.fft.rfft(hdg.hg_unnormalised(t, g)).real / M       # (1/2pi) int p e^{-imt}
    c_m = c_m / (2 * math.pi * c_m[0]) * 1.0                     # normalise: 2pi c_0 = 1
    dth = 2 * math.pi / n_angles
    d = np.arange(n_angles)[:, None] - np.arange(n_angles)[None, :]
    m = np.arange(1, 4000)
    if angular == "fv0":
        fac = (np.sin(m * dth / 2) / (m * dth / 2)) ** 2
        W = dth * (c_m[0] + 2 * np.sum(c_m[1:4000, None, None] * fac[:, None, None]
                                       * np.cos(m[:, None, None] * d[None] * dth), axis=0))
    else:
        W = dth * (c_m[0] + 2 * np.sum(c_m[1:4000, None, None] * np.cos(m[:, None, None] * d[None] * dth), axis=0))
    return W / W.sum(axis=1, keepdims=True)


@pytest.mark.parametrize("angular", ["fv0", "do"])
@pytest.mark.parametrize("n_angles,g", [(8, 0.0), (16, 0.85), (28, 0.8), (16, 0.5)])
def test_phase_matrix(angular, n_angles, g):
    Wm = hdg.phase_matrix(n_angles, g, angular)
    np.testing.assert_allclose(Wm.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(Wm, Wm.T, atol=1e-14)                       # HG depends on cos only
    for s in range(n_angles):                                               # circulant
        np.testing.assert_allclose(np.roll(np.roll(Wm, s, 0), s, 1), Wm, atol=1e-14)
    if g == 0.0:
        np.testing.assert_allclose(Wm, 1.0 / n_angles, atol=1e-15)
    np.testing.assert_allclose(Wm, _phase_by_fourier(n_angles, g, angular), atol=1e-11)


def test_phase_quadrature_converged():
    a = hdg.phase_matrix(16, 0.85, "fv0", nq=64)
    b = hdg.phase_matrix(16, 0.85, "fv0", nq=128)
    np.testing.assert_allclose(a, b, atol=1e-14)


def test_fv0_directions_are_cell_means():
    """fv0 direction = sinc(dth/2) times the cell-centre direction (closed form of the cell mean)."""
    for N in (8, 16, 28):
        sx, sz = hdg.directions(N, "fv0")
        cx, cz = hdg.directions(N, "do")
        dth = 2 * math.pi / N
        f = math.sin(dth / 2) / (dth / 2)
        np.testing.assert_allclose(sx, f * cx, atol=1e-15)
        np.testing.assert_allclose(sz, f * cz, atol=1e-15)


# --------------------------------------------------------------------------------------- local
CASES = [(2, 4, "fv0"), (3, 8, "fv0"), (4, 8, "do"), (3, 12, "fv0"), (2, 16, "do")]


@pytest.mark.parametrize("p,N,angular", CASES)
def test_row_sums_are_one_at_albedo_one(p, N, angular):
    """Constant preservation: with omega = 1 a constant isotropic inflow c gives u = c exactly, so
    every row of A_i2o and A_i2m sums to 1 (SBP property of LGL collocation + rows of W sum to 1)."""
    rng = np.random.default_rng(1)
    d = hdg.Disc(p, N, 0.7, angular)
    kh = rng.uniform(0.0, 5.0, d.nm)
    A_i2o, A_i2m, _ = d.local_operators(kh, 1.0)
    np.testing.assert_allclose(A_i2o.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(A_i2m.sum(axis=1), 1.0, atol=1e-12)
    # with absorption (omega < 1) the mean intensity of a unit inflow drops below 1 on average
    # (single rows may overshoot: high-order DG has no maximum principle)
    A_i2o, A_i2m, _ = d.local_operators(kh, 0.8)
    assert np.mean(A_i2m.sum(axis=1)) < 0.99


@pytest.mark.parametrize("p,N,angular", CASES)
def test_energy_balance_identity(p, N, angular):
    rng = np.random.default_rng(2)
    d = hdg.Disc(p, N, 0.85, angular)
    kh = rng.uniform(0.0, 3.0, d.nm)
    A_i2o, A_i2m, _ = d.local_operators(kh, 0.9)
    assert np.max(np.abs(d.energy_defect(kh, 0.9, A_i2o, A_i2m))) < 1e-12
    # a wrong operator fails the same check
    assert np.max(np.abs(d.energy_defect(kh, 0.9, A_i2o * 1.001, A_i2m))) > 1e-4


def test_local_solve_residual():
    rng = np.random.default_rng(3)
    d = hdg.Disc(4, 8, 0.85)
    kh = rng.uniform(0.0, 10.0, d.nm)
    A, Bh = d.local_system(kh, 0.95)
    _, _, X = d.local_operators(kh, 0.95)
    assert np.linalg.norm(A @ X + Bh) / np.linalg.norm(Bh) < 1e-13


def test_no_scattering_decouples_angles():
    """omega = 0: A is block diagonal per angular cell, so in2out never mixes cells."""
    d = hdg.Disc(3, 8, 0.85)
    A, _ = d.local_system(np.full(d.nm, 1.5), 0.0)
    for k in range(8):
        for l in range(8):
            if k != l:
                assert not np.any(A[k * d.nm:(k + 1) * d.nm, l * d.nm:(l + 1) * d.nm])


# --------------------------------------------------------------------------------------- global
def _tiny(p, N, angular, nx=3, nz=2, g=0.5, omega=0.9):
    prob = W.problem_gaussian_slab(n=nx, p=p, n_angles=N)
    rng = np.random.default_rng(4)
    cloud = W.GaussianClouds(0.3, np.array([4.0]), np.array([[1.0 * nx * 10 / nx / 2, 4.0]]), np.array([2.0]))
    offs, total = W.inflow_layout(nx, nz, p, N)
    return dataclasses.replace(prob, name="tiny", nz=nz, h=10.0 / nx, hg_g=g, omega=np.full(nx * nz, omega),
                               kappa=cloud, inflow=rng.uniform(0.0, 1.0, total), angular=angular)


@pytest.mark.parametrize("p,N,angular", [(2, 4, "fv0"), (3, 8, "fv0"), (2, 8, "do"), (3, 4, "do")])
def test_hybridised_equals_direct_dg(p, N, angular):
    prob = _tiny(p, N, angular)
    res = hdg.solve_problem(prob, dense=True)
    um = hdg.dg_direct(prob)
    assert np.max(np.abs(res["u_mean"] - um)) <= 1e-12 * np.max(np.abs(um))


def test_gmres_equals_dense():
    prob = _tiny(3, 8, "fv0", nx=4, nz=3, omega=0.99, g=0.85)
    a = hdg.solve_problem(prob, dense=True)
    b = hdg.solve_problem(prob, dense=False, rtol=1e-13)
    assert b["iterations"] > 0
    assert np.max(np.abs(a["x"] - b["x"])) <= 1e-11 * np.max(np.abs(a["x"]))


def test_exact_transport_solution_spectral_convergence():
    """No scattering, constant kappa, inflow = the exact solution exp(-kappa sbar.x/|sbar|^2):
    the error falls exponentially in p (Sec. 3.3: spectral accuracy of higher p)."""
    errs = []
    for p in range(2, 9):
        prob = W.problem_unit_square(p=p, n_angles=8, n=2, kappa=2.0)
        d, m = hdg.Disc(p, 8, 0.0), hdg.Mesh(2, 2, 0.5)
        prob = dataclasses.replace(prob, inflow=hdg.exact_transport_inflow(d, m, 2.0))
        res = hdg.solve_problem(prob, dense=True)
        errs.append(hdg.rel_l2(res["u_mean"], hdg.exact_transport_mean(prob, d, m, 2.0), d))
    assert all(b < a / 10 for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-9


def test_exact_transport_do_mode():
    prob = W.problem_unit_square(p=7, n_angles=12, n=3, kappa=1.0, angular="do")
    d, m = hdg.Disc(7, 12, 0.0, "do"), hdg.Mesh(3, 3, 1 / 3)
    prob = dataclasses.replace(prob, inflow=hdg.exact_transport_inflow(d, m, 1.0))
    res = hdg.solve_problem(prob, dense=False, rtol=1e-13)
    assert hdg.rel_l2(res["u_mean"], hdg.exact_transport_mean(prob, d, m, 1.0), d) < 1e-9


def _boundary_flux(prob, res):
    """Net outflow minus inflow through the domain boundary (reference units of one element)."""
    d, m = res["disc"], res["mesh"]
    x = res["x"].reshape(m.n_elems, d.n_out)
    offs, _ = hdg.inflow_side_offsets(m, d)
    half = d.n_angles // 2
    net = 0.0
    for e in range(m.n_elems):
        for F in range(4):
            if m.neighbour(e, F) >= 0:
                continue
            s0 = offs[F] + m.boundary_face(e, F) * d.n_face
            for mm in range(d.n1):
                for kk in range(half):
                    ko, ki = d.out_cells[F][kk], d.in_cells[F][kk]
                    net += d.w[mm] * d.s_dot_n[F, ko] * x[e, F * d.n_face + mm * half + kk]
                    net += d.w[mm] * d.s_dot_n[F, ki] * prob.inflow[s0 + mm * half + kk]
    return net


def test_flux_conservation():
    """omega = 1: what enters the domain leaves it; omega < 1: the deficit is the absorption
    N sum_K sum_i w_i kappa_hat_i (1 - omega) u^m_i."""
    prob = _tiny(3, 8, "fv0", nx=4, nz=3, omega=1.0, g=0.85)
    res = hdg.solve_problem(prob, dense=True)
    assert abs(_boundary_flux(prob, res)) < 1e-12 * np.abs(prob.inflow).sum()
    prob = _tiny(3, 8, "fv0", nx=4, nz=3, omega=0.8, g=0.85)
    res = hdg.solve_problem(prob, dense=True)
    d = res["disc"]
    absorb = d.n_angles * np.sum(d.w2[None, :] * res["kappa_hat"] * 0.2 * res["u_mean"])
    assert absorb > 0
    assert abs(_boundary_flux(prob, res) + absorb) < 1e-11 * absorb


# --------------------------------------------------------------------------------------- sizes
def test_sizes_match_paper_tables():
    gold = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    p, N = gold["p"], gold["n_angles"]
    for lvl, n_el, dofs in gold["dg_dofs_by_level"]:
        nx, nz = (6, 4) if lvl == 0 else (3 * (lvl + 2), 2 * (lvl + 2))
        assert nx * nz == n_el
        assert n_el * (p + 1) ** 2 * N == dofs
    d = hdg.Disc(p, N, 0.8)
    assert d.n_out * (d.n_in + d.nm) == gold["n_out_network"]


def test_inflow_layout_agrees_with_workloads():
    """The boundary-data layout of the workloads module and the oracle's face/cell classification agree."""
    from workloads.fields import _entering_cells
    for N in (4, 8, 16, 28):
        d = hdg.Disc(2, N, 0.0)
        for F in range(4):
            assert d.in_cells[F] == _entering_cells(F, N)
        offs, total = hdg.inflow_side_offsets(hdg.Mesh(5, 3, 1.0), d)
        woffs, wtotal = W.inflow_layout(5, 3, 2, N)
        assert list(offs) == woffs and total == wtotal


def test_unit_square_exact_solution_by_ray_marching():
    """Pin P3 by brute force: march back from every node along -sbar_k in small steps until the ray
    leaves the unit square; the exact angle-discrete solution is exp(-kappa t) if it leaves through
    the top (unit inflow there) and 0 otherwise.  Independent of the closed-form path lengths."""
    prob = W.problem_unit_square(p=2, n_angles=8, n=3, kappa=1.3)
    d = hdg.Disc(prob.p, prob.n_angles, 0.0, prob.angular)
    mesh = hdg.Mesh(prob.nx, prob.nz, prob.h)
    x, z = mesh.node_coords(d)
    ex = hdg.exact_unit_square_mean(prob, d, mesh, 1.3)
    dt = 2e-4
    total = np.zeros(x.shape)
    for k in range(d.n_angles):
        if d.sz[k] >= 0:
            continue                          # upward cells see zero inflow through the bottom
        px, pz = x.copy(), z.copy()
        t = np.zeros(x.shape)
        inside = np.ones(x.shape, bool)
        for _ in range(int(3.0 / dt)):
            if not inside.any():
                break
            px = np.where(inside, px - dt * d.sx[k], px)
            pz = np.where(inside, pz - dt * d.sz[k], pz)
            t = np.where(inside, t + dt, t)
            inside = (px >= 0) & (px <= 1) & (pz <= 1)
        top = pz > 1.0
        total += np.where(top, np.exp(-1.3 * t), 0.0)
    brute = total / d.n_angles
    # the march overshoots by at most one step; nodes within a step of a shadow line can flip
    close = np.abs(brute - ex) < 3 * dt
    assert close.mean() > 0.97, close.mean()
    np.testing.assert_allclose(brute[close], ex[close], atol=3 * dt)


def test_unit_square_discrete_solution_converges_to_exact():
    """The hybridised solution approaches the closed form under mesh refinement (reading A11: the
    inflow is discontinuous along the corner characteristics, so only about O(h^1/2) in L2)."""
    errs = []
    for n in (4, 8, 16):
        prob = W.problem_unit_square(p=2, n_angles=8, n=n)
        ref = hdg.solve_problem(prob, rtol=1e-12)
        ex = hdg.exact_unit_square_mean(prob, ref["disc"], ref["mesh"], 1.0)
        errs.append(hdg.rel_l2(ref["u_mean"], ex, ref["disc"]))
    assert errs[0] < 0.15 and errs[1] < errs[0] / 1.2 and errs[2] < errs[1] / 1.2, errs


def test_golden_headline_field_is_the_recorded_oracle_output():
    """The stored whole-field expectation of the benchmark slab is the file its generator recorded
    (SHA-256), finite, of the documented shape, from a GMRES solve converged to 1e-12."""
    import hashlib
    path = os.path.join(GOLDEN, "gaussian_slab_64x64_mean.npy")
    meta = json.load(open(os.path.join(GOLDEN, "gaussian_slab_64x64_mean.json")))
    assert hashlib.sha256(open(path, "rb").read()).hexdigest() == meta["sha256"]
    u = np.load(path)
    assert u.shape == (4096, 49) and np.all(np.isfinite(u)) and meta["rel_residual"] < 1e-11
    assert u.max() > 0.1                     # the beam enters: not a zero field


# ---------------------------------------------------------------------------------- volume source
def _with_source(prob, kind):
    if kind == "emission":
        src = W.IsotropicEmission(prob.kappa, float(prob.omega[0]), 1.0, 0.6, prob.nz * prob.h, prob.n_angles)
    else:
        src = W.BeamLikeSource(3.0, (0.4 * prob.nx * prob.h, 0.6 * prob.nz * prob.h), 0.3 * prob.nx * prob.h, 1.0,
                               prob.n_angles)
    return dataclasses.replace(prob, source=src)


@pytest.mark.parametrize("p,N,nx,nz,kind", [(2, 4, 2, 2, "emission"), (3, 8, 3, 2, "beamlike"), (2, 8, 2, 3, "beamlike")])
def test_source_hybridised_equals_direct_dg(p, N, nx, nz, kind):
    """With a volume source the hybridised solve (local source terms f^_u, f_u in the global
    right-hand side and the recovery) reproduces the direct upwind-DG solution: mean intensity and
    radiance, to round-off."""
    from tests import _helpers as H
    prob = _with_source(H.small_cloud(nx, nz, p, N, random_inflow=True), kind)
    ref = hdg.solve_problem(prob, dense=True, radiance=True)
    u_dg = hdg.dg_direct_radiance(prob)
    np.testing.assert_allclose(ref["radiance"], u_dg, atol=1e-12 * np.abs(u_dg).max())
    np.testing.assert_allclose(ref["u_mean"], u_dg.mean(axis=1), atol=1e-12 * np.abs(u_dg).max())
    assert np.abs(ref["f2o"]).max() > 1e-3                 # the source is not negligible


def _manufactured(p, n_angles, n=2, kappa=1.3, omega=0.7, g=0.5):
    """A smooth exact radiance u_k(x, z) per angular cell and the source that makes it the solution
    of the angle-discrete equation sbar_k . grad u_k + kappa u_k - omega kappa sum_l W_kl u_l = f_k,
    with inflow data taken from u_k on the boundary of the unit square (n x n elements)."""
    d = hdg.Disc(p, n_angles, g)
    th = (np.arange(n_angles) + 0.5) * 2 * math.pi / n_angles
    amp = 1.0 + 0.5 * np.sin(th + 0.3)                       # angular profile of u

    def u(x, z):                                              # [..., N]
        x = np.asarray(x, dtype=np.float64)[..., None]
        z = np.asarray(z, dtype=np.float64)[..., None]
        return amp * np.exp(0.4 * x - 0.3 * z) * (1.0 + 0.2 * np.sin(2.0 * x + z))

    def grad(x, z):
        x = np.asarray(x, dtype=np.float64)[..., None]
        z = np.asarray(z, dtype=np.float64)[..., None]
        e = np.exp(0.4 * x - 0.3 * z)
        s = 1.0 + 0.2 * np.sin(2.0 * x + z)
        c = 0.2 * np.cos(2.0 * x + z)
        return amp * e * (0.4 * s + 2.0 * c), amp * e * (-0.3 * s + c)

    def f(x, z):
        gx, gz = grad(x, z)
        uu = u(x, z)
        return d.sx * gx + d.sz * gz + kappa * uu - omega * kappa * uu @ d.W.T

    offs, total = W.inflow_layout(n, n, p, n_angles)
    gin = np.zeros(total)
    pos = (d.xi + 1.0) * 0.5 / n
    for F in range(4):
        for fa in range(n):
            for m in range(p + 1):
                px, pz = [(fa / n + pos[m], 0.0), (1.0, fa / n + pos[m]), (fa / n + pos[m], 1.0), (0.0, fa / n + pos[m])][F]
                for kk, k in enumerate(d.in_cells[F]):
                    gin[offs[F] + (fa * (p + 1) + m) * (n_angles // 2) + kk] = u(px, pz)[k]
    prob = W.Problem("manufactured", n, n, 1.0 / n, p, n_angles, g, np.full(n * n, omega),
                     lambda x, z: np.full(np.broadcast(np.asarray(x), np.asarray(z)).shape, kappa), gin, "fv0", f)
    return prob, u


def test_manufactured_solution_with_source_converges_spectrally():
    """Pin of the source terms (eqs. hdg_local_f2u_i2u, hdg_local_f2o_i2o and the recovery): for a
    smooth manufactured radiance with scattering the hybridised solution converges exponentially in
    p; a dropped, mis-scaled or sign-flipped source term stalls it at O(1)."""
    errs = []
    for p in range(2, 8):
        prob, u = _manufactured(p, 8)
        ref = hdg.solve_problem(prob, dense=True, radiance=True)
        x, z = ref["mesh"].node_coords(ref["disc"])
        exact = np.transpose(u(x, z), (0, 2, 1))              # [E, N, nm]
        errs.append(np.abs(ref["radiance"] - exact).max() / np.abs(exact).max())
        np.testing.assert_allclose(ref["u_mean"], exact.mean(axis=1), atol=2 * errs[-1] * np.abs(exact).max())
    assert errs[-1] < 1e-7, errs
    assert all(b < a / 4 for a, b in zip(errs, errs[1:])), errs
