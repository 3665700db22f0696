"""Pins of the oracle's sweep preconditioner (upwind block Gauss-Seidel on the skeleton system
of eq. hdg_global_mat; Sec. 2.3 names sweeps among the solvers of radiative transfer), CPU only.

Exactness where the mathematics fixes it: when every element takes its interior inflow only from
the neighbours one wavefront closer to a corner, (I - A_int) is block triangular in that corner's
order and one sweep from it that recomputes every outflow value is the exact inverse (checked
against a dense solve, which shares no code with the sweep); a mesh without interior faces makes M
the identity; and on the physical skeleton system right-preconditioned GMRES reaches the plain
solution in far fewer steps.  The library's form recomputes only each sweep's downwind faces:
it is pinned against the same sweeps written as a multiplicative Schwarz iteration with dense
block solves (no sweep loop), and by the one-sided operators it inverts exactly."""

import numpy as np
import pytest

import workloads as W
from oracle import hdg


def _random_blocks(mesh, disc, keep_faces, seed=0):
    """Random in2out blocks whose inflow from the faces not in keep_faces is cut off."""
    rng = np.random.default_rng(seed)
    E, no, ni, nf = mesh.n_elems, disc.n_out, disc.n_in, disc.n_face
    A = rng.standard_normal((E, no, ni)) * (0.5 / np.sqrt(ni))
    for F in range(4):
        if F not in keep_faces:
            A[:, :, F * nf:(F + 1) * nf] = 0.0
    return A


@pytest.mark.parametrize("corner,faces", [("BL", (0, 3)), ("TR", (1, 2)), ("BR", (0, 1)), ("TL", (2, 3))])
def test_one_sweep_inverts_a_one_sided_operator(corner, faces):
    """Inflow only through the faces that look towards the corner (BL: bottom and left): the
    operator is block triangular in that corner's wavefront order and one sweep solves it."""
    disc = hdg.Disc(2, 8, 0.5, "fv0")
    mesh = hdg.Mesh(4, 3, 1.0)
    A = _random_blocks(mesh, disc, faces, seed=len(corner) + faces[0])
    G = hdg.global_dense(mesh, disc, A)
    r = np.random.default_rng(7).standard_normal(G.shape[0])
    exact = np.linalg.solve(G, r)
    np.testing.assert_allclose(hdg.sweep_precond(mesh, disc, A, r, corners=(corner,), rows="all"), exact,
                               rtol=1e-12, atol=1e-12)
    # the further sweeps of the full preconditioner keep the exact solution (a fixed point)
    np.testing.assert_allclose(hdg.sweep_precond(mesh, disc, A, r, rows="all"), exact, rtol=1e-11, atol=1e-11)


def test_opposite_corner_does_not_invert_it():
    """The same one-sided operator swept from the opposite corner is not solved in one sweep: the
    order matters (a sweep that ignored it would pass the test above by accident)."""
    disc = hdg.Disc(2, 8, 0.5, "fv0")
    mesh = hdg.Mesh(4, 3, 1.0)
    A = _random_blocks(mesh, disc, (0, 3), seed=3)
    G = hdg.global_dense(mesh, disc, A)
    r = np.random.default_rng(8).standard_normal(G.shape[0])
    exact = np.linalg.solve(G, r)
    z = hdg.sweep_precond(mesh, disc, A, r, corners=("TR",), rows="all")
    assert np.linalg.norm(z - exact) > 1e-3 * np.linalg.norm(exact)


def test_single_element_is_identity():
    disc = hdg.Disc(2, 8, 0.5, "fv0")
    mesh = hdg.Mesh(1, 1, 1.0)
    A = _random_blocks(mesh, disc, (0, 1, 2, 3), seed=1)
    r = np.random.default_rng(2).standard_normal(disc.n_out)
    np.testing.assert_array_equal(hdg.sweep_precond(mesh, disc, A, r, rows="all"), r)
    np.testing.assert_array_equal(hdg.sweep_precond(mesh, disc, A, r), r)


def test_wavefront_orders():
    """Corner first, neighbours one wavefront apart, every element once."""
    mesh = hdg.Mesh(5, 3, 1.0)
    for corner, first in (("BL", 0), ("TR", 14), ("BR", 4), ("TL", 10)):
        order = hdg.sweep_order(mesh, corner)
        assert sorted(order.tolist()) == list(range(15)) and order[0] == first
        pos = np.empty(15, int)
        pos[order] = np.arange(15)
        ix, iz = np.arange(15) % 5, np.arange(15) // 5
        d = (ix if corner in ("BL", "TL") else 4 - ix) + (iz if corner in ("BL", "BR") else 2 - iz)
        for e in range(15):
            for F in range(4):
                nb = mesh.neighbour(e, F)
                if nb >= 0:
                    assert abs(d[nb] - d[e]) == 1 and (d[nb] < d[e]) == (pos[nb] < pos[e])


def test_preconditioned_gmres_on_the_skeleton_system():
    """The Gaussian-cloud slab (8 x 8, p = 3, N = 8): the same solution as plain GMRES(12) to the
    tolerance, in at most a third of the steps."""
    prob = W.problem_gaussian_slab(n=8, p=3, n_angles=8)
    disc = hdg.Disc(prob.p, prob.n_angles, prob.hg_g, "fv0")
    mesh = hdg.Mesh(prob.nx, prob.nz, prob.h)
    A, _ = hdg.build_local(disc, hdg.nodal_kappa_hat(prob, disc, mesh), np.asarray(prob.omega))
    b = hdg.global_rhs(mesh, disc, A, np.asarray(prob.inflow))
    apply = lambda x: hdg.global_apply(mesh, disc, A, x)
    x0, it0, rel0 = hdg.gmres(apply, b, rtol=1e-10, restart=12)
    for rows in ("all", "downwind"):
        x1, it1, rel1 = hdg.gmres_right(apply, lambda v: hdg.sweep_precond(mesh, disc, A, v, rows=rows), b, rtol=1e-10,
                                        restart=12)
        assert rel0 <= 1e-10 and rel1 <= 1e-10
        assert np.linalg.norm(b - apply(x1)) <= 1e-10 * np.linalg.norm(b) * 1.01
        np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-8 * np.abs(x0).max())
        assert 3 * it1 <= it0, (rows, it0, it1)


def _schwarz(mesh, disc, A, r):
    """The downwind-face sweeps as a multiplicative Schwarz iteration on G = I - A_int from z = 0:
    per corner, the rows S of every element's two downwind faces are solved for exactly, the
    others held: z_S += G_SS^{-1} (r - G z)_S, by a dense solve (no sweep loop, no gather)."""
    G = hdg.global_dense(mesh, disc, A)
    E, no, nf = mesh.n_elems, disc.n_out, disc.n_face
    z = np.zeros(G.shape[0])
    for corner in hdg.SWEEP_CORNERS:
        S = np.concatenate([e * no + F * nf + np.arange(nf) for e in range(E) for F in hdg.SWEEP_DOWNWIND[corner]])
        res = r - G @ z
        z[S] += np.linalg.solve(G[np.ix_(S, S)], res[S])
    return z


@pytest.mark.parametrize("nx,nz", [(4, 3), (1, 5), (3, 3)])
def test_downwind_sweeps_are_multiplicative_schwarz(nx, nz):
    disc = hdg.Disc(2, 8, 0.5, "fv0")
    mesh = hdg.Mesh(nx, nz, 1.0)
    A = _random_blocks(mesh, disc, (0, 1, 2, 3), seed=nx * 7 + nz)
    r = np.random.default_rng(nx + 10 * nz).standard_normal(mesh.n_elems * disc.n_out)
    np.testing.assert_allclose(hdg.sweep_precond(mesh, disc, A, r), _schwarz(mesh, disc, A, r), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("faces,exact", [((0, 3), True), ((0, 1), True), ((1, 2), False), ((2, 3), False)])
def test_downwind_sweeps_on_one_sided_operators(faces, exact):
    """Inflow only from below and from the left (or from below and the right): the bottom-left (the
    bottom-right) sweep, first (second) in turn, makes every value it recomputes exact and the later
    sweeps recompute the rest from exact inflow, so one application is the exact inverse.  Inflow
    only from above: the sweeps that recompute the top faces come before the ones that bring the
    inflow, so it is not."""
    disc = hdg.Disc(2, 8, 0.5, "fv0")
    mesh = hdg.Mesh(4, 3, 1.0)
    A = _random_blocks(mesh, disc, faces, seed=3)
    G = hdg.global_dense(mesh, disc, A)
    r = np.random.default_rng(7).standard_normal(G.shape[0])
    ref = np.linalg.solve(G, r)
    err = np.abs(hdg.sweep_precond(mesh, disc, A, r) - ref).max() / np.abs(ref).max()
    assert (err < 1e-12) == exact, (faces, err)
