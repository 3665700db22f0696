"""GPU parity of the sweep preconditioner of the skeleton GMRES (upwind block Gauss-Seidel sweeps
of eq. hdg_global_mat from the four mesh corners; Sec. 2.3 lists sweeps among the solvers of
radiative transfer) against the oracle, and of the preconditioned solve against the oracle's
solution."""

import numpy as np
import pytest

from oracle import hdg
from tests import _helpers as H

pytestmark = pytest.mark.gpu


def _random_blocks(mesh, disc, faces=(0, 1, 2, 3), seed=0):
    rng = np.random.default_rng(seed)
    E, no, ni, nf = mesh.n_elems, disc.n_out, disc.n_in, disc.n_face
    A = rng.standard_normal((E, no, ni)) * (0.5 / np.sqrt(ni))
    for F in range(4):
        if F not in faces:
            A[:, :, F * nf:(F + 1) * nf] = 0.0
    return A.astype(np.float32)


def _apply(lib, disc, mesh, A32, r):
    import torch
    ctx = lib.Context(disc.p, disc.n_angles, disc.hg_g, 0)
    z = torch.zeros(r.size, dtype=torch.float32, device="cuda")
    ctx.elrt_apply_precond(mesh.nx, mesh.nz, torch.tensor(A32, device="cuda"), torch.tensor(r, device="cuda"), z)
    return z.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("nx,nz,p,N", [(6, 5, 3, 8), (1, 7, 2, 8), (9, 2, 2, 4), (13, 11, 4, 16)])
def test_apply_matches_oracle(lib, nx, nz, p, N):
    """M r on random blocks (non-square meshes, one-element-wide ones, element sizes with ragged
    row blocks) against the oracle's sequential sweeps on the same FP32-rounded blocks."""
    disc, mesh = hdg.Disc(p, N, 0.5, "fv0"), hdg.Mesh(nx, nz, 1.0)
    A32 = _random_blocks(mesh, disc, seed=nx * 31 + nz)
    r = np.random.default_rng(nx + nz).standard_normal(mesh.n_elems * disc.n_out).astype(np.float32)
    ref = hdg.sweep_precond(mesh, disc, A32.astype(np.float64), r.astype(np.float64))
    np.testing.assert_allclose(_apply(lib, disc, mesh, A32, r), ref, rtol=0, atol=2e-5 * np.abs(ref).max())


@pytest.mark.parametrize("faces", [(0, 3), (0, 1)])
def test_apply_inverts_a_one_sided_operator(lib, faces):
    """Blocks that take interior inflow only through the bottom and left faces (or the bottom and
    right): (I - A_int) is block triangular in the first (second) sweep's order, and one application
    of the downwind-face sweeps is its exact inverse: the GPU result against a dense solve,
    independent of the oracle's sweep."""
    disc, mesh = hdg.Disc(3, 8, 0.5, "fv0"), hdg.Mesh(7, 6, 1.0)
    A32 = _random_blocks(mesh, disc, faces, seed=5)
    G = hdg.global_dense(mesh, disc, A32.astype(np.float64))
    r = np.random.default_rng(4).standard_normal(G.shape[0]).astype(np.float32)
    exact = np.linalg.solve(G, r.astype(np.float64))
    np.testing.assert_allclose(_apply(lib, disc, mesh, A32, r), exact, rtol=0, atol=2e-5 * np.abs(exact).max())


def test_preconditioned_solve_matches_oracle(lib):
    """A scattering cloud (12 x 10, p = 3, N = 8, omega = 0.99, g = 0.85): the preconditioned GMRES
    reaches the oracle's solution of the same FP32-rounded skeleton system, in at most a third of
    the Arnoldi steps of plain GMRES (66 against 15 measured), with and without CUDA-graph replay."""
    import torch
    prob = H.small_cloud(12, 10, 3, 8)
    d = hdg.Disc(prob.p, prob.n_angles, prob.hg_g, prob.angular)
    m = hdg.Mesh(prob.nx, prob.nz, prob.h)
    A_i2o, _ = hdg.build_local(d, hdg.nodal_kappa_hat(prob, d, m), prob.omega)
    A32 = A_i2o.astype(np.float32)
    A64 = A32.astype(np.float64)
    b = hdg.global_rhs(m, d, A64, np.asarray(prob.inflow))
    x_ref = np.linalg.solve(hdg.global_dense(m, d, A64), b)
    g = torch.tensor(prob.inflow, device="cuda")
    At = torch.tensor(A32, device="cuda")
    its = {}
    for pc, graphs in ((lib.PRECOND_NONE, 1), (lib.PRECOND_SWEEP, 1), (lib.PRECOND_SWEEP, 0)):
        ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, 0)
        ctx.elrt_set_precond(pc)
        ctx.elrt_set_graphs(graphs)
        x = torch.empty(m.n_elems * d.n_out, dtype=torch.float64, device="cuda")
        st = ctx.elrt_solve_global(prob.nx, prob.nz, At, g, x, rtol=1e-10, restart=12)
        assert st.converged == 1 and st.rel_residual <= 1e-10
        np.testing.assert_allclose(x.cpu().numpy(), x_ref, rtol=0, atol=1e-8 * np.abs(x_ref).max())
        its[(pc, graphs)] = st.iterations
    assert 3 * its[(lib.PRECOND_SWEEP, 1)] <= its[(lib.PRECOND_NONE, 1)], its
    assert its[(lib.PRECOND_SWEEP, 1)] == its[(lib.PRECOND_SWEEP, 0)], its


def test_bad_arguments(lib):
    import torch
    ctx = lib.Context(2, 8, 0.5, 0)
    with pytest.raises(lib.ElrtError):
        ctx.elrt_set_precond(2)
    A = torch.zeros(4, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    r = torch.zeros(4 * ctx.nin, dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        ctx.elrt_apply_precond(2, 2, A, r, r.clone())   # FP64 blocks
