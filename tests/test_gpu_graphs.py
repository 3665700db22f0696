"""CUDA-graph replay of the GMRES restart cycles gives the results of plain launches: the same
kernels in the same order, so the same iterations, residual and solution.  The launch count counts
every kernel of every replayed cycle, including the last cycle's, which the convergence test on the
device turns into no-ops (plain launches stop on the host before them)."""

import numpy as np
import pytest

from tests import _helpers as H

pytestmark = pytest.mark.gpu


def _solve(lib, prob, dtype, graphs, rtol=1e-9, max_iter=20000, restart=12, precond=None):
    import torch
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, lib.ANG_FV0)
    ctx.elrt_set_graphs(graphs)
    if precond is not None:
        ctx.elrt_set_precond(precond)
    E = prob.n_elems
    kap = torch.tensor(H.lib_kappa(prob), device="cuda")
    om = torch.tensor(prob.omega, device="cuda")
    g = torch.tensor(prob.inflow, device="cuda")
    dt = torch.float32 if dtype == "f32" else torch.float64
    a = torch.empty(E, ctx.nin, ctx.nin, dtype=dt, device="cuda")
    m = torch.empty(E, ctx.nm, ctx.nin, dtype=dt, device="cuda")
    ctx.elrt_build_local(kap, om, prob.h, a, m, mode=lib.LOCAL_FP32_IR, refine_steps=2)
    sk = torch.empty(E * ctx.nin, dtype=torch.float64, device="cuda")
    ctx.elrt_profile_reset()
    st = ctx.elrt_solve_global(prob.nx, prob.nz, a, g, sk, rtol=rtol, restart=restart, max_iter=max_iter,
                               raise_on_noconv=False)
    launches = ctx.elrt_launch_count()
    out = (st.iterations, st.restarts, st.converged, st.rel_residual, sk.cpu().numpy(), launches)
    ctx.close()
    return out


@pytest.mark.parametrize("dtype,nx,p,N", [("f32", 12, 4, 8), ("f64", 6, 3, 8), ("f32", 9, 6, 16)])
def test_graph_replay_equals_plain_launches(lib, dtype, nx, p, N):
    prob = H.small_cloud(nx, nx, p, N)
    g = _solve(lib, prob, dtype, True)
    n = _solve(lib, prob, dtype, False)
    assert g[0] == n[0] and g[1] == n[1] and g[2] == n[2] == 1, (g[:3], n[:3])
    assert g[3] == n[3]
    assert np.array_equal(g[4], n[4])
    assert g[5] >= n[5], (g[5], n[5])          # every replayed kernel counted


def test_graph_replay_iteration_limit(lib):
    """max_iter not a multiple of the restart length: full cycles from the graph, the last partial
    cycle and the final residual check from plain launches; ENOCONV with the same state (plain
    GMRES, which does not reach the unreachable tolerance before the limit)."""
    prob = H.small_cloud(10, 10, 4, 8)
    g = _solve(lib, prob, "f32", True, rtol=1e-14, max_iter=29, precond=lib.PRECOND_NONE)
    n = _solve(lib, prob, "f32", False, rtol=1e-14, max_iter=29, precond=lib.PRECOND_NONE)
    assert g[0] == n[0] == 29 and g[2] == n[2] == 0
    assert g[3] == n[3] and np.array_equal(g[4], n[4])
