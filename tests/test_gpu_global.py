"""GPU parity of the global stage (skeleton operator, GMRES, mean recovery) and of the whole
classical pipeline (Algorithm 1) against the FP64 oracle."""

import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import hdg
from tests import _helpers as H

pytestmark = pytest.mark.gpu


def _oracle_ops(problem):
    d = hdg.Disc(problem.p, problem.n_angles, problem.hg_g, problem.angular)
    m = hdg.Mesh(problem.nx, problem.nz, problem.h)
    A_i2o, A_i2m = hdg.build_local(d, hdg.nodal_kappa_hat(problem, d, m), problem.omega)
    return d, m, A_i2o, A_i2m


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_skeleton_operator_matches_oracle(lib, dtype):
    import torch
    prob = H.small_cloud(5, 3, 3, 8, random_inflow=True)
    d, m, A_i2o, _ = _oracle_ops(prob)
    if dtype == "f32":
        A_i2o = A_i2o.astype(np.float32).astype(np.float64)    # both sides see the same rounded operator
    x = np.random.default_rng(1).normal(size=m.n_elems * d.n_out)
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, 0)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    At = torch.tensor(A_i2o, device="cuda", dtype=tdt)
    y = torch.empty(x.size, dtype=torch.float64, device="cuda")
    ctx.elrt_global_apply(prob.nx, prob.nz, At, torch.tensor(x, device="cuda"), y)
    np.testing.assert_allclose(y.cpu().numpy(), hdg.global_apply(m, d, A_i2o, x), atol=1e-13)


def test_gmres_matches_dense_solve(lib):
    import torch
    prob = H.small_cloud(4, 4, 3, 8, random_inflow=True)
    d, m, A_i2o, A_i2m = _oracle_ops(prob)
    ref = hdg.solve_problem(prob, dense=True, ops=(A_i2o, A_i2m))
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, 0)
    g = torch.tensor(prob.inflow, device="cuda")
    x = torch.empty(m.n_elems * d.n_out, dtype=torch.float64, device="cuda")
    st = ctx.elrt_solve_global(prob.nx, prob.nz, torch.tensor(A_i2o, device="cuda"), g, x, rtol=1e-13, restart=20)
    assert st.converged == 1 and st.rel_residual <= 1e-13 and st.restarts >= 1
    np.testing.assert_allclose(x.cpu().numpy(), ref["x"], atol=1e-11 * np.abs(ref["x"]).max())
    mean = torch.empty(m.n_elems, d.nm, dtype=torch.float64, device="cuda")
    ctx.elrt_recover_mean(prob.nx, prob.nz, torch.tensor(A_i2m, device="cuda"), x, g, mean)
    np.testing.assert_allclose(mean.cpu().numpy(), ref["u_mean"], atol=1e-11 * np.abs(ref["u_mean"]).max())


def test_unit_square_end_to_end_fp64(lib):
    """Unit square, 4 x 4 elements, p = 4, N = 8, kappa = 1, no scattering, unit downward inflow on
    top: identical to the oracle; both sit at the same distance from the exact exp(-kappa s) solution."""
    prob = W.problem_unit_square()
    out = H.gpu_pipeline(prob, lib.LOCAL_FP64, lib.F64, rtol=1e-13)
    ref = hdg.solve_problem(prob, dense=True)
    d, m = ref["disc"], ref["mesh"]
    assert hdg.rel_l2(out["u_mean"], ref["u_mean"], d) < 1e-12
    exact = hdg.exact_unit_square_mean(prob, d, m, 1.0)
    e_gpu, e_orc = hdg.rel_l2(out["u_mean"], exact, d), hdg.rel_l2(ref["u_mean"], exact, d)
    assert abs(e_gpu - e_orc) < 1e-10 and e_orc < 0.1


def test_exact_transport_solution(lib):
    """Constant kappa, no scattering, inflow = exp(-kappa sbar.x/|sbar|^2): spectral accuracy at p = 8."""
    prob = W.problem_unit_square(p=8, n_angles=8, n=2, kappa=2.0)
    d, m = hdg.Disc(8, 8, 0.0), hdg.Mesh(2, 2, 0.5)
    prob = dataclasses.replace(prob, inflow=hdg.exact_transport_inflow(d, m, 2.0))
    out = H.gpu_pipeline(prob, lib.LOCAL_FP32_IR, lib.F64, rtol=1e-13)
    assert hdg.rel_l2(out["u_mean"], hdg.exact_transport_mean(prob, d, m, 2.0), d) < 1e-9


@pytest.mark.parametrize("mode,dt,tol", [("fp64", "f64", 1e-11), ("fp32ir", "f64", 1e-10), ("fp32ir", "f32", 1e-6)])
def test_cloud_end_to_end(lib, mode, dt, tol):
    prob = H.small_cloud(8, 6, 6, 16)
    ref = hdg.solve_problem(prob, rtol=1e-13)
    out = H.gpu_pipeline(prob, lib.LOCAL_FP64 if mode == "fp64" else lib.LOCAL_FP32_IR,
                         lib.F64 if dt == "f64" else lib.F32, rtol=1e-12)
    assert hdg.rel_l2(out["u_mean"], ref["u_mean"], ref["disc"]) < tol


def test_do_mode_and_other_sizes(lib):
    prob = H.small_cloud(5, 4, 4, 12, angular="do", g=0.5, omega=0.9, random_inflow=True)
    ref = hdg.solve_problem(prob, rtol=1e-13)
    out = H.gpu_pipeline(prob, lib.LOCAL_FP32_IR, lib.F64, rtol=1e-12)
    assert hdg.rel_l2(out["u_mean"], ref["u_mean"], ref["disc"]) < 1e-10


def test_zero_inflow_gives_zero(lib):
    prob = H.small_cloud(3, 3, 2, 4)
    prob = dataclasses.replace(prob, inflow=np.zeros_like(prob.inflow))
    out = H.gpu_pipeline(prob, lib.LOCAL_FP64, lib.F64)
    assert not np.any(out["x"]) and not np.any(out["u_mean"])
    assert out["solve_stats"].converged == 1


def test_iteration_limit_reports_noconv(lib):
    import torch
    prob = H.small_cloud(6, 6, 3, 8)
    d, m, A_i2o, _ = _oracle_ops(prob)
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, 0)
    x = torch.empty(m.n_elems * d.n_out, dtype=torch.float64, device="cuda")
    st = ctx.elrt_solve_global(prob.nx, prob.nz, torch.tensor(A_i2o, device="cuda"),
                               torch.tensor(prob.inflow, device="cuda"), x, rtol=1e-14, max_iter=3, restart=2,
                               raise_on_noconv=False)
    assert st.converged == 0 and st.iterations == 3 and st.rel_residual > 1e-14
    with pytest.raises(lib.ElrtError) as ei:
        ctx.elrt_solve_global(prob.nx, prob.nz, torch.tensor(A_i2o, device="cuda"),
                              torch.tensor(prob.inflow, device="cuda"), x, rtol=1e-14, max_iter=3, restart=2)
    assert ei.value.status == 4


def test_flux_conservation_albedo_one(lib):
    """omega = 1: the net boundary flux of the library's solution vanishes (to the GMRES tolerance)."""
    prob = H.small_cloud(6, 4, 4, 8, omega=1.0, random_inflow=True)
    out = H.gpu_pipeline(prob, lib.LOCAL_FP32_IR, lib.F64, rtol=1e-13)
    d, m = hdg.Disc(4, 8, 0.85), hdg.Mesh(6, 4, prob.h)
    x = out["x"].reshape(m.n_elems, d.n_out)
    offs, _ = hdg.inflow_side_offsets(m, d)
    net, tot = 0.0, 0.0
    for e in range(m.n_elems):
        for F in range(4):
            if m.neighbour(e, F) >= 0:
                continue
            s0 = offs[F] + m.boundary_face(e, F) * d.n_face
            for mm in range(d.n1):
                for kk in range(4):
                    net += d.w[mm] * d.s_dot_n[F, d.out_cells[F][kk]] * x[e, F * d.n_face + mm * 4 + kk]
                    v = d.w[mm] * d.s_dot_n[F, d.in_cells[F][kk]] * prob.inflow[s0 + mm * 4 + kk]
                    net += v
                    tot += abs(v)
    assert abs(net) < 1e-11 * tot


@pytest.mark.parametrize("op", ["f16", "f32"])
@pytest.mark.parametrize("restart", [8, 31, 32, 50])
def test_fp32_gmres_paths_agree(lib, restart, op):
    """FP32 operators: restarts up to 31 run the four-launch Arnoldi step (last-block reductions,
    selective second Gram-Schmidt pass), larger ones the general Krylov kernels; with the Arnoldi
    steps on the FP16 copy of in2out or on in2out itself, all reach the oracle's mean intensity to
    the float-float level."""
    prob = H.small_cloud(8, 6, 4, 8)
    ref = hdg.solve_problem(prob, rtol=1e-13)
    out = H.gpu_pipeline(prob, lib.LOCAL_FP32_IR, lib.F32, rtol=1e-12, restart=restart,
                         krylov_op=lib.KRYLOV_F16 if op == "f16" else lib.KRYLOV_F32)
    assert out["solve_stats"].converged == 1 and out["solve_stats"].rel_residual <= 1e-12
    assert hdg.rel_l2(out["u_mean"], ref["u_mean"], ref["disc"]) < 1e-6


def _solve_f32(lib, prob, A32, op, rtol, restart=12):
    import torch
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, 0)
    ctx.elrt_set_krylov_op(op)
    x = torch.empty(prob.nx * prob.nz * ctx.nin, dtype=torch.float64, device="cuda")
    st = ctx.elrt_solve_global(prob.nx, prob.nz, torch.tensor(A32, device="cuda"),
                               torch.tensor(prob.inflow, device="cuda"), x, rtol=rtol, restart=restart)
    out = x.cpu().numpy()
    ctx.close()
    return out, st


def test_f16_arnoldi_refines_to_fp32_system(lib):
    """The FP16 copy only builds the Krylov basis: the restarts measure the residual with the FP32
    operator, so the iterate solves the FP32 system to rtol, as with FP32 Arnoldi steps.  Both are
    checked against a dense FP64 solve of the same (FP32-rounded) operator."""
    prob = H.small_cloud(6, 5, 4, 8, random_inflow=True)
    d, m, A_i2o, A_i2m = _oracle_ops(prob)
    A32 = A_i2o.astype(np.float32)
    ref = hdg.solve_problem(prob, dense=True, ops=(A32.astype(np.float64), A_i2m))
    x16, st16 = _solve_f32(lib, prob, A32, lib.KRYLOV_F16, 1e-11)
    x32, st32 = _solve_f32(lib, prob, A32, lib.KRYLOV_F32, 1e-11)
    for x, st in ((x16, st16), (x32, st32)):
        assert st.converged == 1 and st.rel_residual <= 1e-11
        np.testing.assert_allclose(x, ref["x"], atol=1e-9 * np.abs(ref["x"]).max())


def test_f16_copy_out_of_range_keeps_fp32(lib):
    """An in2out entry beyond the FP16 range (here 1e5 on a column that only ever multiplies zero
    boundary data) must not reach the Arnoldi steps: the FP16 copy would hold inf and inf * 0 = NaN.
    The solve detects the range and stays on the FP32 operator, giving the FP32-path result."""
    prob = H.small_cloud(4, 4, 3, 8, random_inflow=True)
    d, m, A_i2o, _ = _oracle_ops(prob)
    offs, _ = hdg.inflow_side_offsets(m, d)
    s0 = offs[0] + m.boundary_face(0, 0) * d.n_face     # element 0, bottom face: domain boundary
    inflow = prob.inflow.copy()
    inflow[s0:s0 + d.n_face] = 0.0
    prob = dataclasses.replace(prob, inflow=inflow)
    A32 = A_i2o.astype(np.float32)
    A32[0, 0, 0] = 1e5                                   # row 0, inflow column 0 (bottom face)
    x16, st16 = _solve_f32(lib, prob, A32, lib.KRYLOV_F16, 1e-11)
    x32, st32 = _solve_f32(lib, prob, A32, lib.KRYLOV_F32, 1e-11)
    assert np.all(np.isfinite(x16)) and st16.converged == 1
    np.testing.assert_allclose(x16, x32, atol=1e-9 * np.abs(x32).max())


@pytest.mark.parametrize("p,n_angles,nx,nz", [(1, 4, 9, 7), (4, 8, 8, 6), (7, 16, 3, 3), (8, 16, 3, 2)])
def test_f16_arnoldi_matvec_kernels(lib, p, n_angles, nx, nz):
    """The FP16 Arnoldi-step matvec runs on the tensor cores for 32 <= n_in <= 256 (128-row tiles of
    the flat operator crossing element boundaries: n_in = 80 gives tiles over 2-3 elements, n_in =
    256 the widest K) and on the CUDA cores otherwise (n_in = 16 and 288); every case reaches the
    dense FP64 solution of the same FP32 operator."""
    prob = H.small_cloud(nx, nz, p, n_angles, random_inflow=True)
    d, m, A_i2o, A_i2m = _oracle_ops(prob)
    A32 = A_i2o.astype(np.float32)
    ref = hdg.solve_problem(prob, dense=True, ops=(A32.astype(np.float64), A_i2m))
    x16, st16 = _solve_f32(lib, prob, A32, lib.KRYLOV_F16, 1e-11)
    assert st16.converged == 1 and st16.rel_residual <= 1e-11
    np.testing.assert_allclose(x16, ref["x"], atol=1e-9 * np.abs(ref["x"]).max())


def test_krylov_op_rejects_unknown_value(lib):
    ctx = lib.Context(3, 8, 0.0, 0)
    with pytest.raises(lib.ElrtError) as ei:
        ctx.elrt_set_krylov_op(7)
    assert ei.value.status == 1
    ctx.close()
