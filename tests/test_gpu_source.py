"""GPU parity of the volume-source terms and the radiance recovery (eqs. hdg_local_f2u_i2u and
hdg_local_f2o_i2o; Algorithm 1 step 4) against the FP64 oracle: the element-local source solution
f_u, its outflow trace and angular mean, the full A_i2u, and whole solves with a source."""

import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import hdg
from tests import _helpers as H

pytestmark = pytest.mark.gpu

MODES = [("fp64", 0, 1e-11), ("fp32ir", 2, 1e-10), ("tf32ir", 2, 1e-10)]


@pytest.mark.parametrize("mode,refine,tol", MODES)
@pytest.mark.parametrize("p,N,n", [(3, 8, 7), (6, 16, 5)])
def test_source_terms_and_radiance_operator_match_oracle(lib, mode, refine, tol, p, N, n):
    import torch
    kappa, omega, h = H.random_elements(n, p, seed=500 + p)
    r = np.random.default_rng(600 + p)
    src = r.uniform(0.0, 2.0, (n, N, (p + 1) ** 2))
    ctx = lib.Context(p, N, 0.85, lib.ANG_FV0)
    m = {"fp64": lib.LOCAL_FP64, "fp32ir": lib.LOCAL_FP32_IR, "tf32ir": lib.LOCAL_TF32_IR}[mode]
    dev = lambda a: torch.tensor(a, device="cuda")
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
    rad = torch.empty(n, ctx.nu, ctx.nin, dtype=torch.float64, device="cuda")
    f2o = torch.empty(n, ctx.nin, dtype=torch.float64, device="cuda")
    f2m = torch.empty(n, ctx.nm, dtype=torch.float64, device="cuda")
    f2u = torch.empty(n, ctx.nu, dtype=torch.float64, device="cuda")
    st = ctx.elrt_build_local_ex(dev(kappa), dev(omega), h, i2o, i2m, mode=m, refine_steps=refine, source=dev(src),
                                 f2o=f2o, f2m=f2m, f2u=f2u, in2rad=rad)
    assert st.n_flagged == 0
    d = hdg.Disc(p, N, 0.85)
    for e in range(n):
        kh = kappa[e] * h / 2
        a, mm, X = d.local_operators(kh, omega[e])
        fo, fm, fu = d.local_source(kh, omega[e], src[e] * h / 2)
        np.testing.assert_allclose(i2o[e].cpu().numpy(), a, atol=tol)
        np.testing.assert_allclose(i2m[e].cpu().numpy(), mm, atol=tol)
        np.testing.assert_allclose(rad[e].cpu().numpy(), X, atol=tol)
        scale = np.abs(fu).max()
        np.testing.assert_allclose(f2u[e].cpu().numpy(), fu, atol=tol * scale)
        np.testing.assert_allclose(f2o[e].cpu().numpy(), fo, atol=tol * scale)
        np.testing.assert_allclose(f2m[e].cpu().numpy(), fm, atol=tol * scale)
    ctx.close()


def _source_problem(nx, nz, p, N, kind):
    prob = H.small_cloud(nx, nz, p, N)
    if kind == "emission":
        src = W.IsotropicEmission(prob.kappa, 0.99, 1.0, 0.6, nz * prob.h, N)
    else:
        src = W.BeamLikeSource(3.0, (0.4 * nx * prob.h, 0.6 * nz * prob.h), 0.3 * nx * prob.h, 1.0, N)
    return dataclasses.replace(prob, source=src)


@pytest.mark.parametrize("p,N,nx,nz,kind,mode", [(3, 8, 4, 3, "beamlike", "tf32ir"), (6, 16, 4, 4, "emission", "tf32ir"),
                                                  (4, 8, 5, 3, "emission", "fp32ir")])
def test_solve_with_source_and_radiance_match_oracle(lib, p, N, nx, nz, kind, mode):
    """Algorithm 1 with a volume source: FP32 operators with the source column refined alongside,
    GMRES on sum_K (R^o - A_i2o) u^ = sum_K f^_u, mean intensity with f_m, radiance u = A_i2u u^_in
    + f_u; relative L2 against the oracle's solve within 1e-6 (the FP32 operators' rounding)."""
    import torch
    prob = _source_problem(nx, nz, p, N, kind)
    ref = hdg.solve_problem(prob, rtol=1e-13, radiance=True)
    ctx = lib.Context(p, N, prob.hg_g, lib.ANG_FV0)
    E = prob.n_elems
    dev = lambda a: torch.tensor(a, device="cuda")
    kap, om, g = dev(H.lib_kappa(prob)), dev(prob.omega), dev(prob.inflow)
    src = dev(H.lib_source(prob))
    i2o = torch.empty(E, ctx.nin, ctx.nin, dtype=torch.float32, device="cuda")
    i2m = torch.empty(E, ctx.nm, ctx.nin, dtype=torch.float32, device="cuda")
    rad = torch.empty(E, ctx.nu, ctx.nin, dtype=torch.float32, device="cuda")
    f2o = torch.empty(E, ctx.nin, dtype=torch.float64, device="cuda")
    f2m = torch.empty(E, ctx.nm, dtype=torch.float64, device="cuda")
    f2u = torch.empty(E, ctx.nu, dtype=torch.float64, device="cuda")
    m = lib.LOCAL_TF32_IR if mode == "tf32ir" else lib.LOCAL_FP32_IR
    ctx.elrt_build_local_ex(kap, om, prob.h, i2o, i2m, mode=m, refine_steps=2, source=src, f2o=f2o, f2m=f2m, f2u=f2u,
                            in2rad=rad)
    sk = torch.empty(E * ctx.nin, dtype=torch.float64, device="cuda")
    st = ctx.elrt_solve_global_source(nx, nz, i2o, g, f2o, sk, rtol=1e-12, restart=30, max_iter=20000)
    um = torch.empty(E, ctx.nm, dtype=torch.float64, device="cuda")
    ctx.elrt_recover_mean_source(nx, nz, i2m, f2m, sk, g, um)
    u = torch.empty(E, ctx.nu, dtype=torch.float64, device="cuda")
    ctx.elrt_recover_radiance(nx, nz, rad, f2u, sk, g, u)
    torch.cuda.synchronize()
    err_m = hdg.rel_l2(um.cpu().numpy(), ref["u_mean"], ref["disc"])
    got_u = u.cpu().numpy().reshape(E, N, ctx.nm)
    err_u = np.linalg.norm(got_u - ref["radiance"]) / np.linalg.norm(ref["radiance"])
    print(f"source solve p={p} N={N} {kind}: GMRES {st.iterations} it, mean rel L2 {err_m:.1e}, radiance {err_u:.1e}")
    assert st.converged
    assert err_m < 1e-6 and err_u < 1e-6, (err_m, err_u)
    # the source matters: dropping it changes the answer at O(1)
    without = hdg.solve_problem(dataclasses.replace(prob, source=None), rtol=1e-13)
    assert hdg.rel_l2(without["u_mean"], ref["u_mean"], ref["disc"]) > 1e-2
    ctx.close()


def test_radiance_without_source_matches_oracle(lib):
    """The radiance of the benchmark-like cloud (no source): u = A_i2u u^_in from the FP32 operators."""
    import torch
    prob = H.small_cloud(4, 4, 4, 8)
    ref = hdg.solve_problem(prob, rtol=1e-13, radiance=True)
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, lib.ANG_FV0)
    E = prob.n_elems
    dev = lambda a: torch.tensor(a, device="cuda")
    kap, om, g = dev(H.lib_kappa(prob)), dev(prob.omega), dev(prob.inflow)
    i2o = torch.empty(E, ctx.nin, ctx.nin, dtype=torch.float32, device="cuda")
    i2m = torch.empty(E, ctx.nm, ctx.nin, dtype=torch.float32, device="cuda")
    rad = torch.empty(E, ctx.nu, ctx.nin, dtype=torch.float32, device="cuda")
    ctx.elrt_build_local_ex(kap, om, prob.h, i2o, i2m, mode=lib.LOCAL_TF32_IR, refine_steps=1, in2rad=rad)
    sk = torch.empty(E * ctx.nin, dtype=torch.float64, device="cuda")
    ctx.elrt_solve_global(prob.nx, prob.nz, i2o, g, sk, rtol=1e-12)
    u = torch.empty(E, ctx.nu, dtype=torch.float64, device="cuda")
    ctx.elrt_recover_radiance(prob.nx, prob.nz, rad, None, sk, g, u)
    torch.cuda.synchronize()
    got = u.cpu().numpy().reshape(E, prob.n_angles, ctx.nm)
    err = np.linalg.norm(got - ref["radiance"]) / np.linalg.norm(ref["radiance"])
    assert err < 1e-6, err
    np.testing.assert_allclose(got.mean(axis=1), ref["u_mean"], atol=1e-6 * np.abs(ref["u_mean"]).max())
    ctx.close()
