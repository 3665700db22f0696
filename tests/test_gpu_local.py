"""GPU parity of the local stage (assembly, LU, refinement, restriction) against the FP64 oracle."""

import numpy as np
import pytest

from oracle import hdg
from tests import _helpers as H

pytestmark = pytest.mark.gpu

CASES = [  # (p, N, angular, n_elems): ragged panels (nu % NB != 0) and several tiles
    (2, 4, "fv0", 7),
    (4, 8, "fv0", 16),
    (3, 12, "do", 5),
    (6, 16, "fv0", 9),
    (8, 16, "fv0", 3),
]


def _ctx(E, p, N, g, ang):
    return E.Context(p, N, g, 0 if ang == "fv0" else 1)


def _oracle_ops(p, N, g, ang, kappa, omega, h):
    d = hdg.Disc(p, N, g, ang)
    return d, hdg.build_local(d, kappa * h / 2, omega)


@pytest.mark.parametrize("p,N,ang,n", CASES[:4])
def test_assembly_matches_oracle(lib, p, N, ang, n):
    import torch
    kappa, omega, h = H.random_elements(n, p, seed=p * 100 + N)
    ctx = _ctx(lib, p, N, 0.85, ang)
    A = torch.empty(n, ctx.nu, ctx.nu, dtype=torch.float64, device="cuda")
    R = torch.empty(n, ctx.nu, ctx.nin, dtype=torch.float64, device="cuda")
    ctx.elrt_assemble(torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda"), h, A, R)
    A, R = A.cpu().numpy(), R.cpu().numpy()
    d = hdg.Disc(p, N, 0.85, ang)
    for e in range(n):
        Ao, Bo = d.local_system(kappa[e] * h / 2, omega[e])
        np.testing.assert_allclose(A[e], Ao, atol=1e-13 * np.abs(Ao).max())
        np.testing.assert_allclose(R[e], -Bo, atol=1e-15)
        assert np.array_equal(A[e] != 0, Ao != 0)       # same sparsity pattern


@pytest.mark.parametrize("p,N,ang,n", CASES)
def test_local_fp64_matches_oracle(lib, p, N, ang, n):
    import torch
    kappa, omega, h = H.random_elements(n, p, seed=p * 10 + N)
    ctx = _ctx(lib, p, N, 0.85, ang)
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
    st = ctx.elrt_build_local(torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda"), h, i2o, i2m,
                              mode=lib.LOCAL_FP64)
    assert st.n_flagged == 0 and st.max_rel_residual < 1e-12
    _, (o_i2o, o_i2m) = _oracle_ops(p, N, 0.85, ang, kappa, omega, h)
    np.testing.assert_allclose(i2o.cpu().numpy(), o_i2o, atol=1e-11)
    np.testing.assert_allclose(i2m.cpu().numpy(), o_i2m, atol=1e-11)


@pytest.mark.parametrize("p,N,ang,n", CASES)
def test_local_fp32_refined_matches_oracle(lib, p, N, ang, n):
    """FP32 LU + 2 FP64 refinement steps reaches FP64-level agreement (target 1e-6)."""
    import torch
    kappa, omega, h = H.random_elements(n, p, seed=p * 10 + N + 1)
    ctx = _ctx(lib, p, N, 0.85, ang)
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
    k, o = torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda")
    _, (o_i2o, o_i2m) = _oracle_ops(p, N, 0.85, ang, kappa, omega, h)
    st0 = ctx.elrt_build_local(k, o, h, i2o, i2m, mode=lib.LOCAL_FP32_IR, refine_steps=0)
    err0 = np.abs(i2o.cpu().numpy() - o_i2o).max()
    st = ctx.elrt_build_local(k, o, h, i2o, i2m, mode=lib.LOCAL_FP32_IR, refine_steps=2)
    err2 = np.abs(i2o.cpu().numpy() - o_i2o).max()
    assert st.n_flagged == 0 and st.max_rel_residual < 1e-12
    assert err0 < 1e-3 and st0.max_rel_residual > 1e-9     # unrefined: FP32 accuracy
    assert err2 < 1e-10, (err0, err2)
    np.testing.assert_allclose(i2m.cpu().numpy(), o_i2m, atol=1e-10)


def test_fp32_output_dtype(lib):
    import torch
    p, N, n = 4, 8, 6
    kappa, omega, h = H.random_elements(n, p, seed=3)
    ctx = _ctx(lib, p, N, 0.5, "fv0")
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float32, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float32, device="cuda")
    ctx.elrt_build_local(torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda"), h, i2o, i2m,
                         mode=lib.LOCAL_FP32_IR)
    _, (o_i2o, o_i2m) = _oracle_ops(p, N, 0.5, "fv0", kappa, omega, h)
    np.testing.assert_allclose(i2o.cpu().numpy(), o_i2o, atol=1e-6, rtol=1e-6)
    np.testing.assert_allclose(i2m.cpu().numpy(), o_i2m, atol=1e-6, rtol=1e-6)


def test_albedo_one_row_sums(lib):
    """Constant preservation holds for the library's operators too (omega = 1)."""
    import torch
    p, N, n = 6, 16, 8
    kappa, _, h = H.random_elements(n, p, seed=11)
    ctx = _ctx(lib, p, N, 0.85, "fv0")
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
    ctx.elrt_build_local(torch.tensor(kappa, device="cuda"), torch.ones(n, dtype=torch.float64, device="cuda"), h,
                         i2o, i2m, mode=lib.LOCAL_FP32_IR)
    np.testing.assert_allclose(i2o.sum(-1).cpu().numpy(), 1.0, atol=1e-11)
    np.testing.assert_allclose(i2m.sum(-1).cpu().numpy(), 1.0, atol=1e-11)


def test_per_element_h_and_empty_batch(lib):
    import torch
    p, N, n = 3, 8, 5
    kappa, omega, _ = H.random_elements(n, p, seed=5)
    hs = np.linspace(0.05, 1.0, n)
    ctx = _ctx(lib, p, N, 0.85, "fv0")
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
    ctx.elrt_build_local(torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda"), 1.0, i2o, i2m,
                         mode=lib.LOCAL_FP64, h_elem=torch.tensor(hs, device="cuda"))
    d = hdg.Disc(p, N, 0.85)
    for e in range(n):
        a, m, _ = d.local_operators(kappa[e] * hs[e] / 2, omega[e])
        np.testing.assert_allclose(i2o[e].cpu().numpy(), a, atol=1e-11)
    z = torch.empty(0, dtype=torch.float64, device="cuda")
    ctx.elrt_build_local(z.view(0, ctx.nm), z, 1.0, z, z, mode=lib.LOCAL_FP64)


@pytest.mark.parametrize("bad", ["negative", "nan", "omega"])
def test_bad_inputs_rejected(lib, bad):
    import torch
    p, N, n = 2, 4, 3
    kappa, omega, h = H.random_elements(n, p, seed=1)
    if bad == "negative":
        kappa[1, 3] = -1.0
    elif bad == "nan":
        kappa[2, 0] = np.nan
    else:
        omega[0] = 1.5
    ctx = _ctx(lib, p, N, 0.85, "fv0")
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.ElrtError) as ei:
        ctx.elrt_build_local(torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda"), h, i2o, i2m)
    assert ei.value.status == 1


@pytest.mark.parametrize("mode,refine", [("fp32ir", 2), ("tf32ir", 1)])
def test_full_size_slab_sampled_parity_and_energy_balance(lib, mode, refine):
    """The 64 x 64, p = 6, N = 16 Gaussian-cloud slab in the benchmark's launch configuration
    (tf32ir, one refinement sweep): sampled elements against the oracle one by one; the energy
    balance on every element."""
    import torch
    import workloads as W
    prob = W.problem_gaussian_slab()
    ctx = _ctx(lib, 6, 16, 0.85, "fv0")
    kap = torch.tensor(H.lib_kappa(prob), device="cuda")
    om = torch.tensor(prob.omega, device="cuda")
    n = prob.n_elems
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float32, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float32, device="cuda")
    st = ctx.elrt_build_local(kap, om, prob.h, i2o, i2m,
                              mode=lib.LOCAL_FP32_IR if mode == "fp32ir" else lib.LOCAL_TF32_IR, refine_steps=refine)
    assert st.n_flagged == 0
    d = hdg.Disc(6, 16, 0.85)
    mesh = hdg.Mesh(prob.nx, prob.nz, prob.h)
    kh_o = hdg.nodal_kappa_hat(prob, d, mesh)
    rng = np.random.default_rng(0)
    for e in list(rng.choice(n, 6, replace=False)) + [0, n - 1, 32 * 64 + 32]:
        a, m, _ = d.local_operators(kh_o[e], prob.omega[e])
        np.testing.assert_allclose(i2o[e].double().cpu().numpy(), a, atol=2e-6, rtol=2e-6)
        np.testing.assert_allclose(i2m[e].double().cpu().numpy(), m, atol=2e-6, rtol=2e-6)
    # energy balance on every element, evaluated in FP64 from the library's FP32 operators
    xi, w = lib.elrt_lgl(6)
    sx, sz = hdg.directions(16, "fv0")
    normals = ((0, -1), (1, 0), (0, 1), (-1, 0))
    sdn = [sx * a + sz * b for a, b in normals]
    inc = [[k for k in range(16) if sdn[F][k] < 0] for F in range(4)]
    outc = [[k for k in range(16) if sdn[F][k] > 0] for F in range(4)]
    w2 = np.outer(w, w).reshape(-1)
    khl = H.lib_kappa(prob) * prob.h / 2
    A = i2o.double().cpu().numpy()
    Mm = i2m.double().cpu().numpy()
    worst = max(np.abs(H.energy_defect(w, sdn, inc, outc, w2, khl[e], prob.omega[e], 16, A[e], Mm[e])).max()
                for e in range(0, n, 7))
    assert worst < 1e-5


@pytest.mark.parametrize("p,N,ang,n", CASES)
def test_local_tensor_core_lu_matches_oracle(lib, p, N, ang, n):
    """No-pivot LU with 3xTF32 tcgen05 trailing updates, then FP64-class refinement."""
    import torch
    kappa, omega, h = H.random_elements(n, p, seed=p * 10 + N + 2)
    ctx = _ctx(lib, p, N, 0.85, ang)
    i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
    k, o = torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda")
    _, (o_i2o, o_i2m) = _oracle_ops(p, N, 0.85, ang, kappa, omega, h)
    st0 = ctx.elrt_build_local(k, o, h, i2o, i2m, mode=lib.LOCAL_TF32_IR, refine_steps=0)
    err0 = np.abs(i2o.cpu().numpy() - o_i2o).max()
    st = ctx.elrt_build_local(k, o, h, i2o, i2m, mode=lib.LOCAL_TF32_IR, refine_steps=2)
    err2 = np.abs(i2o.cpu().numpy() - o_i2o).max()
    assert st.n_flagged == 0                  # (unrefined results are flagged by the residual check)
    assert err0 < 1e-4 and st0.max_rel_residual > 1e-10, err0   # 3xTF32: FP32-level before refinement
    assert err2 < 1e-10 and st.max_rel_residual < 1e-12, (err0, err2, st.max_rel_residual)
    np.testing.assert_allclose(i2m.cpu().numpy(), o_i2m, atol=1e-10)



@pytest.mark.parametrize("mode", ["tf32ir", "fp32ir"])
def test_small_batch_matches_large_batch(lib, mode):
    """A batch smaller than the GPU spreads each element's residual over several blocks (column
    chunks per block); a large batch runs one block per element.  The arithmetic per entry is the
    same, so nine elements built alone and the same nine inside a batch of 640 give bit-identical
    operators and the same residual statistics."""
    import torch
    p, N = 6, 16
    kappa, omega, h = H.random_elements(640, p, seed=91)
    ctx = _ctx(lib, p, N, 0.85, "fv0")
    m = {"tf32ir": lib.LOCAL_TF32_IR, "fp32ir": lib.LOCAL_FP32_IR}[mode]

    def build(k, o, refine):
        n = o.size
        a = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
        b = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
        st = ctx.elrt_build_local(torch.tensor(k, device="cuda"), torch.tensor(o, device="cuda"), h, a, b, mode=m,
                                  refine_steps=refine, stats=True)
        return a.cpu().numpy(), b.cpu().numpy(), st

    pick = np.array([0, 5, 77, 150, 300, 301, 450, 600, 639])
    for refine in (1, 2):
        a_all, b_all, st_all = build(kappa, omega, refine)
        a_few, b_few, st_few = build(kappa[pick], omega[pick], refine)
        assert np.array_equal(a_few, a_all[pick]) and np.array_equal(b_few, b_all[pick]), refine
        assert st_few.n_flagged == 0 and st_all.n_flagged == 0
        assert st_few.max_rel_residual <= st_all.max_rel_residual


@pytest.mark.parametrize("p,N,ang,n", [CASES[1], CASES[3], CASES[4]])
def test_local_lu_products_fp16_and_tf32(lib, p, N, ang, n):
    """The trailing updates of the factorisation with 3xFP16 products (the default when the
    assembled entries lie in FP16's range) and with 3xTF32: before refinement both at FP32-level
    accuracy and different from each other (so the FP16 path ran), after two refinement sweeps both
    at the FP64 oracle to 1e-10."""
    import torch
    kappa, omega, h = H.random_elements(n, p, seed=p * 10 + N + 5)
    ctx = _ctx(lib, p, N, 0.85, ang)
    k, o = torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda")
    _, (o_i2o, o_i2m) = _oracle_ops(p, N, 0.85, ang, kappa, omega, h)
    out = {}
    for prod in (lib.LU_PRODUCTS_TF32, lib.LU_PRODUCTS_AUTO):
        ctx.elrt_set_lu_products(prod)
        i2o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
        i2m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
        ctx.elrt_build_local(k, o, h, i2o, i2m, mode=lib.LOCAL_TF32_IR, refine_steps=0)
        a0 = i2o.cpu().numpy()
        st = ctx.elrt_build_local(k, o, h, i2o, i2m, mode=lib.LOCAL_TF32_IR, refine_steps=2)
        out[prod] = (a0, np.abs(a0 - o_i2o).max(), np.abs(i2o.cpu().numpy() - o_i2o).max(), st,
                     np.abs(i2m.cpu().numpy() - o_i2m).max())
    a_t, e0_t, e2_t, st_t, m_t = out[lib.LU_PRODUCTS_TF32]
    a_h, e0_h, e2_h, st_h, m_h = out[lib.LU_PRODUCTS_AUTO]
    assert not np.array_equal(a_t, a_h)                      # the two product forms differ before refinement
    assert e0_t < 1e-4 and e0_h < 1e-4 and e0_h < 10 * e0_t + 1e-7, (e0_t, e0_h)
    assert e2_t < 1e-10 and e2_h < 1e-10 and m_t < 1e-10 and m_h < 1e-10, (e2_t, e2_h, m_t, m_h)
    assert st_t.n_flagged == 0 and st_h.n_flagged == 0 and st_h.max_rel_residual < 1e-12


def test_lu_products_setting_rejects_other_values(lib):
    ctx = _ctx(lib, 4, 8, 0.85, "fv0")
    ctx.elrt_set_lu_products(lib.LU_PRODUCTS_TF32)
    ctx.elrt_set_lu_products(lib.LU_PRODUCTS_AUTO)
    for bad in (-1, 2, 7):
        with pytest.raises(lib.ElrtError):
            ctx.elrt_set_lu_products(bad)
