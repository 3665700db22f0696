"""GPU parity of the whole-pipeline entry points (Algorithm 1 in one call; many uneven fields of
mixed degree in waves) against the FP64 oracle."""

import dataclasses

import numpy as np
import pytest

from oracle import hdg
from tests import _helpers as H

pytestmark = pytest.mark.gpu


def _dev(problem):
    import torch
    return (torch.tensor(H.lib_kappa(problem), device="cuda"), torch.tensor(problem.omega, device="cuda"),
            torch.tensor(problem.inflow, device="cuda"))


@pytest.mark.parametrize("mode", ["fp32ir", "tf32ir"])
def test_solve_field_matches_oracle(lib, mode):
    import torch
    prob = H.small_cloud(8, 6, 6, 16)
    ref = hdg.solve_problem(prob, rtol=1e-13)
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, lib.ANG_FV0)
    k, o, g = _dev(prob)
    mean = torch.empty(prob.n_elems, ctx.nm, dtype=torch.float64, device="cuda")
    # two refinement sweeps: the 3xTF32 factors of the thickest elements need the second one to
    # reach the FP32-class residual that the flag threshold asks for
    st = ctx.elrt_solve_field(prob.nx, prob.nz, prob.h, k, o, g, mean, rtol=1e-12,
                              mode=lib.LOCAL_FP32_IR if mode == "fp32ir" else lib.LOCAL_TF32_IR,
                              refine_steps=1 if mode == "fp32ir" else 2)
    assert st.glob.converged == 1 and st.local.n_flagged == 0 and st.local_ms > 0 and st.global_ms > 0
    assert hdg.rel_l2(mean.cpu().numpy(), ref["u_mean"], ref["disc"]) < 1e-6


def test_solve_batch_uneven_fields_in_waves(lib):
    """Five fields of different sizes and degrees through three contexts, with a wave budget small
    enough to force several waves and three concurrent worker streams."""
    import torch
    specs = [(5, 3, 2, 0.9), (4, 4, 3, 0.95), (6, 2, 2, 1.0), (3, 5, 4, 0.9), (2, 2, 3, 0.8)]
    probs = [dataclasses.replace(H.small_cloud(nx, nz, p, 8, omega=om, random_inflow=True, seed=nx * 7 + p),
                                 hg_g=0.6) for nx, nz, p, om in specs]
    degrees = sorted({p.p for p in probs})
    ctxs = [lib.Context(p, 8, 0.6, lib.ANG_FV0) for p in degrees]
    fields, fctx, means = [], [], []
    for pr in probs:
        k, o, g = _dev(pr)
        fields.append((pr.nx, pr.nz, pr.h, k, o, g))
        fctx.append(degrees.index(pr.p))
        means.append(torch.empty(pr.n_elems, (pr.p + 1) ** 2, dtype=torch.float64, device="cuda"))
    stats = lib.elrt_solve_batch(ctxs, fields, fctx, means, rtol=1e-12, wave_bytes=200_000, workers=3)
    for pr, m, st in zip(probs, means, stats):
        ref = hdg.solve_problem(pr, rtol=1e-13)
        assert st.glob.converged == 1
        assert hdg.rel_l2(m.cpu().numpy(), ref["u_mean"], ref["disc"]) < 1e-6
