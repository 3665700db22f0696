"""The benchmark workload at full size in the benchmark's launch configuration, against the FP64
oracle's solution of the whole field: the 64 x 64 Gaussian-cloud slab (p = 6, N = 16, 4096
elements), TF32-IR local solves with one refinement sweep, GMRES(12) to 1e-8 with FP16 Arnoldi
matvecs, mean-intensity recovery.  The expected mean intensity was written by
tests/golden/make_gaussian_slab_golden.py, which calls only the oracle."""

import json
import os

import numpy as np
import pytest

import workloads as W
from tests import _helpers as H

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_benchmark_slab_matches_oracle_whole_field(lib):
    import torch
    ref = np.load(os.path.join(GOLDEN, "gaussian_slab_64x64_mean.npy"))
    meta = json.load(open(os.path.join(GOLDEN, "gaussian_slab_64x64_mean.json")))
    assert meta["rel_residual"] < 1e-11
    prob = W.problem_gaussian_slab()
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, lib.ANG_FV0)
    ctx.elrt_set_krylov_op(lib.KRYLOV_F16)
    n = prob.n_elems
    kap = torch.tensor(H.lib_kappa(prob), device="cuda")
    om = torch.tensor(prob.omega, device="cuda")
    g = torch.tensor(prob.inflow, device="cuda")
    a = torch.empty(n, ctx.nin, ctx.nin, device="cuda", dtype=torch.float32)
    m = torch.empty(n, ctx.nm, ctx.nin, device="cuda", dtype=torch.float32)
    sk = torch.empty(n * ctx.nin, device="cuda", dtype=torch.float64)
    um = torch.empty(n, ctx.nm, device="cuda", dtype=torch.float64)
    lst = ctx.elrt_build_local(kap, om, prob.h, a, m, mode=lib.LOCAL_TF32_IR, refine_steps=1)
    gst = ctx.elrt_solve_global(prob.nx, prob.nz, a, g, sk, rtol=1e-8, restart=12, max_iter=20000)
    ctx.elrt_recover_mean(prob.nx, prob.nz, m, sk, g, um)
    got = um.cpu().numpy()
    xi, w = lib.elrt_lgl(prob.p)
    w2 = np.outer(w, w).reshape(-1)[None, :]
    rel = float(np.sqrt(np.sum(w2 * (got - ref) ** 2) / np.sum(w2 * ref ** 2)))
    print(f"64x64 slab vs oracle: rel L2 {rel:.2e}, GMRES {gst.iterations} it, local residual {lst.max_rel_residual:.1e}")
    assert lst.n_flagged == 0 and gst.converged
    assert rel <= 1e-6, rel
    ctx.close()
