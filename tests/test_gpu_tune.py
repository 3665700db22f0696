"""The autotuner (elrt_autotune): it times every candidate configuration on the given field, keeps
the fastest, caches it in the file ELRT_TUNE_CACHE names, and a new context of the same device
and discretisation starts from the cached parameters.  Both LU panel schedules and any chunk size
give the same operators."""

import numpy as np
import pytest

from tests import _helpers as H

pytestmark = pytest.mark.gpu


def _inputs(lib, prob):
    import torch
    return (torch.tensor(H.lib_kappa(prob), device="cuda"), torch.tensor(prob.omega, device="cuda"),
            torch.tensor(prob.inflow, device="cuda"))


def test_autotune_measures_keeps_and_caches(lib, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("ELRT_TUNE_CACHE", str(cache))
    prob = H.small_cloud(24, 24, 6, 16)            # 576 elements: chunk candidates 0 (all) and 512
    kap, om, g = _inputs(lib, prob)
    ctx = lib.Context(prob.p, prob.n_angles, prob.hg_g, lib.ANG_FV0)
    assert ctx.elrt_get_tuning()["tuned"] == 0
    rep = ctx.elrt_autotune(prob.nx, prob.nz, prob.h, kap, om, g, mode=lib.LOCAL_TF32_IR, refine_steps=1, rtol=1e-8)
    print("autotune:", rep)
    assert rep["n_candidates"] == 2 * 2 + 5
    assert 0 < rep["local_ms_best"] <= rep["local_ms_default"]
    assert 0 < rep["solve_ms_best"] <= rep["solve_ms_default"] * 1.0001
    t = ctx.elrt_get_tuning()
    assert t["tuned"] == 1 and t["restart"] in (8, 12, 16, 20, 30) and t["local_chunk"] in (0, 512)
    assert (t["local_chunk"], t["lu_pairs"], t["restart"]) == (rep["local_chunk"], rep["lu_pairs"], rep["restart"])
    line = cache.read_text().strip().splitlines()[-1].split()
    assert line[:2] == ["elrt-tune", "v1"] and line[3:6] == ["6", "16", "0"]
    ctx2 = lib.Context(prob.p, prob.n_angles, prob.hg_g, lib.ANG_FV0)
    assert ctx2.elrt_get_tuning() == t
    ctx3 = lib.Context(4, 8, prob.hg_g, lib.ANG_FV0)      # another discretisation: defaults
    assert ctx3.elrt_get_tuning()["tuned"] == 0
    for c in (ctx, ctx2, ctx3):
        c.close()


@pytest.mark.parametrize("p,N", [(6, 16), (4, 8)])
def test_panel_schedules_and_chunks_agree(lib, p, N):
    """Pairs of panels (rank-128 updates) and single panels (rank-64), one chunk or several: the
    refined operators agree to FP64 level."""
    import torch
    n = 40
    kappa, omega, h = H.random_elements(n, p, seed=77)
    ctx = lib.Context(p, N, 0.85, lib.ANG_FV0)
    k, o = torch.tensor(kappa, device="cuda"), torch.tensor(omega, device="cuda")
    res = []
    for chunk, pairs in ((0, 1), (0, 0), (16, 1), (7, 0)):
        ctx.elrt_set_tuning(chunk, pairs, 12)
        a = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
        m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
        st = ctx.elrt_build_local(k, o, h, a, m, mode=lib.LOCAL_TF32_IR, refine_steps=2)
        assert st.n_flagged == 0
        res.append((a.cpu().numpy(), m.cpu().numpy()))
    for a, m in res[1:]:
        np.testing.assert_allclose(a, res[0][0], atol=1e-11)
        np.testing.assert_allclose(m, res[0][1], atol=1e-11)
    ctx.close()
