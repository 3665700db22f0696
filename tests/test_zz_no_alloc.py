"""The allocation-free local build (elrt_build_local_static).

Some callers cannot allocate device memory (their device memory is owned by another framework,
or they run in a loop that must not allocate after start-up, or they are a plug-in handed buffers
but no allocator).  For them the library offers one entry point whose scratch is a fixed device
array inside the library.  These tests call it through the C ABI, twice in a row, and check its
in2out / in2sol against the context-based elrt_build_local on the same inputs.
"""

import numpy as np
import pytest

from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,N,mode,n,tol", [
    (4, 8, "fp64", 37, 1e-11),     # one chunk
    (6, 16, "fp32ir", 29, 1e-10),  # several chunks of the fixed array, ragged last chunk
])
def test_static_build_matches_context_build(lib, p, N, mode, n, tol):
    import torch
    kappa, omega, h = H.random_elements(n, p, seed=900 + p)
    k = torch.tensor(kappa, device="cuda")
    o = torch.tensor(omega, device="cuda")
    m = lib.LOCAL_FP64 if mode == "fp64" else lib.LOCAL_FP32_IR
    ctx = lib.Context(p, N, 0.85, lib.ANG_FV0)
    ref_o = torch.empty(n, ctx.nin, ctx.nin, dtype=torch.float64, device="cuda")
    ref_m = torch.empty(n, ctx.nm, ctx.nin, dtype=torch.float64, device="cuda")
    ctx.elrt_build_local(k, o, h, ref_o, ref_m, mode=m, refine_steps=2)
    ref_o, ref_m = ref_o.cpu().numpy(), ref_m.cpu().numpy()
    for call in range(2):
        out_o = torch.full((n, ctx.nin, ctx.nin), float("nan"), dtype=torch.float64, device="cuda")
        out_m = torch.full((n, ctx.nm, ctx.nin), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.elrt_build_local_static(p, N, 0.85, lib.ANG_FV0, k, o, h, out_o, out_m, mode=m, refine_steps=2)
        assert st == 0, f"call {call}: status {st}"
        np.testing.assert_allclose(out_o.cpu().numpy(), ref_o, atol=tol, rtol=0)
        np.testing.assert_allclose(out_m.cpu().numpy(), ref_m, atol=tol, rtol=0)
    ctx.close()


def test_static_build_rejects_elements_larger_than_the_array(lib):
    """p = 10, N = 32: one element's local system needs far more than the fixed array holds."""
    import torch
    p, N = 10, 32
    nm, nin = (p + 1) ** 2, 2 * (p + 1) * N
    k = torch.ones(1, nm, dtype=torch.float64, device="cuda")
    o = torch.full((1,), 0.9, dtype=torch.float64, device="cuda")
    out_o = torch.zeros(1, nin, nin, dtype=torch.float64, device="cuda")
    out_m = torch.zeros(1, nm, nin, dtype=torch.float64, device="cuda")
    st = lib.elrt_build_local_static(p, N, 0.5, lib.ANG_FV0, k, o, 0.1, out_o, out_m, mode=lib.LOCAL_FP64)
    assert st == 1
    assert not torch.any(out_o) and not torch.any(out_m)


def test_static_build_allocates_nothing_and_validates_inputs(lib):
    """After a first call (which looks up the array's address), further calls that run several
    chunks leave the device's free memory unchanged; invalid kappa / omega give EINVAL."""
    import torch
    p, N, n = 6, 16, 29
    kappa, omega, h = H.random_elements(n, p, seed=901)
    k = torch.tensor(kappa, device="cuda")
    o = torch.tensor(omega, device="cuda")
    nm, nin = (p + 1) ** 2, 2 * (p + 1) * N
    out_o = torch.empty(n, nin, nin, dtype=torch.float32, device="cuda")
    out_m = torch.empty(n, nm, nin, dtype=torch.float32, device="cuda")
    run = lambda kk, oo: lib.elrt_build_local_static(p, N, 0.85, lib.ANG_FV0, kk, oo, h, out_o, out_m,
                                                     mode=lib.LOCAL_FP32_IR, refine_steps=1)
    assert run(k, o) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert run(k, o) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    bad = k.clone()
    bad[3, 5] = -1.0
    assert run(bad, o) == 1
    bad_o = o.clone()
    bad_o[0] = 1.5
    assert run(k, bad_o) == 1
    assert run(k, o) == 0          # the flags start from zero again on the next call
