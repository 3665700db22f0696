"""The C ABI library: it loads, exports every entry point include/elrt.h declares, and its host-side
tables and argument checks behave (CPU only: no compute call needs a GPU here)."""

import ctypes
import os

import numpy as np
import pytest

from oracle import hdg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def E():
    from paper_2308_02467_gb300 import build
    build.build()
    import paper_2308_02467_gb300 as mod
    return mod


def test_every_declared_symbol_is_exported(E):
    lib = ctypes.CDLL(E.LIB_PATH)
    names = E.exported_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_lgl_matches_oracle(E):
    for p in range(1, 11):
        xi, w = E.elrt_lgl(p)
        xo, wo = hdg.lgl(p)
        np.testing.assert_allclose(xi, xo, atol=2e-15)
        np.testing.assert_allclose(w, wo, atol=2e-14)


@pytest.mark.parametrize("N,g,ang", [(16, 0.85, 0), (28, 0.8, 0), (8, 0.0, 1), (16, 0.5, 1), (32, 0.9, 0), (4, 0.3, 0)])
def test_phase_matrix_matches_oracle(E, N, g, ang):
    W = E.elrt_phase_matrix(N, g, ang)
    np.testing.assert_allclose(W, hdg.phase_matrix(N, g, "fv0" if ang == 0 else "do"), atol=1e-14)


def test_node_coords_match_oracle(E):
    x, z = E.elrt_node_coords(3, 8, 4, 3, 0.5)
    xo, zo = hdg.Mesh(4, 3, 0.5).node_coords(hdg.Disc(3, 8, 0.0))
    np.testing.assert_allclose(x, xo, atol=1e-15)
    np.testing.assert_allclose(z, zo, atol=1e-15)


def test_sizes(E):
    assert E.elrt_n_nodes(6, 16) == 49
    assert E.elrt_n_local(6, 16) == 784
    assert E.elrt_n_skel(6, 16) == 224
    assert E.elrt_n_inflow(6, 16, 64, 64) == 2 * 128 * 7 * 8
    assert E.elrt_n_skel(6, 28) == 392           # the paper's Q6, N_a = 28 element
    assert E.elrt_n_nodes(6, 18) == -1           # N must be a multiple of 4
    assert E.elrt_n_nodes(11, 16) == -1          # p <= 10


def test_bad_discretisation_rejected_before_any_cuda_call(E):
    from paper_2308_02467_gb300._binding import _lib, Disc
    h = ctypes.c_void_p()
    for d in (Disc(6, 18, 0, 0.85), Disc(0, 16, 0, 0.85), Disc(6, 16, 2, 0.85), Disc(6, 16, 0, 1.0), Disc(6, 64, 0, 0.5)):
        assert _lib.elrt_create(ctypes.byref(h), ctypes.byref(d), None) == 1
    assert _lib.elrt_lgl(0, None, None) == 1
    assert _lib.elrt_status_str(4) == b"iteration did not converge"


def test_null_context_is_einval(E):
    from paper_2308_02467_gb300._binding import _lib
    assert _lib.elrt_build_local(None, 1, 1.0, None, None, None, 0, 0, 0, None, None, None, None) == 1
    assert _lib.elrt_solve_global(None, 1, 1, None, 0, None, 1e-6, 10, 10, 0, None, None) == 1
    assert _lib.elrt_destroy(None) == 0
