"""bench.py's refinement-study interpolation on the CPU: the per-element Lagrange interpolation of
a coarse nodal solution to the nodes of a refined mesh is exact for fields the coarse degree
represents, and the Lagrange matrix is the identity at the nodes themselves."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import hdg  # noqa: E402


def test_lagrange_matrix_is_identity_at_nodes_and_exact_on_polynomials():
    xi, _ = hdg.lgl(5)
    np.testing.assert_allclose(bench.lagrange_matrix(xi, xi), np.eye(6), atol=1e-13)
    pts = np.linspace(-1, 1, 17)
    for q in range(6):
        np.testing.assert_allclose(bench.lagrange_matrix(xi, pts) @ xi ** q, pts ** q, atol=1e-12)


def test_subcell_interpolation_reproduces_a_polynomial_field():
    p, r = 4, 3
    xi, _ = hdg.lgl(p)

    def nodal(n):
        h = 1.0 / n
        u = np.zeros((n, n, p + 1, p + 1))
        for iz in range(n):
            for ix in range(n):
                x = ix * h + (xi + 1) / 2 * h
                z = iz * h + (xi + 1) / 2 * h
                u[iz, ix] = x[None, :] ** 3 + z[:, None] ** 2 * x[None, :]
        return u

    coarse, fine = nodal(2), nodal(2 * r)
    for si in range(r):
        Lx = bench.lagrange_matrix(xi, -1 + (2.0 / r) * (si + (xi + 1) / 2))
        for sj in range(r):
            Lz = bench.lagrange_matrix(xi, -1 + (2.0 / r) * (sj + (xi + 1) / 2))
            uc = np.einsum("qb,zxba,pa->zxqp", Lz, coarse, Lx)
            np.testing.assert_allclose(uc, fine[sj::r, si::r], atol=1e-12)
