"""FP64 oracle of the classical HDG element method.  TEST INFRASTRUCTURE ONLY.

Plain, slow, dense numpy code that follows the paper's formulation:

* Sec. 2.1, eq. RT_PDE: steady transport with extinction, scattering and the
  Henyey-Greenstein phase function normalised on the circle.
* Sec. 2.2.1-2.2.3: Q_p spectral elements on LGL nodes (the nodes are the
  quadrature points), P0 angular cells, upwind DG (eqs. dg, dg_flux), its
  hybridisation (eqs. hdg_local, hdg_global) and the element matrices
  B, B^, C, M, S of eq. hdg_local_all_sub_mat / Appendix A.
* eq. hdg_local_i2u: A_i2u = -(B - C + M - S)^{-1} B^.
* eq. hdg_local_i2o: A_i2o = R^o A_i2u.  Sec. 2.4, eq. ang_ave: A_i2m = R_u2m A_i2u.
* eq. hdg_global_mat: sum_K (R^o_K - A_i2o^K) u^ = 0 (f = 0), solved by GMRES
  (Sec. 2.3) or densely on tiny meshes.
* Algorithm 1, step 4: mean-intensity recovery u^m = A_i2m u^_in.
* Sec. 2.3 names transport sweeps among the solvers of radiative transfer: sweep_precond applies
  upwind block Gauss-Seidel sweeps of eq. hdg_global_mat (the elements taken in the wavefront
  order of one mesh corner, then of the others; each sweep recomputes every outflow value, or only
  those of the faces pointing away from its corner), the preconditioner of the library's GMRES.

Readings where the paper is silent:
* every integral uses the (p+1)-point LGL rule per direction (diagonal mass);
* every equation of element K is divided by (h/2) * dtheta, so only
  kappa_hat = kappa * h / 2 enters (Sec. 2.4.1, second paragraph);
* "fv0" angular mode: cell-averaged directions sbar_k and the cell-averaged
  phase matrix W_kl = (1/dtheta) int_k int_l p; "do" mode: directions and
  phase sampled at cell centres; W is rescaled so its rows sum to exactly 1;
* sigma_s = omega * sigma_e with omega constant per element (Sec. 2.4.1).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
from numpy.polynomial import legendre as npleg

# faces of the reference square, in the order used for every face-indexed array
FACE_NORMALS = ((0.0, -1.0), (1.0, 0.0), (0.0, 1.0), (-1.0, 0.0))   # bottom, right, top, left
OPPOSITE = (2, 3, 0, 1)


# ----------------------------------------------------------------------------------------------
# 1D spectral element ingredients (Sec. 2.2.1 and eq. sigma_se)
# ----------------------------------------------------------------------------------------------

def lgl(p: int):
    """LGL nodes (ascending) and weights on [-1, 1].

    Interior nodes are the roots of P_p'; weights are 2 / (p (p+1) P_p(x)^2).
    """
    if p < 1:
        raise ValueError("p >= 1")
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    d1 = npleg.legder(cp)
    d2 = npleg.legder(d1)
    inner = np.sort(np.real(npleg.legroots(d1))) if p >= 2 else np.zeros(0)
    for _ in range(3):                     # Newton polish of the companion-matrix roots
        inner = inner - npleg.legval(inner, d1) / npleg.legval(inner, d2)
    xi = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (p * (p + 1) * npleg.legval(xi, cp) ** 2)
    return xi, w


def lagrange_derivative(xi: np.ndarray) -> np.ndarray:
    """D[m, a] = l_a'(xi_m), with l_a the Lagrange polynomial of node a (product rule, written out)."""
    n = len(xi)
    D = np.zeros((n, n))
    for a in range(n):
        for m in range(n):
            s = 0.0
            for c in range(n):
                if c == a:
                    continue
                t = 1.0 / (xi[a] - xi[c])
                for b in range(n):
                    if b != a and b != c:
                        t *= (xi[m] - xi[b]) / (xi[a] - xi[b])
                s += t
            D[m, a] = s
    return D


# ----------------------------------------------------------------------------------------------
# angular discretisation (Sec. 2.2.1, Sec. 2.4.1: uniform cells on [0, 2pi], p_a = 0)
# ----------------------------------------------------------------------------------------------

def directions(n_angles: int, angular: str = "fv0"):
    """(s_x, s_z) per angular cell k = [k dth, (k+1) dth).

    fv0: the cell average (1/dth) int_k (cos t, sin t) dt (what int_{K^a} s ds / |K^a| gives);
    do:  the direction at the cell centre.
    """
    dth = 2.0 * math.pi / n_angles
    k = np.arange(n_angles)
    if angular == "fv0":
        sx = (np.sin((k + 1) * dth) - np.sin(k * dth)) / dth
        sz = (np.cos(k * dth) - np.cos((k + 1) * dth)) / dth
    elif angular == "do":
        sx = np.cos((k + 0.5) * dth)
        sz = np.sin((k + 0.5) * dth)
    else:
        raise ValueError(angular)
    return sx, sz


def hg_unnormalised(t, g):
    """Henyey-Greenstein kernel of Sec. 2.1 without the constant c: (1-g^2)/(1+g^2-2g cos t)^(3/2)."""
    return (1.0 - g * g) / (1.0 + g * g - 2.0 * g * np.cos(t)) ** 1.5


def phase_matrix(n_angles: int, g: float, angular: str = "fv0", nq: int = 64) -> np.ndarray:
    """W[k, l]: coupling of cell l into cell k after dividing the scattering term by dth.

    c is fixed by int_0^{2pi} p = 1 (Sec. 2.1).  fv0: W_kl = (1/dth) int_k int_l p(t - t') dt' dt,
    by an nq x nq Gauss-Legendre rule per pair of cells.  do: W_kl = dth p(t_k - t_l).
    Finally every row is divided by its sum (exactly 1 up to quadrature error).
    """
    dth = 2.0 * math.pi / n_angles
    x, wq = npleg.leggauss(nq)
    # normalisation constant over the whole circle, cell by cell
    c = 0.0
    for k in range(n_angles):
        t = k * dth + 0.5 * dth * (x + 1.0)
        c += 0.5 * dth * np.dot(wq, hg_unnormalised(t, g))
    W = np.zeros((n_angles, n_angles))
    if angular == "fv0":
        for k in range(n_angles):
            t = k * dth + 0.5 * dth * (x + 1.0)
            for l in range(n_angles):
                tp = l * dth + 0.5 * dth * (x + 1.0)
                vals = hg_unnormalised(t[:, None] - tp[None, :], g) / c
                W[k, l] = (0.5 * dth) ** 2 * (wq @ vals @ wq) / dth
    elif angular == "do":
        tc = (np.arange(n_angles) + 0.5) * dth
        W = dth * hg_unnormalised(tc[:, None] - tc[None, :], g) / c
    else:
        raise ValueError(angular)
    return W / W.sum(axis=1, keepdims=True)


# ----------------------------------------------------------------------------------------------
# element discretisation
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Disc:
    """Everything that depends only on (p, N, g, angular mode)."""
    p: int
    n_angles: int
    hg_g: float = 0.0
    angular: str = "fv0"

    def __post_init__(self):
        p, N = self.p, self.n_angles
        if N % 4:
            raise ValueError("the angular cells must respect the faces: N multiple of 4")
        self.n1 = p + 1
        self.nm = self.n1 ** 2                     # spatial nodes per element
        self.nu = self.nm * N                      # local unknowns
        self.xi, self.w = lgl(p)
        self.D = lagrange_derivative(self.xi)
        self.sx, self.sz = directions(N, self.angular)
        self.W = phase_matrix(N, self.hg_g, self.angular)
        self.w2 = np.outer(self.w, self.w).reshape(-1)          # w_a w_b at node a + n1 b
        n1 = self.n1
        # volume node of face position m (ascending coordinate along the face)
        self.face_nodes = [
            [m for m in range(n1)],                 # bottom: b = 0
            [p + n1 * m for m in range(n1)],        # right:  a = p
            [m + n1 * p for m in range(n1)],        # top:    b = p
            [n1 * m for m in range(n1)],            # left:   a = 0
        ]
        sn = [self.sx * nx + self.sz * nz for (nx, nz) in FACE_NORMALS]   # sbar_k . n_F
        self.s_dot_n = np.array(sn)                                         # [4, N]
        self.out_cells = [[k for k in range(N) if sn[F][k] > 0] for F in range(4)]
        self.in_cells = [[k for k in range(N) if sn[F][k] < 0] for F in range(4)]
        for F in range(4):
            if len(self.out_cells[F]) != N // 2 or len(self.in_cells[F]) != N // 2:
                raise ValueError("an angular cell is tangent to a face")
        half = N // 2
        self.n_face = n1 * half                    # skeleton DOFs per face and direction sense
        self.n_in = 4 * self.n_face
        self.n_out = 4 * self.n_face
        # outflow skeleton DOF (F, m, kk) -> local row k*nm + node; inflow (F, m, kk) -> column
        self.out_rows = np.array([self.out_cells[F][kk] * self.nm + self.face_nodes[F][m]
                                  for F in range(4) for m in range(n1) for kk in range(half)])

    def local_system(self, kappa_hat: np.ndarray, omega: float):
        """A = B - C + M - S (nu x nu) and B^ (nu x n_in) for one element (eq. hdg_local_mat).

        Unknown (k, i) sits at row k*nm + i, node i = a + (p+1) b.  Per angular cell k:
          B^k_ii   = sum over faces F with sbar_k.n_F > 0 and i on F of w_m (sbar_k.n_F)
          C^k_ij   = w_j (sbar_k . grad phi_i)(x_j)       (volume term, LGL quadrature)
          M_ij     = delta_ij w_i kappa_hat_i
          S_(k,i),(l,j) = delta_ij w_i omega kappa_hat_i W_kl
          B^_(k,i),(F,m,k) = w_m (sbar_k.n_F) for inflow (F, k), i the node at face position m.
        """
        n1, nm, N = self.n1, self.nm, self.n_angles
        kappa_hat = np.asarray(kappa_hat, dtype=np.float64).reshape(nm)
        I = np.eye(n1)
        Gx = np.kron(I, self.D)      # Gx[j, i] = d/dx phi_i at node j
        Gz = np.kron(self.D, I)      # Gz[j, i] = d/dz phi_i at node j
        A = np.zeros((self.nu, self.nu))
        mass = self.w2 * kappa_hat
        for k in range(N):
            C = (self.sx[k] * Gx + self.sz[k] * Gz).T * self.w2[None, :]
            B = np.zeros(nm)
            for F in range(4):
                if self.s_dot_n[F, k] > 0:
                    for m, node in enumerate(self.face_nodes[F]):
                        B[node] += self.w[m] * self.s_dot_n[F, k]
            blk = slice(k * nm, (k + 1) * nm)
            A[blk, blk] += np.diag(B) - C + np.diag(mass)
        scat = self.w2 * omega * kappa_hat
        for k in range(N):
            for l in range(N):
                A[k * nm:(k + 1) * nm, l * nm:(l + 1) * nm] -= np.diag(scat * self.W[k, l])
        Bhat = np.zeros((self.nu, self.n_in))
        half = N // 2
        for F in range(4):
            for m, node in enumerate(self.face_nodes[F]):
                for kk, k in enumerate(self.in_cells[F]):
                    col = F * self.n_face + m * half + kk
                    Bhat[k * nm + node, col] = self.w[m] * self.s_dot_n[F, k]
        return A, Bhat

    def local_operators(self, kappa_hat, omega):
        """(A_i2o, A_i2m, A_i2u) of one element: eqs. hdg_local_i2u, hdg_local_i2o, ang_ave."""
        A, Bhat = self.local_system(kappa_hat, omega)
        X = np.linalg.solve(A, -Bhat)                     # A_i2u
        A_i2o = X[self.out_rows]                          # R^o A_i2u
        A_i2m = X.reshape(self.n_angles, self.nm, self.n_in).mean(axis=0)   # (1/|S|) int_S = (1/N) sum_k
        return A_i2o, A_i2m, X

    def source_vector(self, f_hat):
        """Right-hand side of a volume source in the local equation (eq. hdg_local_mat with f != 0):
        F[(k, i)] = w_i f_hat[k, i], where f_hat = f h / 2 is the source at node i averaged over angular
        cell k and scaled to the reference element like sigma (Sec. 2.4.1), the equation divided by
        (h/2) dtheta as everywhere."""
        f_hat = np.asarray(f_hat, dtype=np.float64).reshape(self.n_angles, self.nm)
        return (f_hat * self.w2[None, :]).reshape(-1)

    def local_source(self, kappa_hat, omega, f_hat):
        """Source parts of eqs. hdg_local_f2u_i2u and hdg_local_f2o_i2o: f_u = (B - C + M - S)^{-1} F,
        its outflow restriction f^_u = R^o f_u and its angular mean (eq. ang_ave).  Returns
        (f^_u [n_out], mean [nm], f_u [nu])."""
        A, _ = self.local_system(kappa_hat, omega)
        f_u = np.linalg.solve(A, self.source_vector(f_hat))
        return f_u[self.out_rows], f_u.reshape(self.n_angles, self.nm).mean(axis=0), f_u

    def energy_defect(self, kappa_hat, omega, A_i2o, A_i2m):
        """Per inflow column, the discrete energy balance of an element (test function v = 1):

            w_j |sbar.n|_j  =  sum_r w_r (sbar.n)_r A_i2o[r, j]  +  N sum_i w_i kappa_hat_i (1-omega) A_i2m[i, j]

        Returns (lhs - rhs) / lhs per column; exactly 0 for the classical operators.
        """
        half = self.n_angles // 2
        lhs = np.array([self.w[m] * abs(self.s_dot_n[F, k]) for F in range(4) for m in range(self.n1)
                        for k in self.in_cells[F]])
        wout = np.array([self.w[m] * self.s_dot_n[F, k] for F in range(4) for m in range(self.n1)
                         for k in self.out_cells[F]])
        absorb = self.n_angles * self.w2 * np.asarray(kappa_hat).reshape(-1) * (1.0 - omega)
        rhs = wout @ A_i2o + absorb @ A_i2m
        assert lhs.shape[0] == self.n_in and half * 4 * self.n1 == self.n_in
        return (lhs - rhs) / lhs


# ----------------------------------------------------------------------------------------------
# mesh and global skeleton system (eq. hdg_global_mat)
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Mesh:
    nx: int
    nz: int
    h: float

    @property
    def n_elems(self):
        return self.nx * self.nz

    def neighbour(self, e: int, F: int) -> int:
        ix, iz = e % self.nx, e // self.nx
        jx, jz = ix + (0, 1, 0, -1)[F], iz + (-1, 0, 1, 0)[F]
        if 0 <= jx < self.nx and 0 <= jz < self.nz:
            return jx + self.nx * jz
        return -1

    def boundary_face(self, e: int, F: int) -> int:
        """Position of face F of element e inside its side of the domain boundary."""
        ix, iz = e % self.nx, e // self.nx
        return ix if F in (0, 2) else iz

    def node_coords(self, disc: Disc):
        """Physical coordinates (x, z) [E, nm] of the LGL nodes of every element."""
        E = self.n_elems
        ix = np.arange(E) % self.nx
        iz = np.arange(E) // self.nx
        off = (disc.xi + 1.0) * 0.5 * self.h
        a = np.arange(disc.nm) % disc.n1
        b = np.arange(disc.nm) // disc.n1
        return ix[:, None] * self.h + off[a][None, :], iz[:, None] * self.h + off[b][None, :]


def inflow_side_offsets(mesh: Mesh, disc: Disc):
    """Start of each domain side (bottom, right, top, left) in the boundary inflow array."""
    counts = [mesh.nx, mesh.nz, mesh.nx, mesh.nz]
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]) * disc.n_face
    return offs, sum(counts) * disc.n_face


def gather_inflow(mesh: Mesh, disc: Disc, x: np.ndarray, g: np.ndarray | None):
    """Inflow skeleton values [E, n_in] of every element.

    x: outflow skeleton DOFs [E, n_out]; the inflow of K through face F is the outflow of
    the neighbour through the opposite face (same nodes, same cells); on the domain boundary
    it is the projected data g (None: zero).
    """
    E, nf = mesh.n_elems, disc.n_face
    offs, _ = inflow_side_offsets(mesh, disc)
    out = np.zeros((E, disc.n_in))
    for e in range(E):
        for F in range(4):
            nb = mesh.neighbour(e, F)
            if nb >= 0:
                G = OPPOSITE[F]
                out[e, F * nf:(F + 1) * nf] = x[nb, G * nf:(G + 1) * nf]
            elif g is not None:
                s = offs[F] + mesh.boundary_face(e, F) * nf
                out[e, F * nf:(F + 1) * nf] = g[s:s + nf]
    return out


def global_apply(mesh, disc, A_i2o, x):
    """(I - A_int) x: per element x_out(K) - A_i2o^K x_in(K) with interior inflow only."""
    xin = gather_inflow(mesh, disc, x.reshape(mesh.n_elems, disc.n_out), None)
    return (x.reshape(mesh.n_elems, -1) - np.einsum("eij,ej->ei", A_i2o, xin)).reshape(-1)


def global_rhs(mesh, disc, A_i2o, g, f2o=None):
    """Right-hand side of eq. hdg_global_mat: per element A_i2o^K applied to the boundary part of the
    inflow, plus the source term f^_u^K (f2o [E, n_out]) when there is a source."""
    gin = gather_inflow(mesh, disc, np.zeros((mesh.n_elems, disc.n_out)), g)
    b = np.einsum("eij,ej->ei", A_i2o, gin)
    if f2o is not None:
        b = b + f2o
    return b.reshape(-1)


def nodal_source_hat(problem, disc: Disc, mesh: Mesh):
    """f_hat = f h / 2 [E, N, nm] at the LGL nodes of every element, per angular cell (Sec. 2.4.1)."""
    x, z = mesh.node_coords(disc)
    f = np.asarray(problem.source(x, z), dtype=np.float64)         # [E, nm, N]
    return np.transpose(f, (0, 2, 1)) * (mesh.h * 0.5)


def global_dense(mesh, disc, A_i2o):
    """Dense matrix of the skeleton system (tiny meshes only)."""
    E, no, nf = mesh.n_elems, disc.n_out, disc.n_face
    G = np.eye(E * no)
    for e in range(E):
        for F in range(4):
            nb = mesh.neighbour(e, F)
            if nb >= 0:
                Fo = OPPOSITE[F]
                G[e * no:(e + 1) * no, nb * no + Fo * nf: nb * no + (Fo + 1) * nf] -= A_i2o[e][:, F * nf:(F + 1) * nf]
    return G


SWEEP_CORNERS = ("BL", "BR", "TR", "TL")


def sweep_order(mesh: Mesh, corner: str):
    """Elements in wavefront order from one corner of the mesh (bottom-left, top-right,
    bottom-right, top-left): by the sum of the two distances from that corner, element number
    breaking ties.  Neighbours differ by one in that sum, so the elements of one wavefront do not
    touch and every neighbour is either one wavefront earlier (upwind) or one later."""
    E = mesh.n_elems
    ix, iz = np.arange(E) % mesh.nx, np.arange(E) // mesh.nx
    dx = ix if corner in ("BL", "TL") else mesh.nx - 1 - ix
    dz = iz if corner in ("BL", "BR") else mesh.nz - 1 - iz
    return np.argsort(dx + dz, kind="stable")


# The faces (0 bottom, 1 right, 2 top, 3 left) whose outflow travels away from a sweep's corner:
# the downwind faces of the sweep.
SWEEP_DOWNWIND = {"BL": (1, 2), "BR": (3, 2), "TR": (3, 0), "TL": (1, 0)}


def sweep_rows(disc: Disc, corner: str, rows: str):
    """Outflow rows of an element that a sweep from `corner` recomputes: all of them, or those of
    its two downwind faces."""
    if rows == "all":
        return np.arange(disc.n_out)
    nf = disc.n_face
    return np.concatenate([np.arange(F * nf, (F + 1) * nf) for F in SWEEP_DOWNWIND[corner]])


def sweep_precond(mesh: Mesh, disc: Disc, A_i2o, r, corners=SWEEP_CORNERS, rows="downwind"):
    """z = M r: block Gauss-Seidel sweeps of eq. hdg_global_mat, (I - A_int) z = r, from z = 0,
    one sweep per corner in turn.  A sweep visits the elements in wavefront order and replaces
    outflow values of each element by z_K = r_K + A_i2o^K z_in(K), the inflow gathered from the
    current z (already swept neighbours: this sweep's values; the others: the latest earlier
    sweep's, zero before any).  rows = "all": every outflow value of the element; rows = "downwind"
    (the library's): only those of the two faces that point away from the corner, the values the
    sweep's later elements read — each face is then recomputed by two of the four sweeps.  A
    linear operator: the preconditioner of the library's GMRES."""
    E, no = mesh.n_elems, disc.n_out
    r = np.asarray(r, dtype=np.float64).reshape(E, no)
    z = np.zeros((E, no))
    for corner in corners:
        sel = sweep_rows(disc, corner, rows)
        for e in sweep_order(mesh, corner):
            zin = gather_inflow_one(mesh, disc, z, e)
            z[e, sel] = r[e, sel] + A_i2o[e][sel] @ zin
    return z.reshape(-1)


def gather_inflow_one(mesh: Mesh, disc: Disc, x: np.ndarray, e: int):
    """Interior inflow [n_in] of element e from the outflow x [E, n_out] (zero on the boundary)."""
    nf = disc.n_face
    out = np.zeros(disc.n_in)
    for F in range(4):
        nb = mesh.neighbour(e, F)
        if nb >= 0:
            G = OPPOSITE[F]
            out[F * nf:(F + 1) * nf] = x[nb, G * nf:(G + 1) * nf]
    return out


def gmres_right(apply, precond, b, rtol=1e-12, restart=50, max_iter=20000):
    """GMRES on A M y = b, x = M y (right preconditioning: the residual it minimises is the true
    one, b - A x).  Returns (x, iterations, relative residual)."""
    y, it, rel = gmres(lambda v: apply(precond(v)), b, rtol=rtol, restart=restart, max_iter=max_iter)
    return precond(y), it, rel


def gmres(apply, b, rtol=1e-12, restart=50, max_iter=20000, x0=None):
    """Restarted GMRES (Saad & Schultz) with classical Gram-Schmidt applied twice; stops when
    ||b - A x|| <= rtol ||b||.  Returns (x, iterations, relative residual)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    it = 0
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * bn or it >= max_iter:
            return x, it, beta / bn
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        V[0] = r / beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        gvec = np.zeros(restart + 1)
        gvec[0] = beta
        j_done = 0
        for j in range(restart):
            w = apply(V[j])
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            H[:j + 1, j] = h + h2
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            it += 1
            j_done = j + 1
            if abs(gvec[j + 1]) <= rtol * bn or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), gvec[:j_done])
        x = x + V[:j_done].T @ y


# ----------------------------------------------------------------------------------------------
# whole-problem drivers (Algorithm 1)
# ----------------------------------------------------------------------------------------------

def nodal_kappa_hat(problem, disc: Disc, mesh: Mesh):
    """kappa_hat = kappa(x_i) h / 2 at the LGL nodes of every element (Sec. 2.4.1)."""
    x, z = mesh.node_coords(disc)
    return np.asarray(problem.kappa(x, z), dtype=np.float64) * (mesh.h * 0.5)


def build_local(disc: Disc, kappa_hat: np.ndarray, omega: np.ndarray):
    """in2out [E, n_out, n_in] and in2sol (mean) [E, nm, n_in] of every element."""
    E = kappa_hat.shape[0]
    A_i2o = np.zeros((E, disc.n_out, disc.n_in))
    A_i2m = np.zeros((E, disc.nm, disc.n_in))
    for e in range(E):
        A_i2o[e], A_i2m[e], _ = disc.local_operators(kappa_hat[e], float(omega[e]))
    return A_i2o, A_i2m


def solve_problem(problem, rtol=1e-12, dense=None, ops=None, radiance=False):
    """Algorithm 1 on a workload problem. Returns a dict with the skeleton solution, the mean
    intensity [E, nm], the local operators and GMRES statistics.  With a volume source
    (problem.source) the local source terms f^_u, f_u enter the global right-hand side and the
    recovery (eqs. hdg_local_f2u_i2u, hdg_local_f2o_i2o); radiance=True also recovers the radiance
    u_h = A_i2u u^_in + f_u of every element ([E, N, nm])."""
    disc = Disc(problem.p, problem.n_angles, problem.hg_g, problem.angular)
    mesh = Mesh(problem.nx, problem.nz, problem.h)
    kh = nodal_kappa_hat(problem, disc, mesh)
    if ops is None:
        A_i2o, A_i2m = build_local(disc, kh, problem.omega)
    else:
        A_i2o, A_i2m = ops
    E = mesh.n_elems
    f2o = f2m = f2u = None
    if getattr(problem, "source", None) is not None:
        fh = nodal_source_hat(problem, disc, mesh)
        f2o, f2m, f2u = np.zeros((E, disc.n_out)), np.zeros((E, disc.nm)), np.zeros((E, disc.nu))
        for e in range(E):
            f2o[e], f2m[e], f2u[e] = disc.local_source(kh[e], float(problem.omega[e]), fh[e])
    b = global_rhs(mesh, disc, A_i2o, problem.inflow, f2o)
    n = b.size
    if dense is None:
        dense = n <= 4000
    if dense:
        x = np.linalg.solve(global_dense(mesh, disc, A_i2o), b)
        its, rel = 0, np.linalg.norm(b - global_apply(mesh, disc, A_i2o, x)) / max(np.linalg.norm(b), 1e-300)
    else:
        x, its, rel = gmres(lambda v: global_apply(mesh, disc, A_i2o, v), b, rtol=rtol)
    xin = gather_inflow(mesh, disc, x.reshape(mesh.n_elems, disc.n_out), problem.inflow)
    um = np.einsum("eij,ej->ei", A_i2m, xin)
    if f2m is not None:
        um = um + f2m
    out = dict(disc=disc, mesh=mesh, kappa_hat=kh, A_i2o=A_i2o, A_i2m=A_i2m, x=x, u_mean=um,
               iterations=its, rel_residual=rel, f2o=f2o, f2m=f2m, f2u=f2u)
    if radiance:
        u = np.zeros((E, disc.nu))
        for e in range(E):
            _, _, A_i2u = disc.local_operators(kh[e], float(problem.omega[e]))
            u[e] = A_i2u @ xin[e] + (f2u[e] if f2u is not None else 0.0)
        out["radiance"] = u.reshape(E, disc.n_angles, disc.nm)
    return out


def dg_direct_radiance(problem):
    """Upwind DG (eqs. dg, dg_flux; a volume source f enters as F of each element) assembled over the
    whole mesh and solved densely; returns the radiance [E, N, nm].  Tiny meshes only; used to check
    the hybridised path."""
    disc = Disc(problem.p, problem.n_angles, problem.hg_g, problem.angular)
    mesh = Mesh(problem.nx, problem.nz, problem.h)
    kh = nodal_kappa_hat(problem, disc, mesh)
    E, nu, nm, half = mesh.n_elems, disc.nu, disc.nm, problem.n_angles // 2
    G = np.zeros((E * nu, E * nu))
    rhs = np.zeros(E * nu)
    offs, _ = inflow_side_offsets(mesh, disc)
    fh = nodal_source_hat(problem, disc, mesh) if getattr(problem, "source", None) is not None else None
    for e in range(E):
        A, _ = disc.local_system(kh[e], float(problem.omega[e]))
        G[e * nu:(e + 1) * nu, e * nu:(e + 1) * nu] = A
        if fh is not None:
            rhs[e * nu:(e + 1) * nu] += disc.source_vector(fh[e])
        for F in range(4):
            nb = mesh.neighbour(e, F)
            for m, node in enumerate(disc.face_nodes[F]):
                for kk, k in enumerate(disc.in_cells[F]):
                    row = e * nu + k * nm + node
                    coef = disc.w[m] * disc.s_dot_n[F, k]          # (s.n) uhat v with uhat upwind
                    if nb >= 0:
                        nbnode = disc.face_nodes[OPPOSITE[F]][m]
                        G[row, nb * nu + k * nm + nbnode] += coef
                    else:
                        gval = problem.inflow[offs[F] + mesh.boundary_face(e, F) * disc.n_face + m * half + kk]
                        rhs[row] -= coef * gval
    return np.linalg.solve(G, rhs).reshape(E, problem.n_angles, nm)


def dg_direct(problem):
    """Mean intensity [E, nm] of the direct upwind-DG solve (dg_direct_radiance)."""
    return dg_direct_radiance(problem).mean(axis=1)


def exact_transport_mean(problem, disc: Disc, mesh: Mesh, kappa: float, ref=(0.0, 0.0)):
    """Mean over cells of u_k(x) = exp(-kappa sbar_k.(x - ref) / |sbar_k|^2): the exact solution of the
    angle-discrete equation sbar_k . grad u + kappa u = 0 with that inflow (no scattering)."""
    x, z = mesh.node_coords(disc)
    u = 0.0
    for k in range(disc.n_angles):
        s2 = disc.sx[k] ** 2 + disc.sz[k] ** 2
        u = u + np.exp(-kappa * (disc.sx[k] * (x - ref[0]) + disc.sz[k] * (z - ref[1])) / s2)
    return u / disc.n_angles


def exact_transport_inflow(disc: Disc, mesh: Mesh, kappa: float, ref=(0.0, 0.0)):
    """Inflow data (nodal values at the boundary face nodes) of the exact solution above."""
    offs, total = inflow_side_offsets(mesh, disc)
    g = np.zeros(total)
    half = disc.n_angles // 2
    L = (mesh.nx * mesh.h, mesh.nz * mesh.h)
    pos = (disc.xi + 1.0) * 0.5 * mesh.h
    for F in range(4):
        nfaces = mesh.nx if F in (0, 2) else mesh.nz
        for f in range(nfaces):
            for m in range(disc.n1):
                if F == 0:
                    px, pz = f * mesh.h + pos[m], 0.0
                elif F == 1:
                    px, pz = L[0], f * mesh.h + pos[m]
                elif F == 2:
                    px, pz = f * mesh.h + pos[m], L[1]
                else:
                    px, pz = 0.0, f * mesh.h + pos[m]
                for kk, k in enumerate(disc.in_cells[F]):
                    s2 = disc.sx[k] ** 2 + disc.sz[k] ** 2
                    g[offs[F] + f * disc.n_face + m * half + kk] = math.exp(
                        -kappa * (disc.sx[k] * (px - ref[0]) + disc.sz[k] * (pz - ref[1])) / s2)
    return g


def exact_unit_square_mean(problem, disc: Disc, mesh: Mesh, kappa: float):
    """Mean intensity of the exact solution for unit downward inflow on the top only: in cell k
    (downward) u = exp(-kappa * path length back to the top) if the back-traced ray leaves through
    the top, 0 if it leaves through a side; upward cells carry 0."""
    x, z = mesh.node_coords(disc)
    Lx, Lz = mesh.nx * mesh.h, mesh.nz * mesh.h
    u = np.zeros_like(x)
    for k in range(disc.n_angles):
        sx, sz = disc.sx[k], disc.sz[k]
        if sz >= 0:
            continue
        t_top = (Lz - z) / (-sz)                      # parameter back to z = Lz along -s
        if sx > 0:
            t_side = x / sx
        else:
            t_side = (Lx - x) / (-sx)
        # along x + t sbar the solution decays like exp(-kappa t), so u(x) = exp(-kappa t_top)
        u = u + np.where(t_top <= t_side, np.exp(-kappa * t_top), 0.0)
    return u / disc.n_angles


def rel_l2(u, ref, disc: Disc):
    """Relative L2 error with the LGL quadrature weights of every element (uniform h cancels)."""
    w = disc.w2[None, :]
    return math.sqrt(np.sum(w * (u - ref) ** 2) / np.sum(w * ref ** 2))
