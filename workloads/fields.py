"""Seeded optical fields, element batches and boundary inflow data.

Everything here is problem *data*: random draws from numpy's Philox generator
and closed-form fields kappa(x, z) in km^-1 on the x-z plane (z points up).
Nothing here discretises the transport equation.

Inflow array layout (the layout the library's C ABI and the oracle both take):
the four sides of the rectangular domain in the order bottom, right, top,
left; a side is a run of boundary faces (bottom/top: nx faces left to right;
right/left: nz faces bottom to top); each face holds p+1 node values in the
order of increasing coordinate along the face; each node holds the N/2 angular
cells that point *into* the domain through that side, in increasing cell
index k, cell k being the angle interval [k*2pi/N, (k+1)*2pi/N).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

SEED_BASE = 2308024670  # seed of workload c is SEED_BASE + c


def philox(config_index: int, stream: int = 0) -> np.random.Generator:
    """Counter-based generator for one workload; `stream` selects an independent counter block."""
    return np.random.Generator(np.random.Philox(key=SEED_BASE + config_index, counter=[0, 0, stream, 0]))


# ----------------------------------------------------------------------------------------------
# boundary inflow data
# ----------------------------------------------------------------------------------------------

def _entering_cells(side: int, n_angles: int) -> list[int]:
    """Angular cells whose directions enter the domain through `side` (0 bottom,1 right,2 top,3 left)."""
    q = n_angles // 4
    if side == 0:      # through the bottom: upward cells
        return list(range(0, 2 * q))
    if side == 1:      # through the right side: cells pointing to -x
        return list(range(q, 3 * q))
    if side == 2:      # through the top: downward cells
        return list(range(2 * q, 4 * q))
    return list(range(0, q)) + list(range(3 * q, 4 * q))  # through the left side: cells pointing to +x


def inflow_layout(nx: int, nz: int, p: int, n_angles: int) -> tuple[list[int], int]:
    """Offsets of the four sides in the inflow array and its total length."""
    per_face = (p + 1) * (n_angles // 2)
    counts = [nx, nz, nx, nz]
    offs, o = [], 0
    for c in counts:
        offs.append(o)
        o += c * per_face
    return offs, o


def beam_inflow(nx, nz, p, n_angles, theta_deg, sides=(2,), amplitude=None) -> np.ndarray:
    """Collimated beam of direction theta entering through `sides`.

    The beam is represented by its angular-cell projection: the whole cell that
    contains theta (cell k with k*dtheta <= theta < (k+1)*dtheta) carries
    N/(2 pi) so that the angular integral of the inflow is 1; every other cell is 0.
    """
    offs, total = inflow_layout(nx, nz, p, n_angles)
    g = np.zeros(total)
    kb = math.floor(round(theta_deg * n_angles / 360.0, 9)) % n_angles
    amp = n_angles / (2 * math.pi) if amplitude is None else amplitude
    half = n_angles // 2
    for s in sides:
        cells = _entering_cells(s, n_angles)
        if kb not in cells:
            raise ValueError(f"beam cell {kb} does not enter through side {s}")
        kk = cells.index(kb)
        nf = nx if s in (0, 2) else nz
        blk = g[offs[s]: offs[s] + nf * (p + 1) * half].reshape(nf, p + 1, half)
        blk[:, :, kk] = amp
    return g


def downward_unit_inflow(nx, nz, p, n_angles) -> np.ndarray:
    """Unit radiance in every downward cell on the top side, zero elsewhere."""
    offs, total = inflow_layout(nx, nz, p, n_angles)
    g = np.zeros(total)
    g[offs[2]: offs[2] + nx * (p + 1) * (n_angles // 2)] = 1.0
    return g


# ----------------------------------------------------------------------------------------------
# optical fields
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class GaussianClouds:
    """kappa = kappa0 + sum_c A_c exp(-|x - x_c|^2 / (2 w_c^2))   [km^-1]."""
    kappa0: float
    amps: np.ndarray
    centres: np.ndarray  # [C, 2] (x, z) km
    widths: np.ndarray

    def __call__(self, x, z):
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        k = np.full(np.broadcast(x, z).shape, self.kappa0)
        for a, (cx, cz), w in zip(self.amps, self.centres, self.widths):
            k = k + a * np.exp(-((x - cx) ** 2 + (z - cz) ** 2) / (2.0 * w * w))
        return k


@dataclasses.dataclass
class LognormalSlab:
    """kappa = kappa_bg + mask(x, z) * exp(mu + sd * f(x, z)).

    f is a unit-variance Gaussian random field with Gaussian covariance of
    correlation length `ell`, realised by random Fourier features
    f = sqrt(2/M) sum_j cos(k_j . x + b_j), k_j ~ N(0, I/ell^2), b_j ~ U[0, 2pi).
    The mask is a product of four tanh ramps of width `edge` around the box
    [x0, x1] x [z0, z1].
    """
    kappa_bg: float
    mu: float
    sd: float
    wavevectors: np.ndarray  # [M, 2]
    phases: np.ndarray       # [M]
    box: tuple
    edge: float

    def grf(self, x, z):
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        shape = np.broadcast(x, z).shape
        xf = np.broadcast_to(x, shape).reshape(-1)
        zf = np.broadcast_to(z, shape).reshape(-1)
        m = len(self.phases)
        out = np.zeros(xf.shape)
        for s in range(0, xf.size, 8192):
            arg = (np.outer(xf[s:s + 8192], self.wavevectors[:, 0])
                   + np.outer(zf[s:s + 8192], self.wavevectors[:, 1]) + self.phases)
            out[s:s + 8192] = np.cos(arg).sum(axis=1) * math.sqrt(2.0 / m)
        return out.reshape(shape)

    def mask(self, x, z):
        x0, x1, z0, z1 = self.box
        e = self.edge
        return (0.5 * (1 + np.tanh((x - x0) / e)) * 0.5 * (1 + np.tanh((x1 - x) / e))
                * 0.5 * (1 + np.tanh((z - z0) / e)) * 0.5 * (1 + np.tanh((z1 - z) / e)))

    def __call__(self, x, z):
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        return self.kappa_bg + self.mask(x, z) * np.exp(self.mu + self.sd * self.grf(x, z))

    def evaluate_torch(self, x, z, chunk=16384):
        """The same field evaluated with torch (FP64) on the device of the 1-D tensors x, z: the
        512 x 256 slab has 6.4 M nodes x 4096 modes, too many cosines for numpy."""
        import torch
        dev = x.device
        kv = torch.as_tensor(self.wavevectors, dtype=torch.float64, device=dev)
        ph = torch.as_tensor(self.phases, dtype=torch.float64, device=dev)
        scale = math.sqrt(2.0 / len(self.phases))
        x0, x1, z0, z1 = self.box
        e = self.edge
        out = torch.empty_like(x, dtype=torch.float64)
        for s in range(0, x.numel(), chunk):
            xs, zs = x[s:s + chunk].double(), z[s:s + chunk].double()
            arg = torch.outer(xs, kv[:, 0]) + torch.outer(zs, kv[:, 1]) + ph
            f = torch.cos(arg).sum(dim=1) * scale
            mask = (0.5 * (1 + torch.tanh((xs - x0) / e)) * 0.5 * (1 + torch.tanh((x1 - xs) / e))
                    * 0.5 * (1 + torch.tanh((zs - z0) / e)) * 0.5 * (1 + torch.tanh((z1 - zs) / e)))
            out[s:s + chunk] = self.kappa_bg + mask * torch.exp(self.mu + self.sd * f)
        return out


@dataclasses.dataclass
class IsotropicEmission:
    """Thermal emission, the same in every angular cell: f(x, z) = (1 - omega) kappa(x, z) B(z) with a
    source function rising linearly with height, B(z) = b0 + b1 z / height."""
    kappa: Callable
    omega: float
    b0: float
    b1: float
    height: float
    n_angles: int

    def __call__(self, x, z):
        f = (1.0 - self.omega) * self.kappa(x, z) * (self.b0 + self.b1 * np.asarray(z, dtype=np.float64) / self.height)
        return np.repeat(np.asarray(f)[..., None], self.n_angles, axis=-1)


@dataclasses.dataclass
class BeamLikeSource:
    """An angle-dependent volume source peaked around direction theta0: f(x, z, cell k) =
    a exp(-|x - c|^2 / (2 w^2)) (1 + cos(theta_k - theta0)), theta_k the centre of cell k."""
    amplitude: float
    centre: tuple
    width: float
    theta0: float
    n_angles: int

    def __call__(self, x, z):
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        blob = self.amplitude * np.exp(-((x - self.centre[0]) ** 2 + (z - self.centre[1]) ** 2) / (2 * self.width ** 2))
        th = (np.arange(self.n_angles) + 0.5) * 2 * math.pi / self.n_angles
        return blob[..., None] * (1.0 + np.cos(th - self.theta0))


# ----------------------------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """One steady transport problem on a uniform nx x nz grid of square elements of side h (km)."""
    name: str
    nx: int
    nz: int
    h: float
    p: int
    n_angles: int
    hg_g: float
    omega: np.ndarray                         # single-scattering albedo per element [nx*nz]
    kappa: Callable                           # kappa(x, z) in km^-1
    inflow: np.ndarray                        # boundary inflow, layout described in the module doc
    angular: str = "fv0"                      # "fv0" (cell-averaged directions) or "do" (cell centres)
    source: Callable | None = None            # volume source f(x, z) -> [..., N] per angular cell, or None

    @property
    def n_elems(self) -> int:
        return self.nx * self.nz


def problem_unit_square(p=4, n_angles=8, n=4, kappa=1.0, angular="fv0") -> Problem:
    """Unit square, n x n elements, constant kappa, no scattering, unit downward inflow on top."""
    return Problem("unit-square", n, n, 1.0 / n, p, n_angles, 0.0, np.zeros(n * n),
                   lambda x, z: np.full(np.broadcast(np.asarray(x), np.asarray(z)).shape, float(kappa)),
                   downward_unit_inflow(n, n, p, n_angles), angular)


def problem_gaussian_slab(n=64, p=6, n_angles=16) -> Problem:
    """10 km x 10 km slab, one Gaussian cloud 0.1 + 20 exp(-r^2/(2*1.5^2)) at the centre,
    albedo 0.99, g=0.85, solar beam 30 deg from zenith towards +x (direction 300 deg) on top."""
    cloud = GaussianClouds(0.1, np.array([20.0]), np.array([[5.0, 5.0]]), np.array([1.5]))
    return Problem("gaussian-slab", n, n, 10.0 / n, p, n_angles, 0.85, np.full(n * n, 0.99), cloud,
                   beam_inflow(n, n, p, n_angles, 300.0), "fv0")


def problem_batch_fields(n_fields=256, n_angles=16, first=0) -> list[Problem]:
    """Independent fields with seed-drawn mesh sizes in {16..128}^2 and p in {4,6,8}; each a sum of
    1-5 Gaussian clouds (amplitude U[1,30], width U[0.5,3] km) on kappa0 = 0.1, albedo U[0.9,1]."""
    out = []
    for i in range(first, first + n_fields):
        r = philox(3, stream=i)
        nx, nz = (int(v) for v in r.integers(16, 129, size=2))
        p = int(r.choice([4, 6, 8]))
        omega = float(r.uniform(0.9, 1.0))
        h = 10.0 / max(nx, nz)
        lx, lz = nx * h, nz * h
        nc = int(r.integers(1, 6))
        cloud = GaussianClouds(0.1, r.uniform(1.0, 30.0, nc),
                               np.stack([r.uniform(0, lx, nc), r.uniform(0, lz, nc)], axis=1),
                               r.uniform(0.5, 3.0, nc))
        out.append(Problem(f"field-{i}", nx, nz, h, p, n_angles, 0.85, np.full(nx * nz, omega), cloud,
                           beam_inflow(nx, nz, p, n_angles, 300.0), "fv0"))
    return out


def problem_cloud_slab(nx=512, nz=256, p=6, n_angles=16, modes=4096) -> Problem:
    """50 km x 25 km slab: lognormal cloud (log-mean 2, log-sd 1, correlation 2 km) inside a
    tanh-edged box (edge width 50 m) on kappa = 0.02; albedo 0.99, g=0.85, beam at 45 deg (315 deg)."""
    r = philox(5)
    ell = 2.0
    field = LognormalSlab(0.02, 2.0, 1.0, r.normal(0.0, 1.0 / ell, size=(modes, 2)),
                          r.uniform(0.0, 2 * math.pi, modes), (5.0, 45.0, 5.0, 15.0), 0.05)
    h = 50.0 / nx
    return Problem("cloud-slab", nx, nz, h, p, n_angles, 0.85, np.full(nx * nz, 0.99), field,
                   beam_inflow(nx, nz, p, n_angles, 315.0), "fv0")


# ----------------------------------------------------------------------------------------------
# independent elements for the element network
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class ElementBatch:
    """Independent square elements of side h with lognormal kappa and albedo.

    log kappa(x) = mu + sd * f(x), f a unit-variance Gaussian-covariance random field of
    correlation length ell realised by `modes` random Fourier features per element; x is the
    physical offset from the element centre, x = (h/2) * xi for reference coordinates xi.
    """
    h: np.ndarray        # [n]
    ell: np.ndarray      # [n]
    mu: np.ndarray       # [n]
    sd: np.ndarray       # [n]
    omega: np.ndarray    # [n]
    wavevectors: np.ndarray  # [n, M, 2] (already divided by ell)
    phases: np.ndarray       # [n, M]

    def __len__(self):
        return len(self.h)

    def kappa_at(self, xi_x: np.ndarray, xi_z: np.ndarray) -> np.ndarray:
        """kappa [n, P] at reference points (xi_x[P], xi_z[P]) of every element (km^-1)."""
        hx = (self.h[:, None] * 0.5) * np.asarray(xi_x)[None, :]
        hz = (self.h[:, None] * 0.5) * np.asarray(xi_z)[None, :]
        m = self.phases.shape[1]
        arg = (hx[:, :, None] * self.wavevectors[:, None, :, 0] + hz[:, :, None] * self.wavevectors[:, None, :, 1]
               + self.phases[:, None, :])
        f = np.cos(arg).sum(axis=2) * math.sqrt(2.0 / m)
        return np.exp(self.mu[:, None] + self.sd[:, None] * f)


@dataclasses.dataclass
class ModalSampleBatch:
    """Optical-coefficient samples on the reference element [-1, 1]^2 drawn by the paper's data
    generation (Sec. 2.4.2, Algorithm 2): Legendre-modal coefficients with a low-frequency bias,
    sigma~_mn = exp(-c_sm ((m/p)^2 + (n/p)^2)) (X_mn - 1/2) with X_mn ~ U[0, 1] (the '+' between the
    two squares is the reading taken where the printed formula has '-', which would favour high
    frequencies in y); their nodal values at the points a caller gives, shifted to a minimum of 0,
    divided by their maximum and multiplied by X_A ~ U[0, A_sigma]."""
    modal: np.ndarray       # [n, p+1 (m, along x), p+1 (n, along z)] biased modal coefficients
    amplitude: np.ndarray   # [n] X_A

    def __len__(self):
        return len(self.amplitude)

    def sigma_at(self, xi: np.ndarray) -> np.ndarray:
        """Nodal sigma [n, (p+1)^2] at the tensor points (xi_a, xi_b), node a + (p+1) b."""
        from numpy.polynomial import legendre
        xi = np.asarray(xi, dtype=np.float64)
        V = legendre.legvander(xi, self.modal.shape[1] - 1)              # V[a][m] = L_m(xi_a)
        s = np.einsum("am,emn,bn->eba", V, self.modal, V)                 # [n][b][a]
        s = s.reshape(len(self), -1)
        s = s - s.min(axis=1, keepdims=True)
        s = s / s.max(axis=1, keepdims=True)
        return s * self.amplitude[:, None]


def modal_sample_batch(n: int, p: int = 6, c_sm: float = 2.0, a_sigma: float = 10.0, holdout: bool = False):
    """n samples of Algorithm 2 (the paper's training set: c_sm = 2, A_sigma = 10, Q_6); the held-out
    set comes from an independent counter block."""
    r = philox(6, stream=1 if holdout else 0)
    m = np.arange(p + 1) / p
    decay = np.exp(-c_sm * (m[:, None] ** 2 + m[None, :] ** 2))
    X = r.uniform(0.0, 1.0, size=(n, p + 1, p + 1))
    return ModalSampleBatch(decay[None] * (X - 0.5), r.uniform(0.0, a_sigma, n))


def element_batch(n: int, holdout: bool = False, modes: int = 64, chunk: int = 4096) -> ElementBatch:
    """n training (or, with holdout=True, held-out) elements: h ~ U[0.05,1] km, ell = U[0.1,2] h,
    log-mean U[-2,3.5], log-sd U[0,1.5], albedo U[0.9,1]."""
    parts = []
    base = 1_000_000 if holdout else 0
    for c in range(0, n, chunk):
        m = min(chunk, n - c)
        r = philox(4, stream=base + c // chunk)
        h = r.uniform(0.05, 1.0, m)
        ell = r.uniform(0.1, 2.0, m) * h
        mu = r.uniform(-2.0, 3.5, m)
        sd = r.uniform(0.0, 1.5, m)
        om = r.uniform(0.9, 1.0, m)
        kv = r.normal(0.0, 1.0, size=(m, modes, 2)) / ell[:, None, None]
        ph = r.uniform(0.0, 2 * math.pi, size=(m, modes))
        parts.append((h, ell, mu, sd, om, kv, ph))
    cat = [np.concatenate([p[i] for p in parts]) for i in range(7)]
    return ElementBatch(*cat)
