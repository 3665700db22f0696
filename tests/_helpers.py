"""Shared test utilities: seeded inputs for the library (at the library's own node coordinates)
and for the oracle (at the oracle's own node coordinates)."""

from __future__ import annotations

import dataclasses

import numpy as np

import workloads as W


def small_cloud(nx, nz, p, n_angles, omega=0.99, g=0.85, angular="fv0", theta=300.0, random_inflow=False, seed=7):
    """A Gaussian cloud on an nx x nz mesh of 10/max(nx,nz) km elements with a solar beam on top."""
    h = 10.0 / max(nx, nz)
    cloud = W.GaussianClouds(0.1, np.array([12.0, 6.0]), np.array([[0.45 * nx * h, 0.5 * nz * h],
                                                                  [0.7 * nx * h, 0.3 * nz * h]]),
                             np.array([0.25 * nx * h, 0.15 * nx * h]))
    if random_inflow:
        _, total = W.inflow_layout(nx, nz, p, n_angles)
        g_in = np.random.default_rng(seed).uniform(0, 1, total)
    else:
        g_in = W.beam_inflow(nx, nz, p, n_angles, theta)
    return W.Problem("small-cloud", nx, nz, h, p, n_angles, g, np.full(nx * nz, omega), cloud, g_in, angular)


def random_elements(n, p, seed, kmax=20.0):
    """Per-node kappa in km^-1 (lognormal) and albedo per element, with element side h = 0.2 km."""
    r = np.random.default_rng(seed)
    kappa = np.exp(r.uniform(np.log(0.05), np.log(kmax), size=(n, (p + 1) ** 2)))
    omega = r.uniform(0.8, 1.0, n)
    return kappa, omega, 0.2


def lib_kappa(problem):
    """kappa at the library's LGL nodes (library node coordinates, workload field)."""
    import paper_2308_02467_gb300 as E
    x, z = E.elrt_node_coords(problem.p, problem.n_angles, problem.nx, problem.nz, problem.h)
    return problem.kappa(x, z)


def ang_code(problem):
    return 0 if problem.angular == "fv0" else 1


def gpu_pipeline(problem, mode, out_dtype, rtol=1e-12, refine_steps=2, restart=50, max_iter=20000, krylov_op=None):
    """Algorithm 1 through the C ABI: local operators, global GMRES, mean recovery."""
    import torch
    import paper_2308_02467_gb300 as E
    ctx = E.Context(problem.p, problem.n_angles, problem.hg_g, ang_code(problem))
    if krylov_op is not None:
        ctx.elrt_set_krylov_op(krylov_op)
    dev = "cuda"
    kappa = torch.tensor(lib_kappa(problem), device=dev, dtype=torch.float64).contiguous()
    omega = torch.tensor(problem.omega, device=dev, dtype=torch.float64)
    Ne = problem.nx * problem.nz
    dt = torch.float32 if out_dtype == E.F32 else torch.float64
    in2out = torch.empty(Ne, ctx.nin, ctx.nin, device=dev, dtype=dt)
    in2sol = torch.empty(Ne, ctx.nm, ctx.nin, device=dev, dtype=dt)
    lst = ctx.elrt_build_local(kappa, omega, problem.h, in2out, in2sol, mode=mode, refine_steps=refine_steps)
    g = torch.tensor(problem.inflow, device=dev, dtype=torch.float64)
    x = torch.empty(Ne * ctx.nin, device=dev, dtype=torch.float64)
    gst = ctx.elrt_solve_global(problem.nx, problem.nz, in2out, g, x, rtol=rtol, restart=restart, max_iter=max_iter)
    mean = torch.empty(Ne, ctx.nm, device=dev, dtype=torch.float64)
    ctx.elrt_recover_mean(problem.nx, problem.nz, in2sol, x, g, mean)
    torch.cuda.synchronize()
    out = dict(in2out=in2out.double().cpu().numpy(), in2sol=in2sol.double().cpu().numpy(),
               x=x.cpu().numpy(), u_mean=mean.cpu().numpy(), local_stats=lst, solve_stats=gst)
    ctx.close()
    return out


def energy_defect(w, sdn, in_cells, out_cells, w2, kappa_hat, omega, n_angles, A_i2o, A_i2m):
    """Energy balance of one element's operators (test function v = 1), relative per inflow column.
    Written here independently of the oracle so it can be applied to library outputs."""
    n1 = len(w)
    lhs = np.array([w[m] * abs(sdn[F][k]) for F in range(4) for m in range(n1) for k in in_cells[F]])
    wout = np.array([w[m] * sdn[F][k] for F in range(4) for m in range(n1) for k in out_cells[F]])
    rhs = wout @ A_i2o + n_angles * (w2 * kappa_hat * (1 - omega)) @ A_i2m
    return (lhs - rhs) / lhs


def with_(problem, **kw):
    return dataclasses.replace(problem, **kw)


def thick_and_thin_elements(n, p, seed):
    """Per-node kappa spanning 1e-3 .. 1e4 km^-1 (a log-uniform element mean with +-0.5 per-node
    log variation) at sides h ~ U[0.05, 1] km, so kappa_hat = kappa h / 2 covers ~1e-5 .. 5e3; the
    first two elements are the extremes: kappa_hat = 1.5e3 and 1e-4 everywhere.  Albedo U[0.9, 1]."""
    r = np.random.default_rng(seed)
    nm = (p + 1) ** 2
    h = r.uniform(0.05, 1.0, n)
    mu = r.uniform(np.log(1e-3), np.log(1e4), n)
    kappa = np.exp(mu[:, None] + r.uniform(-0.5, 0.5, (n, nm)))
    h[0], kappa[0] = 1.0, 3.0e3
    h[1], kappa[1] = 0.2, 1.0e-3
    omega = r.uniform(0.9, 1.0, n)
    return kappa, omega, h


def lib_source(problem):
    """The problem's volume source at the library's LGL nodes, [E][N][nm] (cell k, node i)."""
    import paper_2308_02467_gb300 as E
    x, z = E.elrt_node_coords(problem.p, problem.n_angles, problem.nx, problem.nz, problem.h)
    return np.ascontiguousarray(np.transpose(problem.source(x, z), (0, 2, 1)))
