#!/usr/bin/env python
"""Writes the expected mean intensity of the 64 x 64 Gaussian-cloud slab (the benchmark workload:
10 km x 10 km, p = 6, N = 16, g = 0.85, albedo 0.99, beam at 300 deg on top) from the FP64 oracle
alone: dense LU per element (eq. hdg_local_i2u), restriction (eqs. hdg_local_i2o, ang_ave),
GMRES(50) with classical Gram-Schmidt twice on eq. hdg_global_mat to a relative residual of 1e-12,
and the recovery of Algorithm 1.

    python tests/golden/make_gaussian_slab_golden.py

Output: gaussian_slab_64x64_mean.npy ([4096, 49] float64, element e = ix + 64 iz, node
a + 7 b) and gaussian_slab_64x64_mean.json (solver statistics and the file's SHA-256).
Takes a few minutes on a multi-core host.
"""

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import hdg  # noqa: E402


def main():
    prob = W.problem_gaussian_slab(n=64)
    t0 = time.time()
    ref = hdg.solve_problem(prob, rtol=1e-12)
    path = os.path.join(HERE, "gaussian_slab_64x64_mean.npy")
    np.save(path, ref["u_mean"])
    with open(path, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    meta = {"workload": "gaussian-cloud slab 64x64 elements, p=6, N=16, g=0.85, albedo 0.99, beam 300 deg",
            "quantity": "mean intensity u^m at the LGL nodes, [element][node]", "dtype": "float64",
            "shape": list(ref["u_mean"].shape), "gmres_restart": 50, "gmres_rtol": 1e-12,
            "gmres_iterations": int(ref["iterations"]), "rel_residual": float(ref["rel_residual"]),
            "sha256": digest, "seconds": round(time.time() - t0, 1),
            "command": "python tests/golden/make_gaussian_slab_golden.py"}
    with open(os.path.join(HERE, "gaussian_slab_64x64_mean.json"), "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
