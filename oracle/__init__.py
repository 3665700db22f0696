"""FP64 CPU oracle of the element method.  TEST INFRASTRUCTURE ONLY.

Only the tests, the entry point's smoke check and the benchmark's CPU-baseline
and reference legs may import this package.  The library never calls it and
shares no code with it: the oracle computes its own LGL nodes, directions,
phase matrix, element matrices, DOF maps and global solve, in plain numpy
FP64, following the paper's equations step by step.

Modules
-------
hdg   classical method: Sec. 2.2 (eqs. dg, hdg_local, hdg_local_mat,
      hdg_local_i2u, hdg_local_i2o, hdg_global_mat), Sec. 2.4 (eq. ang_ave),
      Appendix A, plus the direct upwind-DG solve used as a pin.
mlp   the element network of Sec. 2.4.1 (fully connected, linear output)
      with its backward pass, MAE loss and Adam step.

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, exact discrete identities or brute force, except the learned
operators themselves (parity unpinned beyond the classical labels: the paper
gives no trained weights).
"""
