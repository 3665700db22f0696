"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package holds no arithmetic of the element method itself: it only draws
random numbers (numpy's counter-based Philox generator) and defines optical
fields kappa(x, z) and volume sources f(x, z) as plain functions of physical
coordinates, plus the boundary inflow data of each workload.  Whoever needs kappa at the LGL nodes
of an element evaluates these functions at its own node coordinates.
"""

from .fields import (  # noqa: F401
    SEED_BASE,
    philox,
    Problem,
    GaussianClouds,
    LognormalSlab,
    IsotropicEmission,
    BeamLikeSource,
    ElementBatch,
    inflow_layout,
    beam_inflow,
    downward_unit_inflow,
    problem_unit_square,
    problem_gaussian_slab,
    problem_batch_fields,
    problem_cloud_slab,
    element_batch,
    ModalSampleBatch,
    modal_sample_batch,
)
