"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This package only evaluates the coefficient functions of the workloads on
the grid and draws seeded random numbers.  It contains none of the method's
arithmetic (no L1 weights, no fractional coefficients, no operator): data
that need a solve of the discretised problem (for example mu from a fixed
source f) are produced by whoever consumes these inputs.
"""
from .synthetic import (  # noqa: F401
    Workload,
    config_small_1d,
    config_2d,
    config_3d,
    config_adjoint_2d,
    config_batch,
    paper_1d,
    paper_2d,
    add_noise_gaussian,
    add_noise_uniform,
    random_vector,
    CONFIG_SEED_BASE,
)
