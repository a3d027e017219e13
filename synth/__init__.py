"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side
tests and bench.

This package holds only input generation: design matrices A and responses b
shaped like the tall-and-skinny regression workloads the method is evaluated
on.  It holds none of the method's arithmetic (no transform, no draw of the
method's own random variables, no sampling).
"""
from .inputs import (  # noqa: F401
    Workload,
    WORKLOADS,
    make_problem,
    make_batched_problems,
    kappa_test_matrix,
    canonical_design,
    r1_for,
)
