"""Seeded synthetic inputs shared by the tests, the oracle runs and the bench.

This package holds input generation only: surfaces, the discrete operators that
assemble A = M + t L (Sec. 5.2), the right-hand sides, and the host hierarchy
builder of Sec. 4 whose prolongations P_l are an input of the multigrid solve.
It contains none of the solve's arithmetic (Galerkin products, smoothing,
residuals, transfers, coarse solves), which the oracle and the CUDA library
each implement on their own.
"""
from .hierarchy import Prolongation, build_hierarchy, build_level, compile_builder  # noqa: F401
from .workloads import (System, cached, cached_batch, cloud_system, heat_system, icosphere_system,  # noqa: F401
                        is_cached, nonmanifold_system, spheres_batch, torus_system, workload)
