"""Seeded synthetic workloads shared by the FP64 oracle tests, the GPU tests and the benchmark.

This package holds input recipes only: random Gaussian clouds, phantoms, motion fields, breathing
surrogates and scan geometry. It contains none of the method's arithmetic (no B-spline evaluation,
no deformation, no projection), so neither the oracle nor the CUDA path depends on the other through it.
"""
from .workloads import (  # noqa: F401
    Workload,
    circular_views,
    tiny,
    thorax,
    thorax_batch,
    scale,
    random_grad_proj,
)
