"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds the sparse SPD matrices, the box permutation P and the
right-hand sides.  It holds none of the compress-and-eliminate arithmetic: the
oracle (``oracle/``) and the CUDA path (``paper_1603_09133_gb300``) each take
its output as plain arrays.
"""
from .grids import (  # noqa: F401
    poisson2d,
    poisson3d,
    diffusion2d,
    diffusion3d_tensor,
    grf2d,
    box_perm,
    rhs,
    Workload,
    make_workload,
    WORKLOADS,
    BATCH_SIDES,
    make_batch,
)
