"""Seeded synthetic voxel structures and load cases.

This module produces INPUTS only: binary solid masks, per-voxel Young's moduli,
Poisson ratios, Cartesian subdomain counts and boundary-condition descriptions.
It holds none of the preconditioner's arithmetic, so both the CPU oracle and the
CUDA library can consume its output without sharing any method code.
"""
from .voxels import (  # noqa: F401
    FACES,
    Problem,
    bcs_clamped_traction,
    bcs_dict_to_arrays,
    make_workload,
    porous_mask,
    lognormal_modulus,
    WORKLOADS,
)
