"""Seeded synthetic H-CRAN instances (channel gains and system constants).

This package only draws inputs: node/user geometry, path loss, shadowing and
Rayleigh fading, plus the constant system parameters of each workload.  It
holds none of the resource-allocation arithmetic, so both the FP64 oracle and
the CUDA solver can be fed from it without sharing any solver code.
"""
from .gen import (  # noqa: F401
    SCENARIOS,
    Instance,
    Tolerances,
    WORKLOADS,
    make_instance,
    make_workload,
    pack_batch,
    splitmix64_uniform,
)
