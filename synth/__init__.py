"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds random-number draws only: microstructures (phase images), macroscopic
load cases and random test fields.  It contains none of the solver's arithmetic, so the
oracle and the CUDA path stay independent while reading the same inputs.
"""
from .microstructure import (  # noqa: F401
    rsa_spheres,
    rsa_disks,
    random_phase,
    laminate,
    random_field,
    unit_loads,
    config_seed,
    workload,
)
