"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle's tests.

This module only *generates* particle positions (and small hand-made tetrahedra).
It contains none of the deposit arithmetic: no tessellation, no clipping, no
volumes.  Both sides of every parity test read their inputs from here.
"""
from .lattice import (  # noqa: F401
    CONFIGS,
    WorkloadConfig,
    collapse_positions,
    config_positions,
    jitter_positions,
    lattice_positions,
    random_dyadic_tets,
    zeldovich_positions,
    zeldovich_positions_device,
)
