"""Seeded synthetic inputs for the RGF hot path.

This package only draws random numbers and lays them out as arrays (block-tridiagonal
Hamiltonians, alloy masks, energy and k grids, potentials).  It contains none of the
Green's-function arithmetic; both the CPU oracle (through the tests) and the CUDA path
consume what it produces.
"""
from .synth import (  # noqa: F401
    Device,
    make_device,
    hamiltonian_k,
    chain_device,
    channel_device,
    energy_grid_linspace,
    energy_grid_uniform,
    k_grid,
    random_potential,
    config_workload,
    CONFIGS,
)
