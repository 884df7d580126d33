"""Seeded synthetic transmission grids (inputs only).

This package draws the bus/branch data that both the CUDA path and the CPU
oracle consume.  It holds none of the method's arithmetic: no admittance
matrix, no power flow, no factorisation -- only random geometry, topology and
electrical parameters.
"""
from .synth import CONFIGS, Grid, config_grid, make_grid

__all__ = ["CONFIGS", "Grid", "config_grid", "make_grid"]
