"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds input generation only: a counter-based PRNG (SplitMix64),
Boolean-sphere voxel microstructures, small hand-made label grids for the
closed-form tests, parameter-study samplers, the germ-grain initial plated
lithium (``plating``), and the loader of the parameter table (``params.json``).  It contains none of the method's arithmetic (no
flux, kinetics, time stepping, reduction or 1C conversion); each side of the
parity check implements those on its own.

Phase labels (uint8), shared convention of the C-ABI and the oracle:

    E  = 0  electrolyte
    G  = 1  anode active material (graphite)
    K  = 2  cathode active material
    L  = 3  lithium-metal foil (half-cell counter electrode)
    CN = 4  negative current collector (outer face at t = 0)
    CP = 5  positive current collector (outer face at t = nt-1)

Grids are indexed [t][y][z] with z fastest; t is the through-cell axis.
"""
from .geometry import (E, G, K, L, CN, CP, SplitMix64, boolean_sphere_slab,
                       full_cell, half_cell, slab_1d, load_params)
from .study import sample_rom_params, poisson_arrivals

__all__ = ["E", "G", "K", "L", "CN", "CP", "SplitMix64", "boolean_sphere_slab",
           "full_cell", "half_cell", "slab_1d", "load_params",
           "sample_rom_params", "poisson_arrivals"]
