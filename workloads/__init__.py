"""Seeded synthetic inputs for the shifted-COCG / Dyson transport path.

This module only *draws* inputs: grids, local potentials made of Gaussian
wells, Kleinman-Bylander projector tables, energy grids, boundary-column
samples and random matrices for unit tests.  It holds none of the method's
arithmetic (no Hamiltonian application, no Krylov recurrences, no self-energy,
no Dyson step), so both the CUDA library's tests and the CPU oracle can take
their inputs from here without sharing any of the method's code.

The workloads stand in for the paper's Na wire (Sec. III C) and the
C60@(10,10)CNT peapod (Sec. IV), whose DFT potentials are not available; only
their shapes (grid sizes, spacing, numbers of energies, a localised potential
and, for the peapod, one nonlocal projector per atom) are reproduced.
"""

from .problems import (  # noqa: F401
    Problem,
    Projectors,
    CONFIG_NAMES,
    make_problem,
    small_problem,
    grid_coordinates,
    boundary_plane_points,
    sample_plane_columns,
    random_complex_matrices,
)
