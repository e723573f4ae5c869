"""Seeded synthetic inputs for the event-based Monte Carlo transport hot path.

This module only *draws data*: nuclide energy grids and cross-section tables,
material compositions, geometry and tally descriptions. It holds none of the
transport arithmetic (no lookup, no tracking, no collision physics, no RNG
stream of the method) and is shared by the CPU oracle tests and the CUDA path.

The paper's workloads (a depleted SMR core and a depleted pincell with
evaluated nuclear data, Sec. 3 and Sec. 4.1) are not available, so these
configurations stand in for them with the same shape: many nuclides per fuel
material, pointwise continuous-energy tables of 1e4-6e4 points, and a
cylinder-in-box lattice.
"""
from .problem import (Problem, Geometry, make_config, make_stress_lookup,
                      make_tiny_problem, make_eigen_lattice, GEOM_INFINITE, GEOM_LATTICE, GEOM_SLAB,
                      BC_VACUUM, BC_REFLECT, SRC_BOX, SRC_ORIGIN, SRC_SLAB_FACE,
                      BASE_SEED)

__all__ = ["Problem", "Geometry", "make_config", "make_stress_lookup",
           "make_tiny_problem", "make_eigen_lattice", "GEOM_INFINITE", "GEOM_LATTICE", "GEOM_SLAB",
           "BC_VACUUM", "BC_REFLECT", "SRC_BOX", "SRC_ORIGIN", "SRC_SLAB_FACE",
           "BASE_SEED"]
