"""Seeded synthetic inputs for the PDEP hot path.

This package builds the *inputs* both sides consume: local potentials V(r)
made of periodic Gaussian wells on an orthorhombic FFT grid, the occupied
and PDEP counts of each workload, random start blocks and random
perturbing potentials.  It holds none of the method's arithmetic (no
plane-wave sphere, no Hamiltonian, no response): the CPU oracle and the
CUDA library each build those on their own from these arrays.
"""
from .systems import (  # noqa: F401
    System,
    WORKLOADS,
    gaussian_wells,
    make_system,
    make_batch,
    periodic_gaussian_sum,
    random_grid_potentials,
    random_vectors,
)
