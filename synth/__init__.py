"""Seeded synthetic inputs for the xTC grid build: molecules, quadrature grids,
grid-orthonormal orbitals, reference densities and Jastrow parameters.

This package holds input generation only.  None of the method's arithmetic
(Jastrow gradients, intermediates, contractions) lives here, so the oracle and
the CUDA path can both consume its arrays without sharing any of the method.
"""
from .molecules import (  # noqa: F401
    Problem,
    CANONICAL_TERMS,
    make_batched,
    make_config,
    make_small,
    orbital_gradients,
    random_density,
    permute_grid,
    CONFIG_NAMES,
)
