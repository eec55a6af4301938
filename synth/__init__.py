"""Seeded synthetic molecules for the GW screening pipeline.

This package only draws inputs (geometry, neighbour lists, Kohn-Sham-like
eigenpairs, the block-sparse product vertex and the Coulomb metric).  It holds
none of the GW arithmetic; both the FP64 oracle and the CUDA library consume
the arrays it produces.
"""
from .molecules import (Molecule, Grid, make_molecule, make_config, make_batch,
                        make_serving_trace, local_orbitals, CONFIGS, ETA, D_OMEGA)

__all__ = ["Molecule", "Grid", "make_molecule", "make_config", "make_batch",
           "make_serving_trace", "local_orbitals", "CONFIGS", "ETA", "D_OMEGA"]
