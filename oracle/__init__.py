"""Plain FP64 CPU oracle for the GW screening pipeline.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run this package.  The
CUDA library never calls it and shares no code with it; both sides only share
the seeded input generator in ``synth``.

Every function restates one step of Foerster, Koval and Sanchez-Portal,
"An O(N^3) implementation of Hedin's GW approximation for molecules"
(arXiv:1101.2065), by its plain definition: dense contractions, rank-1
updates, O(N_omega^2) direct Cauchy sums, LAPACK solves, explicit loops.
Readings of points the paper leaves open are listed in the module docstring
of ``oracle.gw``.
"""
from .gw import (pair_table, vertex_products, compression_basis, deposit_spectral,
                 chi0_cauchy, screen, sigma_forms, sigma_grid,
                 sigma_c_grid, sigma_c_re, sigma_x, qp_solve, solve, sigma_grid_range)

__all__ = ["pair_table", "vertex_products", "compression_basis", "deposit_spectral",
           "chi0_cauchy", "screen", "sigma_forms", "sigma_grid",
           "sigma_c_grid", "sigma_c_re", "sigma_x", "qp_solve", "solve", "sigma_grid_range"]
