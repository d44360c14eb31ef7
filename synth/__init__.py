"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module builds initial data and parameter sets only: analytic Fourier-mode
metrics and fluids, a TOV star, random fluid states and the synthetic EOS
table.  It holds none of the substep's arithmetic (no CCZ4 or conserved
variables, no finite differences, no con2prim); each implementation converts
the initial data below with its own code.

Initial data are returned as float64 arrays of shape (NID, n2+6, n1+6, px)
holding, at every point including the three ghost layers per side:
  0-5   gamma_ij (xx xy xz yy yz zz)     6-11  K_ij
  12    alpha                            13-15 beta^i
  16    rho                              17    eps (ideal gas)
  18-20 v^i (contravariant)              21-23 B^i (not densitized)
  24    Ye                               25    T [MeV] (tabulated EOS)
"""
import numpy as np

from .configs import (NID, NG, ideal_params, table_params, hybrid_params, grid_coords, patch_shape)  # noqa: F401
from .fields import config0_id, tov_id, tov_profile, batched_specs, batched_id, EDGES  # noqa: F401
from .eos_table import make_table  # noqa: F401
from .states import c2p_states  # noqa: F401
from .hierarchy import small_hierarchy, nested_cubes, amr_tov_layout, subcycle_hierarchy  # noqa: F401
