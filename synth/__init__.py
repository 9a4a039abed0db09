"""Seeded synthetic inputs shared by the oracle and the GPU path.

Geometry and numbering (`mesh`), the random viscosity model (`kl`), problem
presets, the gPC index convention and seeded random TT cores (`problem`).
None of these modules holds solver arithmetic.
"""
from .mesh import Mesh, step_mesh, channel_mesh
from .kl import viscosity_fields, kl_eigenpairs
from .problem import (Problem, Tolerances, gpc_multi_indices, n_xi, make_problem,
                      preset, random_tt, time_profile, batch)
