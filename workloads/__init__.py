"""Seeded, synthetic problem definitions shared by the oracle side and the CUDA side.

This package holds problem *data* only: grids, physical coefficients, boundary
values, initial fields and the closed-form PDE solutions used as references.
It contains none of the lattice Boltzmann arithmetic; both the CPU oracle
(``oracle/``) and the CUDA library consume the same :class:`Problem` objects.
"""
from .problems import (  # noqa: F401
    Problem, Source, PERIODIC, HBB,
    gaussian_hill, mms_sinsin, nonlinear_modes, steady_diffusion, linear_cde, variable_tensor,
    burgers_fisher, burgers_fisher_solution,
    batched_instances, random_state_problem,
)
from .exact import (  # noqa: F401
    gaussian_hill_exact, mms_sinsin_exact, steady_diffusion_exact, linear_cde_exact,
    variable_tensor_exact, burgers_fisher_exact,
)
from .metrics import gre, rel_l2  # noqa: F401
from .problems3 import (  # noqa: F401
    Problem3, gaussian_hill3, steady_diffusion3, random_state_problem3, rot_tensor3,
    gaussian_hill3_exact, steady_diffusion3_exact,
)
