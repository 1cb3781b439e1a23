"""FP64 CPU oracle of the coupled phi-mu lattice Boltzmann step (arXiv 2111.05960, Sec. 3).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA product path never
imports, links or executes anything under ``oracle/``, and this package imports
nothing from the product.
"""
from .oracle import (  # noqa: F401
    OracleParams, Oracle, build, lattice_tables, gradient, lambda_star_printed,
    stefan_one_sided_root, stefan_two_sided_root,
    PARAM_NAMES, step_adjoint, init_adjoint, trajectory_gradient, tangent_trajectory, tangent_step,
)
