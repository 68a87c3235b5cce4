"""FP64 CPU oracle of the icosahedral C-grid dynamical-core step (plain numpy).

TEST INFRASTRUCTURE ONLY. Only tests/, bench.py's CPU-baseline and reference legs
and __graft_entry__.smoke() import this package. The product library (the CUDA
path and its Python binding) never imports, links or calls anything here, and this
package imports nothing from the product.
"""
from .grid import build_grid, R_EARTH, OMEGA          # noqa: F401
from .state import (vertical_grid, init_state, exner_ref, splitmix64, uniform01,   # noqa: F401
                    member_params, CASE_REST, CASE_SBR, CASE_JET, CASE_MEMBER)
from .dycore import dycore_step, global_mass, tendencies, diffusion    # noqa: F401
from .tracer import tracer_step, tracer_mass, cell_gradient, cell_neighbours, cell_lsq_weights   # noqa: F401
