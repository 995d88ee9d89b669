"""GB300 (sm_103a) library for the two-component D3Q19 Shan-Chen lattice
Boltzmann step of Otomo et al., arXiv:1601.01237.

The step runs in hand-written CUDA kernels behind the C ABI of include/lbm.h;
this package holds the build step, the ctypes binding and the seeded
synthetic workloads.
"""
from ._native import LBMError, STORAGE, COLLISION, WALL_MODEL  # noqa: F401
from .lattice import (Lattice, make_params, lbm_lattice_dirs, lbm_create, lbm_init_fields,  # noqa: F401
                      lbm_step, lbm_step_timed, lbm_moments, lbm_reduce, lbm_get_populations, lbm_set_populations,
                      lbm_state_bytes, lbm_get_state, lbm_set_state, lbm_step_count, lbm_sync,
                      lbm_destroy, lbm_step_noalloc, NOALLOC_MAX_CELLS, lbm_record, lbm_adjoint,
                      lbm_pressure_jump, lbm_droplet_stats, lbm_set_solid)
