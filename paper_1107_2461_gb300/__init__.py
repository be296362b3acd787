"""GB300-native fast direct inverses of Helmholtz, Laplace and Stokes operators on
stretched finite-volume grids (Vitoshkin & Gelfgat, arXiv:1107.2461).

The compute path is libfdi.so (hand-written CUDA for sm_103a behind the C ABI
of include/fdi.h); `fdi` is its thin ctypes binding.
"""
from . import fdi  # noqa: F401
from .fdi import (  # noqa: F401
    BC_DIRICHLET, BC_NEUMANN, ERR_CUDA, ERR_INVALID_ARG, ERR_NOT_CONVERGED, ERR_OUT_OF_MEMORY, ERR_SINGULAR,
    ERR_TIMEOUT, ERR_UNSUPPORTED, FIELD_CELL, FIELD_U, FIELD_V, FIELD_W, GRID_CELL, GRID_MAC, PREC_FP64,
    PREC_MIXED_BF16, PREC_MIXED_F16, PREC_MIXED_TF32, FdiError, Plan, Server, apply_transform, autotune,
    enable_timing,
    field_solve, field_solve_host,
    helmholtz_solve, helmholtz_solve_batched, kernel_times, laplace_solve, last_launch_count, last_result,
    plan_create, plan_create_cyl, plan_destroy, reset_kernel_times, set_graphs, set_krylov, set_stokes_preconditioner,
    set_resident, set_thomas_config,
    set_wait_limit,
    status_string, stokes_plan_bytes_estimate,
    stokes_solve,
)
