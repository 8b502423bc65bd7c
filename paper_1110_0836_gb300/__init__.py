"""GB300 (sm_103a) library for the Phurbas particle right-hand side.

Hot path (all in libphurbas, C ABI in include/phurbas.h): cell binning and the
strict fixed-radius neighbour search, the fused third-order interpolating MLS
fit + ideal-MHD Lagrangian right-hand side (FP32-mixed with FP64 routing, or
FP64), the Heun predictor-corrector step, and the hand-written adjoint.
"""
from ._lib import PhbError  # noqa: F401
from .api import (FIELDS, HostStepGraph, Params, Plan, StepGraph, active_at, adapt,  # noqa: F401
                  adapt_apply,
                  adapt_scan, adjoint_record, block_step,
                  build_neighbors, export_neighbors, fit_tc_experiment, kh_mode_amplitude, mhd_rhs,
                  mhd_rhs_active,
                  mls_derivs, pc_step, pc_step_host, reorder,
                  rhs, rhs_adjoint, rhs_adjoint_stored, tensors_of, timestep_levels)
from .autograd import PhbRHS, rhs_autograd  # noqa: F401


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libphurbas.so in-tree for sm_103a."""
    from ._build import build as _b
    return _b(force=force, verbose=verbose)
