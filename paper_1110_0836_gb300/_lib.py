"""ctypes declarations of the C ABI in include/phurbas.h (argument marshalling only).

The shared library is built in-tree by ``_build.build()``; loading fails loudly
when it is missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphurbas.so")

PHB_OK, PHB_ERR_INVALID_ARG, PHB_ERR_WORKSPACE, PHB_ERR_CUDA, PHB_ERR_CAPACITY = 0, 1, 2, 3, 4
PHB_ERR_SKIN, PHB_WARN_FIT, PHB_ERR_TIMEOUT, PHB_ERR_NONFINITE = 5, 6, 7, 8
FLAG_CAPACITY, FLAG_SKIN, FLAG_FIT_SINGULAR, FLAG_NONFINITE, FLAG_TIMEOUT, FLAG_LAMBDA_RANGE = (
    0x01, 0x02, 0x04, 0x08, 0x10, 0x20)
FLAG_BAD_INDEX = 0x40
PHB_FP64, PHB_FP32_MIXED = 0, 1
# workspace parts (phb_workspace_part)
PART_COMMON, PART_STEP, PART_ADJOINT = 0, 1, 2

EXPORTS = ["phb_plan_init", "phb_workspace_size", "phb_status_string", "phb_check",
           "phb_build_neighbors", "phb_export_neighbors", "phb_neighbor_total", "phb_mls_derivs",
           "phb_mhd_rhs", "phb_pc_step", "phb_rhs_adjoint", "phb_fma_peak", "phb_launch_count",
           "phb_trace_start", "phb_trace_stop", "phb_trace_read", "phb_workspace_stats", "phb_mhd_rhs_noalloc",
           "phb_noalloc_scratch_bytes", "phb_adjoint_record_bytes", "phb_adjoint_record",
           "phb_rhs_adjoint_stored", "phb_mhd_rhs_active", "phb_timestep_levels",
           "phb_struct_sizes", "phb_reorder", "phb_adapt_scan", "phb_adapt_apply",
           "phb_workspace_part", "phb_kh_mode_amplitude", "phb_block_begin",
           "phb_block_substep", "phb_fit_tc_experiment", "phb_pc_step_host", "phb_record_region"]


class Box(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("len", C.c_double * 3), ("periodic", C.c_int32 * 3),
                ("pad_", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("weight_kind", C.c_int32), ("precision", C.c_int32),
                ("cond_threshold", C.c_double), ("zeta", C.c_void_p), ("eta", C.c_void_p),
                ("frozen", C.c_void_p), ("c_zeta_l", C.c_double), ("c_zeta_a", C.c_double),
                ("c_eta", C.c_double), ("refine", C.c_int32), ("refine_schedule", C.c_int32),
                ("refine_kappa", C.c_double)]


class Plan(C.Structure):
    _fields_ = [("box", Box), ("n", C.c_int64), ("rf_factor", C.c_double), ("skin", C.c_double),
                ("lambda_min", C.c_double), ("lambda_max", C.c_double),
                ("nbr_capacity", C.c_int64), ("cell_frac", C.c_double), ("tile", C.c_int32),
                ("stage_cap", C.c_int32), ("schedule", C.c_int32), ("ell_width", C.c_int32),
                ("cell", C.c_double * 3), ("ncell", C.c_int32 * 3), ("nbrick", C.c_int32 * 3),
                ("hilbert_bits", C.c_int32), ("ntiles", C.c_int32),
                ("nkeys", C.c_int64), ("screen_margin", C.c_double), ("ws_bytes", C.c_size_t),
                ("ws_off", C.c_size_t * 48)]


class PhbError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} (code {code})" if what else status_string(code))


_LIB = None
_vp, _i32p = C.c_void_p, C.c_void_p


def lib(path: str | None = None) -> C.CDLL:
    """Open libphurbas.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libphurbas.so not found at {p}: run __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    L = C.CDLL(p)
    P = C.POINTER
    L.phb_plan_init.argtypes = [P(Plan)]
    L.phb_workspace_size.argtypes = [P(Plan), C.c_int32]
    L.phb_workspace_size.restype = C.c_size_t
    L.phb_status_string.argtypes = [C.c_int32]
    L.phb_status_string.restype = C.c_char_p
    L.phb_check.argtypes = [C.c_int32]
    L.phb_build_neighbors.argtypes = [P(Plan), _vp, _vp, _vp, C.c_size_t, _vp, _vp]
    L.phb_export_neighbors.argtypes = [P(Plan), _vp, _vp, _vp, C.c_int64, _vp]
    L.phb_neighbor_total.argtypes = [P(Plan), _vp, _vp]
    L.phb_neighbor_total.restype = C.c_int64
    L.phb_mls_derivs.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, C.c_size_t, _vp, _vp, _vp,
                                 _vp, _vp]
    L.phb_mhd_rhs.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, C.c_size_t, _vp, _vp, _vp, _vp]
    L.phb_pc_step.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, C.c_double, _vp, C.c_size_t, _vp,
                              _vp]
    L.phb_pc_step_host.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, _vp, C.c_double, _vp,
                                   C.c_size_t, _vp, _vp]
    L.phb_rhs_adjoint.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp, _vp,
                                  _vp, _vp]
    L.phb_mhd_rhs_active.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, C.c_int64, _vp,
                                     C.c_size_t, _vp, _vp, _vp, _vp]
    L.phb_mhd_rhs_active.restype = C.c_int
    L.phb_timestep_levels.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, C.c_double, C.c_double,
                                      C.c_int32, _vp, C.c_size_t, _vp, _vp, _vp]
    L.phb_timestep_levels.restype = C.c_int
    L.phb_adjoint_record_bytes.argtypes = [P(Plan)]
    L.phb_adjoint_record_bytes.restype = C.c_size_t
    L.phb_adjoint_record.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, C.c_size_t, _vp,
                                     C.c_size_t, _vp, _vp]
    L.phb_rhs_adjoint_stored.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, _vp, C.c_size_t,
                                         _vp, C.c_size_t, _vp, _vp, _vp, _vp]
    L.phb_fma_peak.argtypes = [C.c_int32, C.c_int32, C.c_int32, _vp, _vp]
    L.phb_fma_peak.restype = C.c_int
    L.phb_launch_count.argtypes = []
    L.phb_launch_count.restype = C.c_int64
    L.phb_trace_start.argtypes = [C.c_int32]
    L.phb_trace_start.restype = C.c_int
    L.phb_trace_stop.argtypes = [_vp, _vp, C.c_int32]
    L.phb_trace_stop.restype = C.c_int
    L.phb_trace_read.argtypes = [_vp, _vp, C.c_int32]
    L.phb_trace_read.restype = C.c_int
    L.phb_workspace_stats.argtypes = [P(Plan), _vp, _vp, C.c_int32, _vp]
    L.phb_record_region.argtypes = [P(Plan), P(C.c_size_t), P(C.c_size_t)]
    L.phb_record_region.restype = C.c_int
    L.phb_workspace_stats.restype = C.c_int
    L.phb_mhd_rhs_noalloc.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.phb_mhd_rhs_noalloc.restype = C.c_int
    L.phb_noalloc_scratch_bytes.argtypes = []
    L.phb_noalloc_scratch_bytes.restype = C.c_size_t
    L.phb_reorder.argtypes = [P(Plan), _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp, _vp]
    L.phb_adapt_scan.argtypes = [P(Plan), _vp, _vp, C.c_double, C.c_double, _vp, C.c_size_t, _vp,
                                 _vp, _vp, _vp, _vp, _vp]
    L.phb_adapt_scan.restype = C.c_int
    L.phb_adapt_apply.argtypes = [P(Plan), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_double,
                                  C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp, _vp]
    L.phb_adapt_apply.restype = C.c_int
    L.phb_reorder.restype = C.c_int
    L.phb_kh_mode_amplitude.argtypes = [P(Plan), _vp, _vp, C.c_double, C.c_double, C.c_double,
                                        _vp, C.c_size_t, _vp, _vp]
    L.phb_kh_mode_amplitude.restype = C.c_int
    L.phb_block_begin.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp, _vp]
    L.phb_block_begin.restype = C.c_int
    L.phb_block_substep.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, _vp, C.c_int32,
                                    C.c_int32, C.c_double, _vp, C.c_size_t, _vp, _vp]
    L.phb_block_substep.restype = C.c_int
    L.phb_fit_tc_experiment.argtypes = [P(Plan), P(Params), _vp, _vp, _vp, _vp, C.c_size_t, _vp,
                                        C.c_size_t, _vp, _vp, _vp]
    L.phb_fit_tc_experiment.restype = C.c_int
    L.phb_workspace_part.argtypes = [P(Plan), C.c_int32, _vp, _vp]
    L.phb_workspace_part.restype = C.c_int
    L.phb_struct_sizes.argtypes = [_vp, C.c_int32]
    L.phb_struct_sizes.restype = C.c_int
    sizes = (C.c_int64 * 3)()
    if L.phb_struct_sizes(sizes, 3) != 0 or tuple(sizes) != (C.sizeof(Box), C.sizeof(Params),
                                                             C.sizeof(Plan)):
        raise RuntimeError(f"{p}: struct sizes {tuple(sizes)} differ from the binding's "
                           f"{(C.sizeof(Box), C.sizeof(Params), C.sizeof(Plan))}; rebuild")
    for f in ("phb_plan_init", "phb_check", "phb_build_neighbors", "phb_export_neighbors",
              "phb_mls_derivs", "phb_mhd_rhs", "phb_pc_step", "phb_pc_step_host", "phb_rhs_adjoint"):
        getattr(L, f).restype = C.c_int
    if path is None:
        _LIB = L
    return L


def workspace_part(plan: Plan, part: int) -> tuple[int, int]:
    """Byte range (begin, end) of a workspace part of an initialised plan."""
    b, e = C.c_size_t(0), C.c_size_t(0)
    if lib().phb_workspace_part(C.byref(plan), int(part), C.byref(b), C.byref(e)) != 0:
        raise ValueError(f"invalid plan or workspace part {part}")
    return int(b.value), int(e.value)


def status_string(code: int) -> str:
    try:
        return lib().phb_status_string(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def check(code: int, what: str = "") -> None:
    if code != PHB_OK:
        raise PhbError(code, what)
