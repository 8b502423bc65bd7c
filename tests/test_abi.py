"""The C ABI: library builds, loads without a GPU, exports every declared entry
point, and validates plans on the host."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1110_0836_gb300 import _build, _lib
    try:
        _build.build()
    except RuntimeError as e:  # pragma: no cover - no toolkit
        pytest.skip(str(e))
    return _lib.lib()


def declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        text = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"^\w[\w\s\*]*?\b(phb_\w+)\(", text, flags=re.M))
    return sorted(names)


def test_exports_every_declared_symbol(L):
    names = declared()
    assert len(names) >= 12
    for nm in names:
        assert hasattr(L, nm), nm
    from paper_1110_0836_gb300 import _lib
    assert sorted(_lib.EXPORTS) == names


def _plan(**kw):
    from paper_1110_0836_gb300 import _lib
    p = _lib.Plan()
    for a in range(3):
        p.box.lo[a] = 0.0
        p.box.len[a] = kw.get("len", 1.0)
        p.box.periodic[a] = 1
    p.n = kw.get("n", 4096)
    p.rf_factor = 2.3
    p.skin = kw.get("skin", 0.0)
    p.lambda_min = kw.get("lmin", 1 / 16)
    p.lambda_max = kw.get("lmax", 1 / 16)
    p.nbr_capacity = 4096 * 64
    return p


def test_plan_init_valid(L):
    p = _plan()
    assert L.phb_plan_init(C.byref(p)) == 0
    assert p.ws_bytes > 0 and L.phb_workspace_size(C.byref(p), 0) == p.ws_bytes
    # cell edge >= the list radius (default cell_frac 1), every axis covered
    for a in range(3):
        assert p.ncell[a] >= 1 and abs(p.cell[a] * p.ncell[a] - 1.0) < 1e-12
        assert p.cell[a] >= 2.3 / 16 * (1 - 1e-12)
    assert p.nkeys == 64 * p.nbrick[0] * p.nbrick[1] * p.nbrick[2]
    offs = list(p.ws_off)[:10]
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    # the shared prefix ends where the step and adjoint parts begin; both end
    # inside the workspace and one of them ends it
    from paper_1110_0836_gb300 import _lib
    b0, end = _lib.workspace_part(p, _lib.PART_COMMON)
    bs, es = _lib.workspace_part(p, _lib.PART_STEP)
    ba, ea = _lib.workspace_part(p, _lib.PART_ADJOINT)
    assert b0 == 0 and end > offs[-1] and bs == end and ba == end
    assert es > bs and ea > ba and max(es, ea) == p.ws_bytes
    # the step holds F(Y^n), F(Y^p) (8 doubles each) and Y^n (11 doubles) per particle
    assert es - bs >= 27 * 8 * p.n
    for bad in (-1, 3):
        assert L.phb_workspace_part(C.byref(p), bad, C.byref(C.c_size_t()), C.byref(C.c_size_t())) == 1


def test_recomputing_adjoint_needs_less_than_the_stored_record(L):
    """The recomputing adjoint keeps per particle only its adjoint seeds and
    own terms plus the reverse lists: its part of the workspace is smaller
    than the stored-factorisation record it avoids (64^3 lattice plan)."""
    from paper_1110_0836_gb300 import _lib
    p = _plan(n=64 ** 3, lmin=1.0 / 64, lmax=1.0 / 64)
    p.nbr_capacity = 72 * p.n + 1024        # the binding's default capacity
    assert L.phb_plan_init(C.byref(p)) == 0
    b, e = _lib.workspace_part(p, _lib.PART_ADJOINT)
    L.phb_adjoint_record_bytes.restype = C.c_size_t
    assert e - b < L.phb_adjoint_record_bytes(C.byref(p)), (e - b, L.phb_adjoint_record_bytes(C.byref(p)))


@pytest.mark.parametrize("tile,schedule", [(64, 0), (128, 1)])
def test_plan_init_tile_and_schedule(L, tile, schedule):
    p = _plan()
    p.tile, p.schedule = tile, schedule
    assert L.phb_plan_init(C.byref(p)) == 0
    assert p.tile == tile and p.schedule == schedule and p.ntiles == -(-p.n // tile)


@pytest.mark.parametrize("field,val", [("tile", 96), ("schedule", 2), ("ell_width", 4),
                                       ("ell_width", 2000)])
def test_plan_init_rejects_launch_shape(L, field, val):
    p = _plan()
    setattr(p, field, val)
    assert L.phb_plan_init(C.byref(p)) == 1


@pytest.mark.parametrize("kw", [dict(n=0), dict(lmin=-1.0), dict(lmin=0.2, lmax=0.1),
                                dict(lmin=0.25, lmax=0.25), dict(skin=-0.1), dict(len=0.0)])
def test_plan_init_rejects(L, kw):
    p = _plan(**kw)
    assert L.phb_plan_init(C.byref(p)) == 1  # PHB_ERR_INVALID_ARG


def test_status_strings_and_check(L):
    for code in range(9):
        assert L.phb_status_string(code)
    assert L.phb_check(0) == 0
    assert L.phb_check(0x04) == 6     # singular fit -> warning
    assert L.phb_check(0x01 | 0x04) == 4
    assert L.phb_check(0x02) == 5
    assert L.phb_check(0x10) == 7


def test_null_arguments_rejected_on_host(L):
    p = _plan()
    assert L.phb_plan_init(C.byref(p)) == 0
    # null workspace / arrays are caught before any CUDA call
    assert L.phb_build_neighbors(C.byref(p), None, None, None, 0, None, None) in (1, 2)
    assert L.phb_mhd_rhs(C.byref(p), None, None, None, None, None, 0, None, None, None, None) == 1


def test_struct_sizes_match_the_binding(L):
    from paper_1110_0836_gb300 import _lib
    out = (C.c_int64 * 3)()
    assert L.phb_struct_sizes(out, 3) == 0
    assert tuple(out) == (C.sizeof(_lib.Box), C.sizeof(_lib.Params), C.sizeof(_lib.Plan))
    assert C.sizeof(_lib.Params) == 88    # gamma, kind, precision, threshold, zeta, eta, frozen, laws, refine
    assert L.phb_struct_sizes(None, 3) == 1 and L.phb_struct_sizes(out, 4) == 1


def test_default_row_width_follows_the_lambda_range(L):
    p = _plan()
    assert L.phb_plan_init(C.byref(p)) == 0 and p.ell_width == 128
    p = _plan(lmin=1 / 32, lmax=1 / 16)
    assert L.phb_plan_init(C.byref(p)) == 0 and p.ell_width == 256


def test_new_entry_points_reject_bad_arguments_on_host(L):
    """The block step, the mode-amplitude diagnostic and the tensor-core
    experiment check their arguments before any CUDA call: a non-null
    workspace pointer is never dereferenced on these paths."""
    from paper_1110_0836_gb300 import _lib
    p = _plan()
    assert L.phb_plan_init(C.byref(p)) == 0
    prm = _lib.Params()
    prm.gamma, prm.precision = 5.0 / 3.0, _lib.PHB_FP64
    ws, big = C.c_void_p(0x1000), p.ws_bytes
    arr = C.c_void_p(0x2000)
    bad = _lib.PHB_ERR_INVALID_ARG
    sub = L.phb_block_substep
    # substep index outside [0, 2^max_level), level range, step length
    assert sub(C.byref(p), C.byref(prm), arr, arr, arr, arr, arr, -1, 2, 0.1, ws, big, None, None) == bad
    assert sub(C.byref(p), C.byref(prm), arr, arr, arr, arr, arr, 4, 2, 0.1, ws, big, None, None) == bad
    assert sub(C.byref(p), C.byref(prm), arr, arr, arr, arr, arr, 0, 31, 0.1, ws, big, None, None) == bad
    assert sub(C.byref(p), C.byref(prm), arr, arr, arr, arr, arr, 0, 2, 0.0, ws, big, None, None) == bad
    assert sub(C.byref(p), C.byref(prm), arr, arr, arr, None, arr, 0, 2, 0.1, ws, big, None, None) == bad
    assert sub(C.byref(p), C.byref(prm), arr, arr, arr, arr, arr, 0, 2, 0.1, ws, 16, None, None) == \
        _lib.PHB_ERR_WORKSPACE
    assert L.phb_block_begin(C.byref(p), C.byref(prm), arr, arr, arr, None, ws, big, None, None) == bad
    kh = L.phb_kh_mode_amplitude
    assert kh(C.byref(p), arr, arr, -1.0, 1.0, 4.0, ws, big, arr, None) == bad
    assert kh(C.byref(p), arr, arr, 1.0, 1.0, 0.0, ws, big, arr, None) == bad
    assert kh(C.byref(p), arr, arr, 1.0, float("nan"), 4.0, ws, big, arr, None) == bad
    tc = L.phb_fit_tc_experiment
    prm.precision = _lib.PHB_FP64   # the experiment is an FP32-mixed form
    assert tc(C.byref(p), C.byref(prm), arr, arr, arr, ws, big, arr, 214 * 4 * p.n, arr, None, None) == bad
    prm.precision = _lib.PHB_FP32_MIXED
    assert tc(C.byref(p), C.byref(prm), arr, arr, arr, ws, big, arr, 214 * 4 * p.n - 4, arr, None,
              None) == bad


def test_host_step_and_record_region_check_arguments_on_host(L):
    """phb_pc_step_host rejects missing outputs and a non-finite step before any
    CUDA call; phb_record_region reports the records' place in the workspace
    from the plan alone."""
    from paper_1110_0836_gb300 import _lib
    p = _plan()
    assert L.phb_plan_init(C.byref(p)) == 0
    prm = _lib.Params()
    prm.gamma, prm.precision = 5.0 / 3.0, _lib.PHB_FP32_MIXED
    ws, big = C.c_void_p(0x1000), p.ws_bytes
    arr = C.c_void_p(0x2000)
    bad = _lib.PHB_ERR_INVALID_ARG
    step = L.phb_pc_step_host
    assert step(C.byref(p), C.byref(prm), arr, arr, arr, None, arr, 0.1, ws, big, None, None) == bad
    assert step(C.byref(p), C.byref(prm), arr, arr, arr, arr, None, 0.1, ws, big, None, None) == bad
    assert step(C.byref(p), C.byref(prm), arr, arr, arr, arr, arr, float("inf"), ws, big, None,
                None) == bad
    assert step(C.byref(p), C.byref(prm), None, arr, arr, arr, arr, 0.1, ws, big, None, None) == bad
    assert step(C.byref(p), C.byref(prm), arr, arr, arr, arr, arr, 0.1, ws, 16, None, None) == \
        _lib.PHB_ERR_WORKSPACE
    off, nbytes = C.c_size_t(), C.c_size_t()
    assert L.phb_record_region(C.byref(p), C.byref(off), C.byref(nbytes)) == 0
    assert nbytes.value == p.n * 24 * 4 and 0 < off.value and off.value + nbytes.value <= p.ws_bytes
    assert off.value % 256 == 0
    assert L.phb_record_region(None, C.byref(off), C.byref(nbytes)) == 1
    assert L.phb_record_region(C.byref(p), None, C.byref(nbytes)) == 1
