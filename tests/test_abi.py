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
    # the shared prefix ends where the predictor-corrector regions begin
    from paper_1110_0836_gb300 import _lib
    end = p.ws_off[_lib.WS_END_COMMON]
    assert end > offs[-1] and end == p.ws_off[_lib.WS_END_COMMON - 9]  # first predictor-corrector region
    # adjoint regions: edge contributions (10 doubles per list entry) first, the
    # per-particle self terms (11 doubles) last, ending the workspace
    assert p.ws_off[_lib.WS_ADJ_SELF] - p.ws_off[_lib.WS_ADJ_EDGE] >= 10 * 8 * p.nbr_capacity
    assert p.ws_off[_lib.WS_ADJ_SELF] + 11 * 8 * p.n <= p.ws_bytes


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
    assert C.sizeof(_lib.Params) == 72    # gamma, kind, precision, threshold, zeta, eta, frozen, laws
    assert L.phb_struct_sizes(None, 3) == 1 and L.phb_struct_sizes(out, 4) == 1


def test_default_row_width_follows_the_lambda_range(L):
    p = _plan()
    assert L.phb_plan_init(C.byref(p)) == 0 and p.ell_width == 128
    p = _plan(lmin=1 / 32, lmax=1 / 16)
    assert L.phb_plan_init(C.byref(p)) == 0 and p.ell_width == 256
