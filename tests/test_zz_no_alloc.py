"""The allocation-free entry point phb_mhd_rhs_noalloc.

It serves callers that cannot allocate device memory where they need the
right-hand side: the scratch comes from a fixed array inside the library, so
the call only needs the caller's input and output arrays.  Here it must agree
with the ordinary workspace path (phb_build_neighbors + phb_mhd_rhs) on two
calls in a row (the second call reuses the array the first one left behind),
and refuse a plan that does not fit the array.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads
from _gpu import need_gpu, torch

pytestmark = pytest.mark.gpu


def _call(L, plan, prm_c, pos, lam, U, out, st, status):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.phb_mhd_rhs_noalloc(C.byref(plan.c), C.byref(prm_c), C.c_void_p(pos.data_ptr()),
                                 C.c_void_p(lam.data_ptr()), C.c_void_p(U.data_ptr()),
                                 C.c_void_p(out.data_ptr()), C.c_void_p(st.data_ptr()),
                                 C.c_void_p(status.data_ptr()), stream)


@pytest.mark.parametrize("prec,tol", [("fp32_mixed", 1e-5), ("fp64", 1e-12)])
def test_no_alloc_matches_workspace_path_twice(prec, tol):
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    L = _lib.lib()
    w = workloads.random_modes(16, seed=77)
    plan = phb.Plan.for_workload(w)
    assert _lib.workspace_part(plan.c, _lib.PART_COMMON)[1] <= L.phb_noalloc_scratch_bytes()
    pos, lam, U = phb.tensors_of(w)
    prm = phb.Params(gamma=w.gamma, precision=prec)
    phb.build_neighbors(plan, pos, lam)
    ref, _ = phb.mhd_rhs(plan, prm, pos, lam, U)
    ref = ref.cpu().numpy()
    scale = np.abs(ref).max(axis=1)
    prm_c = prm.c()
    for _ in range(2):
        out = torch.full((8, w.n), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((w.n,), -1, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert _call(L, plan, prm_c, pos, lam, U, out, st, status) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert (st.cpu().numpy() == 0).all()
        err = np.abs(out.cpu().numpy() - ref).max(axis=1) / scale
        assert err.max() < tol, err


def test_no_alloc_rejects_plan_larger_than_scratch():
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    L = _lib.lib()
    w = workloads.random_modes(40, seed=78)   # 64,000 particles: above the 32 MiB scratch
    plan = phb.Plan.for_workload(w)
    assert _lib.workspace_part(plan.c, _lib.PART_COMMON)[1] > L.phb_noalloc_scratch_bytes()
    pos, lam, U = phb.tensors_of(w)
    out = torch.empty((8, w.n), dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    prm_c = phb.Params(gamma=w.gamma).c()
    rc = L.phb_mhd_rhs_noalloc(C.byref(plan.c), C.byref(prm_c), C.c_void_p(pos.data_ptr()),
                               C.c_void_p(lam.data_ptr()), C.c_void_p(U.data_ptr()),
                               C.c_void_p(out.data_ptr()), None, C.c_void_p(status.data_ptr()),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.PHB_ERR_WORKSPACE
