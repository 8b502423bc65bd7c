"""The tensor-core form of the fit's accumulation (a measured experiment):
moments and right-hand sides as per-particle Gram matrices on mma.sync with
the 3xTF32 split.  Its right-hand side must meet the FP32-mixed bar against
the oracle on the lattice and agree with the FP32 CUDA-core kernel."""
import numpy as np
import pytest

import oracle
import workloads
from _gpu import need_gpu, rhs_err, rhs_term_scales, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("stage_cap", [0, 64])
def test_tc_gram_matches_oracle(stage_cap):
    """Both neighbour sources (staged tiles; every tile from global memory)."""
    phb = need_gpu()
    w = workloads.random_modes(16, seed=61)
    plan = phb.Plan.for_workload(w, stage_cap=stage_cap, cell_frac=0.5)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    prm = phb.Params(gamma=w.gamma, refine="off")
    out, gram = phb.fit_tc_experiment(plan, prm, pos, lam, U)
    ref, _ = phb.mhd_rhs(plan, prm, pos, lam, U)
    torch.cuda.synchronize()
    box = oracle.box_of(w)
    nb = oracle.neighbors(box, w.pos, w.lam)
    exp, _ = oracle.mhd_rhs(box, w.pos, w.lam, w.U, nb, gamma=w.gamma)
    g, h, _ = oracle.mls_derivs(box, w.pos, w.lam, w.U, nb, gamma=w.gamma)
    sc = rhs_term_scales(w.U, g, h, w.gamma)
    e_tc = rhs_err(out.cpu().numpy(), exp, sc)
    e_cc = rhs_err(ref.cpu().numpy(), exp, sc)
    print("tensor-core", e_tc.max(), "CUDA-core", e_cc.max())
    assert e_tc.max() < 1e-5, e_tc
    counts = gram[-1].cpu().numpy()
    assert counts.min() >= 19
    plan.raise_status("tc experiment")
