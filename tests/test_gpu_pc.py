"""GPU predictor-corrector step vs the oracle's Heun step (Paper II Sec. 2)."""
import numpy as np
import pytest

import oracle
import workloads
from _gpu import kind_err, need_gpu, rhs_err, rhs_term_scales, torch

pytestmark = pytest.mark.gpu


def run_pc(phb, w, dt, prec, skin):
    plan = phb.Plan.for_workload(w, skin=skin)
    pos, lam, U = phb.tensors_of(w)
    phb.pc_step(plan, phb.Params(gamma=w.gamma, precision=prec), pos, lam, U, dt)
    return pos.cpu().numpy(), U.cpu().numpy(), plan


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_pc_step_matches_oracle(prec, tol):
    phb = need_gpu()
    w = workloads.random_modes(10, seed=21, amp=0.05)
    dt = 0.002
    pos, U, plan = run_pc(phb, w, dt, prec, skin=0.01)
    assert plan.read_status() == 0
    op, oU, ns = oracle.pc_step(oracle.box_of(w), w.pos, w.lam, w.U, dt, gamma=w.gamma)
    assert ns == 0
    # compare the increments (the states themselves are dominated by Y^n),
    # against dt times each equation's term scale at Y^n
    box = oracle.box_of(w)
    g, h, _ = oracle.mls_derivs(box, w.pos, w.lam, w.U, oracle.neighbors(box, w.pos, w.lam),
                                gamma=w.gamma)
    sc = dt * rhs_term_scales(w.U, g, h, w.gamma)
    assert rhs_err(U - w.U, oU - w.U, sc).max() < tol
    assert kind_err(pos - w.pos, op - w.pos).max() < tol


def test_uniform_flow_advects_exactly():
    phb = need_gpu()
    w = workloads.linear_wave(8, amplitude=0.0)
    w.U[1:4] = np.array([[0.25], [-0.125], [0.5]])
    dt = 0.015625
    pos, U, plan = run_pc(phb, w, dt, "fp32_mixed", skin=0.05)
    assert plan.read_status() == 0
    np.testing.assert_array_equal(U, w.U)
    np.testing.assert_array_equal(pos, w.pos + dt * w.U[1:4])


def test_skin_violation_is_flagged():
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    w = workloads.random_modes(8, seed=22, amp=0.05)
    w.U[1] += 1.0
    pos, U, plan = run_pc(phb, w, 0.01, "fp64", skin=0.005)
    assert plan.read_status() & _lib.FLAG_SKIN
