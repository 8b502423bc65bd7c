"""GPU individual power-of-two time steps (Sec. 2, Sec. 2.1) against the
oracle's block step: increments of U over the step per field, relative to the
largest oracle increment of that field, and of x relative to the largest
oracle displacement (the three axes share one scale; an axis along which the
set hardly moves would otherwise measure rounding against noise) - 1e-12 in
FP64, 1e-5 FP32-mixed."""
import numpy as np
import pytest

import oracle
import workloads
from _gpu import need_gpu, torch

pytestmark = pytest.mark.gpu


def incr_err(p1, u1, po, uo, p0, u0):
    dg = np.concatenate([p1 - p0, u1 - u0])
    do = np.concatenate([po - p0, uo - u0])
    num = np.abs(dg - do).max(axis=1)
    den = np.abs(do).max(axis=1)
    den[:3] = den[:3].max()
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def run_gpu(phb, w, levels, dt, max_level, prec, steps=1):
    plan = phb.Plan.for_workload(w)
    pos, lam, U = phb.tensors_of(w)
    lv = torch.tensor(levels, dtype=torch.int32, device="cuda")
    prm = phb.Params(gamma=w.gamma, precision=prec)
    anchor = None
    for _ in range(steps):
        anchor = phb.block_step(plan, prm, pos, lam, U, lv, dt, max_level, anchor=anchor)
    torch.cuda.synchronize()
    plan.raise_status("block step")
    return pos.cpu().numpy(), U.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_block_step_matches_oracle(prec, tol):
    """Random levels 0..2 on a random-mode lattice, two synchronised steps
    (the second continues from the first one's anchors)."""
    phb = need_gpu()
    w = workloads.random_modes(10, seed=51, amp=0.05)
    levels = np.random.default_rng(3).integers(0, 3, w.n)
    dt = 0.004
    box = oracle.box_of(w)
    po, uo, anc = oracle.block_step(box, w.pos, w.lam, w.U, levels, dt, 2, gamma=w.gamma)
    po, uo, _ = oracle.block_step(box, po, w.lam, uo, levels, dt, 2, anchor=anc, gamma=w.gamma)
    pg, ug = run_gpu(phb, w, levels, dt, 2, prec, steps=2)
    e = incr_err(pg, ug, po, uo, w.pos, w.U)
    assert e.max() < tol, e


def test_block_step_levels_from_the_limiter():
    """Levels from phb_timestep_levels on a density-sampled shock tube (lambda
    varying 2x, so levels differ across the fronts), FP64 against the oracle."""
    phb = need_gpu()
    w = workloads.shock_tube(8000, seed=52)
    plan = phb.Plan.for_workload(w)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    prm = phb.Params(gamma=w.gamma, precision="fp64")
    dt_max = 0.02
    lv = phb.timestep_levels(plan, prm, pos, lam, U, cfl=0.2, dt_max=dt_max, max_level=3)
    levels = lv.cpu().numpy().astype(np.int64)
    assert len(np.unique(levels)) >= 2
    box = oracle.box_of(w)
    po, uo, _ = oracle.block_step(box, w.pos, w.lam, w.U, levels, dt_max, 3, gamma=w.gamma)
    pg, ug = run_gpu(phb, w, levels, dt_max, 3, "fp64")
    e = incr_err(pg, ug, po, uo, w.pos, w.U)
    assert e.max() < 1e-12, e


def test_one_level_equals_the_predictor_corrector_step():
    phb = need_gpu()
    w = workloads.random_modes(10, seed=53, amp=0.05)
    dt = 0.003
    pg, ug = run_gpu(phb, w, np.zeros(w.n, np.int64), dt, 0, "fp64")
    plan = phb.Plan.for_workload(w, skin=0.01)
    pos, lam, U = phb.tensors_of(w)
    phb.pc_step(plan, phb.Params(gamma=w.gamma, precision="fp64"), pos, lam, U, dt)
    e = incr_err(pg, ug, pos.cpu().numpy(), U.cpu().numpy(), w.pos, w.U)
    assert e.max() < 1e-12, e


def test_substeps_without_active_particles():
    """Every particle on level 0 of max_level 2: the first three substeps have
    no particle whose step ends there (nothing is evaluated, the states are
    only predicted), and the result equals the one-level step of dt_max."""
    phb = need_gpu()
    w = workloads.random_modes(10, seed=54, amp=0.05)
    dt = 0.003
    p2, u2 = run_gpu(phb, w, np.zeros(w.n, np.int64), dt, 2, "fp64")
    p0, u0 = run_gpu(phb, w, np.zeros(w.n, np.int64), dt, 0, "fp64")
    e = incr_err(p2, u2, p0, u0, w.pos, w.U)
    assert e.max() < 1e-13, e
