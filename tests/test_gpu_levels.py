"""Individual time-step levels and the active-subset right-hand side on the
GPU, against the oracle (Paper II Sec. 2, Sec. 2.1)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads
from _gpu import need_gpu, rhs_err, rhs_term_scales, torch

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _spread(w, seed):
    rng = np.random.default_rng(seed)
    w.U[7] *= rng.uniform(0.5, 40.0, w.n)
    w.U[4:7] *= rng.uniform(0.2, 3.0, w.n)
    return w


def test_levels_golden_line():
    phb = need_gpu()
    g = json.load(open(os.path.join(HERE, "golden", "timestep_levels_line.json")))
    n = len(g["pos_x"])
    pos = np.zeros((3, n))
    pos[0] = g["pos_x"]
    pos[1:] = 0.5
    lam = np.full(n, g["lambda"])
    U = np.zeros((8, n))
    U[0] = 1.0
    gam = g["gamma"]
    U[7] = np.asarray(g["sound_speed"]) ** 2 / (gam * (gam - 1.0))
    plan = phb.Plan((0, 0, 0), (8, 1, 1), (0, 0, 0), n, 1.0, 1.0)
    t = [torch.as_tensor(a, device="cuda").contiguous() for a in (pos, lam, U)]
    phb.build_neighbors(plan, t[0], t[1])
    L = phb.timestep_levels(plan, phb.Params(gamma=gam), *t, cfl=g["cfl"], dt_max=g["dt_max"],
                            max_level=g["max_level"])
    assert L.cpu().tolist() == g["levels"]


@pytest.mark.parametrize("skin", [0.0, 0.01])
def test_levels_bit_exact_against_oracle(skin):
    """Density-sampled shock tube with spread sound and Alfven speeds; lists
    with and without a skin (the limiter filters exactly at r_f)."""
    phb = need_gpu()
    w = _spread(workloads.shock_tube(20000, seed=4), 4)
    nb = oracle.neighbors(oracle.box_of(w), w.pos, w.lam)
    kw = dict(cfl=0.2, dt_max=0.05, max_level=12)
    exp = oracle.timestep_levels(w.lam, w.U, nb, gamma=w.gamma, **kw)
    plan = phb.Plan.for_workload(w, skin=skin)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    got = phb.timestep_levels(plan, phb.Params(gamma=w.gamma), pos, lam, U, **kw).cpu().numpy()
    assert np.array_equal(got, exp)
    assert exp.max() - exp.min() >= 2
    plan.raise_status()


def test_active_at_binary_block_schedule():
    phb = need_gpu()
    lv = torch.tensor([0, 1, 2, 2, 3], dtype=torch.int32, device="cuda")
    assert phb.active_at(lv, 0, 3).cpu().tolist() == [0, 1, 2, 3, 4]
    assert phb.active_at(lv, 1, 3).cpu().tolist() == [4]
    assert phb.active_at(lv, 2, 3).cpu().tolist() == [2, 3, 4]
    assert phb.active_at(lv, 4, 3).cpu().tolist() == [1, 2, 3, 4]


def _active_case(phb, seed=17):
    w = workloads.random_modes(16, seed=seed)
    rng = np.random.default_rng(seed)
    act = np.sort(rng.choice(w.n, w.n // 3, replace=False)).astype(np.int32)
    act_dup = np.concatenate([act, act[:50]])             # duplicates are evaluated once
    rng.shuffle(act_dup)
    plan = phb.Plan.for_workload(w)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    return w, act, torch.as_tensor(act_dup, device="cuda"), plan, pos, lam, U


def test_active_rhs_fp64_equals_full_evaluation():
    phb = need_gpu()
    w, act, dact, plan, pos, lam, U = _active_case(phb)
    prm = phb.Params(gamma=w.gamma, precision="fp64")
    full, _ = phb.mhd_rhs(plan, prm, pos, lam, U)
    out = torch.full((8, w.n), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((w.n,), -7, dtype=torch.int32, device="cuda")
    phb.mhd_rhs_active(plan, prm, pos, lam, U, dact, out=out, fit_status=st)
    out, st, full = out.cpu().numpy(), st.cpu().numpy(), full.cpu().numpy()
    assert np.array_equal(out[:, act], full[:, act])
    rest = np.setdiff1d(np.arange(w.n), act)
    assert np.isnan(out[:, rest]).all() and (st[rest] == -7).all() and (st[act] == 0).all()


def test_active_rhs_mixed_against_oracle():
    phb = need_gpu()
    w, act, dact, plan, pos, lam, U = _active_case(phb, seed=18)
    out = torch.full((8, w.n), float("nan"), dtype=torch.float64, device="cuda")
    phb.mhd_rhs_active(plan, phb.Params(gamma=w.gamma), pos, lam, U, dact, out=out)
    box = oracle.box_of(w)
    q = act.astype(np.int64)
    nb = oracle.neighbors(box, w.pos, w.lam, q)
    exp, _ = oracle.mhd_rhs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
    g, h, _ = oracle.mls_derivs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
    sc = rhs_term_scales(w.U[:, q], g, h, w.gamma)
    assert rhs_err(out.cpu().numpy()[:, act], exp, sc).max() < 1e-5
    assert np.isnan(out.cpu().numpy()[:, np.setdiff1d(np.arange(w.n), act)]).all()


def test_active_rhs_bad_index_and_empty_subset():
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    w, act, dact, plan, pos, lam, U = _active_case(phb, seed=19)
    prm = phb.Params(gamma=w.gamma)
    out = torch.full((8, w.n), float("nan"), dtype=torch.float64, device="cuda")
    phb.mhd_rhs_active(plan, prm, pos, lam, U, torch.zeros(0, dtype=torch.int32, device="cuda"),
                       out=out)
    assert torch.isnan(out).all() and plan.read_status() == 0
    bad = torch.tensor([3, w.n, -1, 5], dtype=torch.int32, device="cuda")
    phb.mhd_rhs_active(plan, prm, pos, lam, U, bad, out=out)
    assert plan.read_status() & _lib.FLAG_BAD_INDEX
    o = out.cpu().numpy()
    assert np.isfinite(o[:, [3, 5]]).all() and np.isnan(np.delete(o, [3, 5], axis=1)).all()


def test_active_rhs_corrected_step_on_a_shear_layer():
    """The active subset of a density-sampled shear layer: the chunks of
    listed particles take the corrected step like tiles do (refine "on" and
    "auto"), and the subset's time derivatives meet 1e-5 against the oracle;
    without the step they do not."""
    phb = need_gpu()
    w = workloads.shear_layer(200_000, seed=23)
    plan = phb.Plan.for_workload(w)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    rng = np.random.default_rng(5)
    act = np.sort(rng.choice(w.n, 3000, replace=False)).astype(np.int32)
    dact = torch.tensor(act, device="cuda")
    box = oracle.box_of(w)
    q = act.astype(np.int64)
    nb = oracle.neighbors(box, w.pos, w.lam, q)
    exp, _ = oracle.mhd_rhs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
    g, h, _ = oracle.mls_derivs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
    sc = rhs_term_scales(w.U[:, q], g, h, w.gamma)
    errs = {}
    for mode in ("off", "auto", "on"):
        out = torch.full((8, w.n), float("nan"), dtype=torch.float64, device="cuda")
        phb.mhd_rhs_active(plan, phb.Params(gamma=w.gamma, refine=mode), pos, lam, U, dact, out=out)
        errs[mode] = rhs_err(out.cpu().numpy()[:, act], exp, sc).max()
        if mode != "off":
            assert plan.stats()["refined_tiles"] > 0
    print(errs)
    assert errs["on"] < 1e-5 and errs["auto"] < 1e-5
    assert errs["off"] > errs["on"]
