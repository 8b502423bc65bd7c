"""GPU particle-adaptivity scan vs the oracle (Paper II Sec. 2, Sec. 2.1):
void counts, best test points, clump marks and candidate positions exact."""
import numpy as np
import pytest

import oracle
import workloads
from _gpu import need_gpu, sample, torch

pytestmark = pytest.mark.gpu


def gpu_scan(phb, w, skin=0.0, **kw):
    plan = phb.Plan.for_workload(w, skin=skin)
    pos, lam, _ = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    out = phb.adapt_scan(plan, pos, lam, **kw)
    assert plan.read_status() == 0
    return [o.cpu().numpy() for o in out]


def oracle_scan(w, query=None, **kw):
    box = oracle.box_of(w)
    return oracle.adapt_scan(box, w.pos, w.lam, oracle.neighbors(box, w.pos, w.lam, query), query,
                             **kw)


def holes_and_clumps(n_side, seed, drop=0.08, dup=0.02, jitter=0.1):
    """Jittered lattice with a fraction of sites removed (voids) and a fraction
    doubled at 0.1-0.3 lambda (clumps)."""
    w = workloads.random_modes(n_side, seed=seed, amp=0.01)
    rng = np.random.default_rng(seed)
    keep = rng.random(w.n) > drop
    pos, lam, U = w.pos[:, keep], w.lam[keep], w.U[:, keep]
    d = rng.random(pos.shape[1]) < dup
    off = rng.standard_normal((3, d.sum()))
    off *= (0.1 + 0.2 * rng.random(d.sum())) * lam[d] / np.linalg.norm(off, axis=0)
    pos = np.concatenate([pos, (pos[:, d] + off) % 1.0], axis=1)
    lam = np.concatenate([lam, lam[d]])
    U = np.concatenate([U, U[:, d]], axis=1)
    return workloads.Workload("holes", w.box_lo, w.box_len, w.periodic, np.ascontiguousarray(pos),
                              lam, np.ascontiguousarray(U), w.gamma)


def assert_same(got, exp):
    vc, best, cand, clump = got
    evc, ebest, ecand, eclump = exp
    np.testing.assert_array_equal(vc, evc)
    np.testing.assert_array_equal(best, ebest)
    np.testing.assert_array_equal(clump, eclump)
    np.testing.assert_array_equal(cand, ecand)


@pytest.mark.parametrize("skin", [0.0, 0.004])
def test_holes_and_clumps_exact(skin):
    phb = need_gpu()
    w = holes_and_clumps(20, seed=3)
    got = gpu_scan(phb, w, skin=skin)
    exp = oracle_scan(w)
    assert (exp[0] > 0).sum() > 50 and exp[3].sum() > 20   # the case has voids and clumps
    assert_same(got, exp)


@pytest.mark.parametrize("vf,cf", [(0.8, 0.4), (0.6, 0.2)])
def test_thresholds(vf, cf):
    phb = need_gpu()
    w = holes_and_clumps(16, seed=4, drop=0.15)
    assert_same(gpu_scan(phb, w, void_factor=vf, clump_factor=cf),
                oracle_scan(w, void_factor=vf, clump_factor=cf))


def test_open_box_and_variable_lambda():
    """Shock tube (lambda varies 2x across the fronts) in a box with open
    walls: the walls are voids for the particles next to them."""
    phb = need_gpu()
    w = workloads.shock_tube(20000, seed=6)
    w.periodic[:] = 0
    got = gpu_scan(phb, w)
    exp = oracle_scan(w)
    assert (exp[0] > 0).mean() > 0.2
    assert_same(got, exp)


def test_full_size_sampled():
    """8M shear layer in the benchmark's build configuration, sampled particles."""
    phb = need_gpu()
    w = workloads.config("C5")
    got = gpu_scan(phb, w)
    q = sample(w.n, 2000, seed=9)
    exp = oracle_scan(w, query=q)
    assert_same([got[0][q], got[1][q], got[2][:, q], got[3][q]], exp)
    torch.cuda.empty_cache()


def oracle_apply(w, vf=1.0, cf=0.25):
    box = oracle.box_of(w)
    nb = oracle.neighbors(box, w.pos, w.lam)
    scan = oracle.adapt_scan(box, w.pos, w.lam, nb, void_factor=vf, clump_factor=cf)
    g, h, _ = oracle.mls_derivs(box, w.pos, w.lam, w.U, nb, gamma=w.gamma)
    return oracle.adapt_apply(box, w.pos, w.lam, w.U, nb, scan, g, h, void_factor=vf)


@pytest.mark.parametrize("case", ["holes", "open_shock_tube"])
def test_apply_matches_oracle(case):
    """Deletion and creation: the new set's order, origins, positions and
    lambdas are exact; the new particles' states (second-order Taylor values
    of the FP64 fits) within 1e-12 of each field's scale."""
    phb = need_gpu()
    if case == "holes":
        w = holes_and_clumps(16, seed=12, drop=0.1)
    else:
        w = workloads.shock_tube(12000, seed=13)
        w.periodic[:] = 0
    plan = phb.Plan.for_workload(w)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    p2, l2, U2, org = phb.adapt(plan, phb.Params(gamma=w.gamma, precision="fp64"), pos, lam, U)
    assert plan.read_status() & ~0x04 == 0
    ep, el, eU, eorg = oracle_apply(w)
    np.testing.assert_array_equal(org.cpu().numpy(), eorg)
    np.testing.assert_array_equal(p2.cpu().numpy(), ep)
    np.testing.assert_array_equal(l2.cpu().numpy(), el)
    scale = np.abs(w.U).max(axis=1, keepdims=True)
    assert (np.abs(U2.cpu().numpy() - eU) <= 1e-12 * scale).all()
    n = w.n
    assert (eorg >= n).sum() > 10 and (eorg < n).sum() < n or case == "open_shock_tube"
