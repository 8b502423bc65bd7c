"""GPU neighbour sets vs the oracle's brute force: bit-exact (Paper II Sec. 2.1)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads
from _gpu import need_gpu, sample, sets_of, torch

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def gpu_sets(phb, w, skin=0.0, rf_factor=2.3, **kw):
    plan = phb.Plan.for_workload(w, skin=skin, rf_factor=rf_factor, **kw)
    pos, lam, _ = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    off, idx = phb.export_neighbors(plan)
    return sets_of(off, idx), plan


def oracle_sets(w, query=None, skin=0.0, rf_factor=2.3):
    off, idx = oracle.neighbors(oracle.box_of(w), w.pos, w.lam, query, rf_factor=rf_factor, skin=skin)
    return [idx[off[a]:off[a + 1]] for a in range(len(off) - 1)]


def assert_equal_sets(got, exp, query=None):
    q = range(len(exp)) if query is None else query
    for a, i in enumerate(q):
        g = got[i]
        assert np.array_equal(np.sort(g), np.sort(exp[a])), f"particle {i}: {len(g)} vs {len(exp[a])}"
        assert np.all(np.diff(g) > 0)  # exported ascending, no duplicates


def test_lattice_wave_all_particles():
    phb = need_gpu()
    w = workloads.linear_wave(16)
    got, _ = gpu_sets(phb, w)
    assert_equal_sets(got, oracle_sets(w))


def test_golden_ties():
    phb = need_gpu()
    g = json.load(open(os.path.join(HERE, "golden", "neighbors_ties.json")))
    pos = np.ascontiguousarray(np.array(g["pos"], np.float64).T)
    lam = np.array(g["lambda"], np.float64)
    w = workloads.Workload("ties", np.zeros(3), np.ones(3), np.ones(3, np.int32), pos, lam,
                           np.ones((8, len(lam))), 5 / 3)
    got, _ = gpu_sets(phb, w, rf_factor=g["rf_factor"])
    S = [set(x.tolist()) for x in got]
    for i, j, why in g["expect_in"]:
        assert j in S[i], why
    for i, j, why in g["expect_out"]:
        assert j not in S[i], why
    assert_equal_sets(got, oracle_sets(w, rf_factor=g["rf_factor"]))


def test_variable_lambda_shock_tube():
    phb = need_gpu()
    w = workloads.shock_tube(40000, seed=3)
    got, _ = gpu_sets(phb, w)
    q = sample(w.n, 3000)
    assert_equal_sets(got, oracle_sets(w, q), q)


def test_open_box_and_isolated_particle():
    phb = need_gpu()
    w = workloads.random_modes(10, seed=9)
    w.periodic[:] = 0
    w.pos[:, 0] = (0.999, 0.999, 0.999)   # corner: few neighbours
    got, _ = gpu_sets(phb, w)
    assert_equal_sets(got, oracle_sets(w))


def test_skin_lists():
    phb = need_gpu()
    w = workloads.random_modes(12, seed=4)
    got, _ = gpu_sets(phb, w, skin=0.013)
    assert_equal_sets(got, oracle_sets(w, skin=0.013))


def test_particles_on_periodic_faces():
    phb = need_gpu()
    w = workloads.linear_wave(12)
    h = 1.0 / 12
    # pin a few particles exactly on lo and on lo + len, and one at an offset of len/2
    w.pos[0, :12] = 0.0
    w.pos[1, 12:24] = 1.0
    w.pos[2, 24:30] = 0.5
    got, _ = gpu_sets(phb, w)
    assert_equal_sets(got, oracle_sets(w))
    assert h > 0


def test_capacity_overflow_is_flagged_not_fatal():
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    w = workloads.linear_wave(10)
    plan = phb.Plan.for_workload(w, nbr_capacity=1000)
    pos, lam, _ = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam, check_capacity=False)
    assert plan.read_status() & _lib.FLAG_CAPACITY
    assert plan.neighbor_total() > 1000
    # the convenience path regrows and then matches the oracle
    plan.reset_status()
    phb.build_neighbors(plan, pos, lam)
    off, idx = phb.export_neighbors(plan)
    assert_equal_sets(sets_of(off, idx), oracle_sets(w))


def test_full_size_lattice_sampled():
    """262,144-particle jittered lattice (the benchmark's configuration)."""
    phb = need_gpu()
    w = workloads.config("C2")
    got, plan = gpu_sets(phb, w)
    q = sample(w.n, 400, seed=1)
    assert_equal_sets(got, oracle_sets(w, q), q)
    cnt = np.array([len(x) for x in got])
    assert cnt.min() >= 40 and cnt.max() <= 62


@pytest.mark.parametrize("tile,stage_cap,ell_width", [(64, 0, 0), (128, 64, 0), (128, 0, 8),
                                                      (64, 0, 40)])
def test_tiled_and_fallback_search_agree(tile, stage_cap, ell_width):
    """Tile sizes, unstaged tiles, and single-pass scratch rows shorter than
    every list (ell_width 8) or than some lists (40): identical sets."""
    phb = need_gpu()
    w = workloads.shock_tube(20000, seed=5)
    got, plan = gpu_sets(phb, w, tile=tile, stage_cap=stage_cap, ell_width=ell_width)
    q = sample(w.n, 1500, seed=3)
    assert_equal_sets(got, oracle_sets(w, q), q)
    if stage_cap == 64:
        st = plan.stats()
        assert st["build_fallback_tiles"] == st["tiles"]


@pytest.mark.parametrize("name,nq,skin", [("C3", 400, 0.0), ("C5", 200, 0.0), ("C5", 100, 1e-3)])
def test_full_size_density_sampled_sets(name, nq, skin):
    """1,048,576-particle shock tube and 8,000,000-particle shear layer (lambda
    varying 2x, Poisson placement): sampled lists bit-exact, in the launch
    configuration the benchmark times."""
    phb = need_gpu()
    w = workloads.config(name)
    plan = phb.Plan.for_workload(w, skin=skin)
    pos, lam, _ = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    off, idx = phb.export_neighbors(plan)
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    q = sample(w.n, nq, seed=11)
    got = {int(i): idx[off[i]:off[i + 1]] for i in q}
    assert_equal_sets(got, oracle_sets(w, q, skin=skin), q)
    # the 2x jump of lambda at the refinement band of the shear layer gives
    # coarse particles up to ~5x the mean count and fine ones as few as ~10
    cnt = np.diff(off)
    assert cnt.min() >= 5 and cnt.max() < 400 and 40 < cnt.mean() < 70
    del plan, pos, lam, off, idx
    torch.cuda.empty_cache()


def test_particles_on_the_periodic_boundary():
    """Particles at exactly lo + len and lo, and within a cell of them, on a
    grid whose rounded reciprocal cell edge puts lo + len in the top cell
    (93 cells per unit length): every set still equals the brute force."""
    phb = need_gpu()
    rng = np.random.default_rng(31)
    n = 6000
    lam = np.full(n, 1.0 / 215.0)
    r = 2.3 / 215.0
    assert int(np.floor(1.0 * (1.0 / (1.0 / 93.0)))) < 93   # the rounding this test is about
    x = np.concatenate([np.ones(1500), np.zeros(1500), 1.0 - 2 * r * rng.random(1500),
                        2 * r * rng.random(1500)])
    y = 0.2 * rng.random(n)
    z = rng.choice([0.0, 1.0, 0.5], n, p=[0.2, 0.2, 0.6])
    mid = z == 0.5
    z[mid] = np.where(rng.random(mid.sum()) < 0.5, 0.2 * rng.random(mid.sum()),
                      1.0 - 0.2 * rng.random(mid.sum()))
    pos = np.ascontiguousarray(np.stack([x, y, z]))
    w = workloads.Workload("edge", np.zeros(3), np.ones(3), np.ones(3, np.int32), pos, lam,
                           np.ones((8, n)), 5 / 3)
    got, plan = gpu_sets(phb, w)
    assert list(plan.c.ncell) == [93, 93, 93]
    exp = oracle_sets(w)
    assert sum(len(e) for e in exp) > 10 * n
    assert_equal_sets(got, exp)


def test_reorder_into_storage_order():
    """phb_reorder permutes the caller's arrays into slot order: the lists and
    the right-hand side follow the particles bit for bit, without a rebuild,
    and a rebuild on the reordered arrays gives the same sets."""
    phb = need_gpu()
    w = workloads.shock_tube(30000, seed=5)
    plan = phb.Plan.for_workload(w)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    prm = phb.Params(gamma=w.gamma)
    before, _ = phb.mhd_rhs(plan, prm, pos, lam, U)
    off0, idx0 = phb.export_neighbors(plan)
    sets0 = sets_of(off0, idx0)
    perm = phb.reorder(plan, pos, lam, U)
    assert plan.read_status() == 0
    p = perm.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(p), np.arange(w.n))
    assert np.array_equal(pos.cpu().numpy(), w.pos[:, p])
    assert np.array_equal(lam.cpu().numpy(), w.lam[p])
    assert np.array_equal(U.cpu().numpy(), w.U[:, p])
    after, _ = phb.mhd_rhs(plan, prm, pos, lam, U)
    assert torch.equal(after, before[:, perm.long()])
    inv = np.empty_like(p)
    inv[p] = np.arange(w.n)
    for lists in (sets_of(*phb.export_neighbors(plan)), None):
        if lists is None:
            phb.build_neighbors(plan, pos, lam)
            lists = sets_of(*phb.export_neighbors(plan))
        for i in range(0, w.n, 97):
            assert np.array_equal(np.sort(p[lists[i]]), np.sort(sets0[p[i]])), i
    # storage order: consecutive particles mostly share a cell after the reorder
    cells = np.floor(w.pos[:, p] / np.array(plan.c.cell)[:, None]).astype(np.int64)
    same = np.all(cells[:, 1:] == cells[:, :-1], axis=0).mean()
    assert same > 0.5


def test_positions_outside_the_periodic_box():
    """Positions shifted by whole box lengths on periodic axes (the cell wrap's
    integer division below and above the box, and its FP64 form far outside)
    give the brute-force sets of the same (shifted) positions."""
    phb = need_gpu()
    w = workloads.random_modes(12, seed=43)
    rng = np.random.default_rng(9)
    shifted = w.pos.copy()
    k = rng.choice([-3, -2, -1, 1, 2, 5], size=shifted.shape)
    pick = rng.random(shifted.shape) < 0.3
    shifted[pick] += k[pick] * w.box_len[np.nonzero(pick)[0]]
    shifted[0, 7] += 2.0**31 * w.box_len[0]   # far outside: the FP64 form of the wrap
    w.pos = shifted
    got, plan = gpu_sets(phb, w)
    assert_equal_sets(got, oracle_sets(w))
    assert plan.read_status() == 0


def _with_particles(w, extra_pos, extra_lam):
    """w with particles appended (their states copied from the first ones)."""
    k = extra_pos.shape[1]
    w.pos = np.ascontiguousarray(np.concatenate([w.pos, extra_pos], axis=1))
    w.lam = np.concatenate([w.lam, extra_lam])
    w.U = np.ascontiguousarray(np.concatenate([w.U, w.U[:, :k]], axis=1))
    return w


def test_dense_cluster_in_one_cell():
    """100 particles within a tenth of a lattice spacing of one point of a
    12^3 lattice: one cell holds more particles than a warp searches at once
    (the cell-major search takes them 32 at a time against the same
    candidates); every set equals the brute force."""
    phb = need_gpu()
    w = workloads.random_modes(12, seed=21)
    rng = np.random.default_rng(4)
    h = w.box_len[0] / 12
    c = (w.box_lo + 0.37 * w.box_len)[:, None]
    w = _with_particles(w, c + 0.1 * h * (rng.random((3, 100)) - 0.5), np.full(100, w.lam.min()))
    got, plan = gpu_sets(phb, w)
    assert_equal_sets(got, oracle_sets(w))
    assert plan.read_status() == 0


def test_lambda_spread_within_cells():
    """lambda spread 3x at random over a jittered 24^3 periodic lattice
    (particles of 1 to 3 cells of reach side by side; the particle-major
    search): sampled sets equal the brute force."""
    phb = need_gpu()
    w = workloads.random_modes(24, seed=31)
    rng = np.random.default_rng(8)
    w.lam = w.lam.min() * (1.0 + 2.0 * rng.random(w.n))
    got, plan = gpu_sets(phb, w, nbr_capacity=w.n * 1600)
    q = sample(w.n, 1200, seed=5)
    assert_equal_sets(got, oracle_sets(w, q), q)
    assert plan.read_status() == 0


@pytest.mark.parametrize("cell_frac", [0.5, 0.4])
def test_reach_of_two_cells(cell_frac):
    """lambda twice the spacing of a jittered 20^3 lattice (~400 neighbours,
    scratch rows that hold them) and cells of half or 0.4 of the list radius:
    the cell-major search over a reach of two or three cells per axis (up to
    98 runs per warp), cells of ~16 or ~8 particles; sampled sets equal the
    brute force."""
    phb = need_gpu()
    w = workloads.random_modes(20, seed=37)
    w.lam = 2.0 * w.lam
    got, plan = gpu_sets(phb, w, cell_frac=cell_frac, ell_width=512, nbr_capacity=w.n * 480)
    q = sample(w.n, 1000, seed=9)
    assert_equal_sets(got, oracle_sets(w, q), q)
    assert plan.read_status() == 0


@pytest.mark.parametrize("big_factor", [1.0, 7.0])
def test_open_box(big_factor):
    """Open (non-periodic) 20^3 box, one lambda (the cell-major search, reach
    rows outside the box skipped) or 40 particles of 7x the common lambda
    (the particle-major search); sampled sets, with every large one and its
    cell mates, equal the brute force."""
    phb = need_gpu()
    w = workloads.random_modes(20, seed=33)
    w.periodic = np.zeros(3, np.int32)
    rng = np.random.default_rng(6)
    big = rng.choice(w.n, 40, replace=False)
    w.lam = w.lam.copy()
    w.lam[big] *= big_factor
    got, plan = gpu_sets(phb, w, nbr_capacity=w.n * 400)
    h = w.box_len[0] / 20
    near = np.nonzero(np.min(np.abs(w.pos[:, :, None] - w.pos[:, None, big]).max(axis=0), axis=1) < 3 * h)[0]
    q = np.unique(np.concatenate([sample(w.n, 800, seed=7), big, near]))
    assert_equal_sets(got, oracle_sets(w, q), q)
    assert plan.read_status() == 0


def test_tiny_periodic_box_whole_axis_reach():
    """A 6^3 periodic lattice: the reach of every cell covers each periodic
    axis whole, so the cell-major search leaves every list to the
    particle-major, cell-by-cell path; every set equals the brute force."""
    phb = need_gpu()
    w = workloads.random_modes(6, seed=35)
    got, _ = gpu_sets(phb, w)
    assert_equal_sets(got, oracle_sets(w))
