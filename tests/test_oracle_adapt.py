"""Pins of the oracle's particle-adaptivity scan (Paper II Sec. 2: particles
are added in voids and deleted in clumps; Sec. 2.1: void search on a 9^3 grid
of test points).  Thresholds are readings: test points within r_f - d_v of
the particle, covered by a particle closer than d_v = lambda, clumps closer
than lambda / 4 (the larger index is marked)."""
import numpy as np

import workloads


def _scan(orc, pos, lam, box, **kw):
    nb = orc.neighbors(box, pos, lam)
    return orc.adapt_scan(box, pos, lam, nb, **kw)


def test_isolated_particle_counts_the_shell(orc):
    """One particle alone: the uncovered test points are the grid points h k
    (h = r_f / 4 = 0.575 lambda) with lambda <= |h k| < 1.3 lambda, i.e.
    |k|^2 in {4, 5}: 6 + 24 = 30 points (|k|^2 = 3 lies at 0.996 lambda and is
    covered by the particle itself).  The farthest are the |k|^2 = 5 points;
    the first of them in grid order is k = (-2, -1, 0)."""
    pos = np.array([[0.5], [0.5], [0.5]])
    lam = np.array([0.01])
    box = orc.make_box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    vc, best, cand, clump = _scan(orc, pos, lam, box)
    assert vc[0] == 30
    assert best[0] == ((-2 + 4) * 9 + (-1 + 4)) * 9 + (0 + 4)
    h = 2.3 * 0.01 / 4
    np.testing.assert_array_equal(cand[:, 0], [0.5 - 2 * h, 0.5 - h, 0.5])
    assert clump[0] == 0


def test_lattice_has_no_voids_or_clumps(orc):
    """Cubic lattice of spacing a = lambda: every point lies within
    sqrt(3)/2 a < lambda of a site, and all those sites are neighbours."""
    pos, h = workloads.lattice_positions(12, 1, jitter=0.0)
    lam = np.full(pos.shape[1], h)
    box = orc.make_box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    vc, best, cand, clump = _scan(orc, pos, lam, box)
    assert not vc.any() and (best == -1).all() and not clump.any()


def test_hole_in_a_lattice(orc):
    """A 2x2x2 block of sites removed from the lattice leaves a void whose
    centre is 1.66 a from the nearest site: only particles next to the hole
    see it, and every void candidate lies inside the hole."""
    a = 1.0 / 12
    g = (np.arange(12) + 0.5) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    c = np.array([6.0, 6.0, 6.0]) * a            # centre of the removed block
    keep = ~np.all(np.abs(pos - c[:, None]) < a, axis=0)
    pos = np.ascontiguousarray(pos[:, keep])
    lam = np.full(pos.shape[1], a)
    box = orc.make_box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    vc, best, cand, clump = _scan(orc, pos, lam, box)
    dist = np.sqrt(((pos - c[:, None]) ** 2).sum(0))
    assert vc.any() and not clump.any()
    assert (dist[vc > 0] < 2.5 * a).all()              # only the hole's surroundings
    assert (vc[dist > 3.0 * a] == 0).all()
    cd = np.sqrt(((cand[:, vc > 0] - c[:, None]) ** 2).sum(0))
    assert (cd < 0.8 * a).all()                        # candidates inside the hole


def test_clump_marks_the_larger_index(orc):
    """Two particles 0.1 lambda apart in an otherwise empty box: the one with
    the larger index is marked; a third one at 0.2 lambda from both marks
    itself too; at 0.3 lambda nothing is marked."""
    lam0 = 0.02
    box = orc.make_box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    pos = np.array([[0.5, 0.5 + 0.1 * lam0], [0.5, 0.5], [0.5, 0.5]])
    _, _, _, clump = _scan(orc, pos, np.full(2, lam0), box)
    assert clump.tolist() == [0, 1]
    pos3 = np.array([[0.5, 0.5 + 0.1 * lam0, 0.5 + 0.05 * lam0],
                     [0.5, 0.5, 0.5 + 0.19 * lam0], [0.5, 0.5, 0.5]])
    _, _, _, clump = _scan(orc, pos3, np.full(3, lam0), box)
    assert clump.tolist() == [0, 1, 1]
    pos = np.array([[0.5, 0.5 + 0.3 * lam0], [0.5, 0.5], [0.5, 0.5]])
    _, _, _, clump = _scan(orc, pos, np.full(2, lam0), box)
    assert clump.tolist() == [0, 0]


def test_query_subset_matches_the_full_scan(orc):
    """The sampled form (lists of the query particles only) gives the full
    scan's values at those particles."""
    rng = np.random.default_rng(8)
    pos = rng.random((3, 3000))
    lam = np.full(3000, 0.04)
    box = orc.make_box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    full = _scan(orc, pos, lam, box)
    q = np.sort(rng.choice(3000, 200, replace=False)).astype(np.int64)
    sub = orc.adapt_scan(box, pos, lam, orc.neighbors(box, pos, lam, q), q)
    assert full[0].any() and full[3].any()
    for a, b in zip(full, sub):
        np.testing.assert_array_equal(a[..., q], b)


def _hole_lattice(a, field):
    g = (np.arange(12) + 0.5) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    c = np.array([6.0, 6.0, 6.0]) * a
    keep = ~np.all(np.abs(pos - c[:, None]) < a, axis=0)
    pos = np.ascontiguousarray(pos[:, keep])
    U = field(pos)
    return pos, np.full(pos.shape[1], a), U, c


def _quadratic(pos):
    """Fields quadratic in x (reproduced exactly by the fit and by its
    second-order Taylor value), positive density and energy."""
    x, y, z = pos - 0.5
    U = np.empty((8, pos.shape[1]))
    U[0] = 1.0 + 0.3 * x + 0.2 * y * z
    U[1] = 0.1 * x * x - 0.2 * y
    U[2] = 0.05 * x * y + 0.3 * z
    U[3] = -0.1 * z * z + 0.07 * x
    U[4] = 0.5 + 0.1 * y
    U[5] = 0.2 * x * z
    U[6] = -0.3 + 0.04 * y * y
    U[7] = 2.0 + 0.1 * x * y
    return U


def test_apply_fills_the_hole_with_exact_states(orc):
    """New particles sit inside the hole, take the parent's lambda and the
    field's exact value there (quadratic fields: the fit and its second-order
    Taylor value are exact, in an open box to keep the fields smooth); the
    lowest-index parent of a group of nearby points wins; a second scan sees
    fewer voids."""
    a = 1.0 / 12
    pos, lam, U, c = _hole_lattice(a, _quadratic)
    box = orc.make_box((0, 0, 0), (1, 1, 1), (0, 0, 0))
    nb = orc.neighbors(box, pos, lam)
    scan = orc.adapt_scan(box, pos, lam, nb)
    g, h, st = orc.mls_derivs(box, pos, lam, U, nb)
    p2, l2, U2, origin = orc.adapt_apply(box, pos, lam, U, nb, scan, g, h)
    n = pos.shape[1]
    new = origin >= n
    assert new.sum() >= 1 and new.sum() < (scan[0] > 0).sum()    # deduplicated and walls skipped
    assert np.array_equal(origin[~new], np.arange(n))              # no clumps here
    inside = np.all((p2[:, new] >= 0) & (p2[:, new] < 1), axis=0)
    assert inside.all()                                            # none beyond the open walls
    near = np.sqrt(((pos[:, origin[new] - n] - c[:, None]) ** 2).sum(0)) < 2.5 * a
    assert near.any()
    assert (np.sqrt(((p2[:, new][:, near] - c[:, None]) ** 2).sum(0)) < 0.8 * a).all()
    np.testing.assert_allclose(U2[:, new], _quadratic(p2[:, new]), rtol=0, atol=1e-12)
    assert (l2[new] == a).all()
    nb2 = orc.neighbors(box, p2, l2)
    vc2 = orc.adapt_scan(box, p2, l2, nb2)[0]
    assert vc2.sum() < scan[0].sum()


def test_apply_deletes_the_larger_index_of_a_pair(orc):
    lam0 = 0.02
    box = orc.make_box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    pos = np.array([[0.3, 0.5, 0.5 + 0.1 * lam0], [0.5, 0.5, 0.5], [0.5, 0.5, 0.5]])
    lam = np.full(3, lam0)
    U = np.ones((8, 3))
    nb = orc.neighbors(box, pos, lam)
    scan = orc.adapt_scan(box, pos, lam, nb)
    z = np.zeros((8, 3, 3)), np.zeros((8, 6, 3))
    p2, l2, U2, origin = orc.adapt_apply(box, pos, lam, U, nb, scan, *z)
    survivors = origin[origin < 3]
    assert survivors.tolist() == [0, 1]


def test_void_scan_does_not_depend_on_particle_order(orc):
    """Void counts, best test points and candidates belong to the particle,
    not to its index (the clump mark, by design, does)."""
    rng = np.random.default_rng(12)
    pos = rng.random((3, 2500))
    lam = np.full(2500, 0.045)
    box = orc.make_box((0, 0, 0), (1, 1, 1), (1, 1, 1))
    vc, best, cand, _ = _scan(orc, pos, lam, box)
    p = rng.permutation(2500)
    vc2, best2, cand2, _ = _scan(orc, np.ascontiguousarray(pos[:, p]), lam[p], box)
    assert vc.any()
    np.testing.assert_array_equal(vc2, vc[p])
    np.testing.assert_array_equal(best2, best[p])
    np.testing.assert_array_equal(cand2, cand[:, p])
