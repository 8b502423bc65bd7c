"""Pins of the oracle's neighbour sets (Paper II Sec. 2 / Sec. 2.1)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _sets(off, idx):
    return [set(idx[off[a]:off[a + 1]].tolist()) for a in range(len(off) - 1)]


def test_golden_ties_strict_periodic_nonmutual(orc):
    g = json.load(open(os.path.join(HERE, "golden", "neighbors_ties.json")))
    pos = np.ascontiguousarray(np.array(g["pos"], np.float64).T)
    lam = np.array(g["lambda"], np.float64)
    b = g["box"]
    box = orc.make_box(b["lo"], b["len"], b["periodic"])
    off, idx = orc.neighbors(box, pos, lam, rf_factor=g["rf_factor"])
    S = _sets(off, idx)
    for i, j, why in g["expect_in"]:
        assert j in S[i], why
    for i, j, why in g["expect_out"]:
        assert j not in S[i], why


def test_exact_rational_bruteforce_tiny(orc):
    """Brute force in exact rational arithmetic on dyadic inputs (no rounding anywhere)."""
    rng = np.random.default_rng(3)
    n = 60
    pos = rng.integers(0, 64, size=(3, n)) / 64.0
    lam = rng.integers(2, 6, size=n) / 64.0
    box = orc.make_box((0, 0, 0), (1, 1, 1), (1, 1, 0))
    off, idx = orc.neighbors(box, np.ascontiguousarray(pos), lam, rf_factor=2.0)
    S = _sets(off, idx)
    P = [[Fraction(v) for v in pos[:, i]] for i in range(n)]
    for i in range(n):
        r2 = (2 * Fraction(lam[i])) ** 2
        exp = set()
        for j in range(n):
            if j == i:
                continue
            s = Fraction(0)
            for a in range(3):
                d = P[j][a] - P[i][a]
                if a < 2:
                    d -= round(d)
                s += d * d
            if s < r2:
                exp.add(j)
        assert S[i] == exp, i


@pytest.mark.parametrize("periodic", [True, False])
def test_matches_kdtree(orc, periodic):
    """Generic positions (ties have probability zero): scipy's k-d tree ball query."""
    spatial = pytest.importorskip("scipy.spatial")
    w = workloads.shock_tube(6000, seed=11)
    pos, lam = w.pos, w.lam
    if not periodic:
        w.periodic[:] = 0
    box = orc.box_of(w)
    off, idx = orc.neighbors(box, pos, lam)
    S = _sets(off, idx)
    tree = spatial.cKDTree(pos.T, boxsize=w.box_len if periodic else None)
    for i in range(0, w.n, 7):
        ref = set(tree.query_ball_point(pos[:, i], 2.3 * lam[i])) - {i}
        assert S[i] == ref, i


def test_lattice_counts_and_query_subset(orc):
    w = workloads.linear_wave(16)
    box = orc.box_of(w)
    off, idx = orc.neighbors(box, w.pos, w.lam)
    cnt = np.diff(off)
    assert 40 <= cnt.min() and cnt.max() <= 60 and abs(cnt.mean() - 51) < 2
    q = np.array([5, 100, 4095], np.int64)
    off2, idx2 = orc.neighbors(box, w.pos, w.lam, q)
    full = _sets(off, idx)
    assert _sets(off2, idx2) == [full[i] for i in q]
    # skin enlarges the radius additively
    off3, idx3 = orc.neighbors(box, w.pos, w.lam, q, skin=0.01)
    for a, s in enumerate(_sets(off3, idx3)):
        assert full[q[a]] <= s
