"""Pins of the oracle's MLS fit and derivatives (Paper II Sec. 2, Acknowledgements)."""
import numpy as np
import pytest

import workloads
from _analytic import cubic_exponents, poly3, rel_err


def _open_lattice(n_side=12, seed=5):
    pos, h = workloads.lattice_positions(n_side, seed, jitter=0.2)
    lam = np.full(pos.shape[1], h)
    return pos, lam, h


@pytest.mark.parametrize("weight_kind", [0, 1])
def test_cubic_reproduction(orc, weight_kind):
    """A cubic field lies in the span of the interpolating cubic basis, so the
    least-squares fit reproduces it exactly at every particle with a
    non-singular fit: fitted gradient and Hessian equal the analytic ones."""
    pos, lam, h = _open_lattice()
    n = pos.shape[1]
    box = orc.make_box((0, 0, 0), (1, 1, 1), (0, 0, 0))
    rng = np.random.default_rng(1)
    U = np.zeros((8, n))
    G = np.zeros((8, 3, n))
    H = np.zeros((8, 6, n))
    for f in range(8):
        coef = {a: rng.uniform(-1, 1) for a in cubic_exponents()}
        U[f], G[f], H[f] = poly3(coef, pos)
    nb = orc.neighbors(box, pos, lam)
    g, hh, st = orc.mls_derivs(box, pos, lam, U, nb, weight_kind=weight_kind)
    ok = st == 0
    assert ok.mean() > 0.95   # boundary particles with lopsided sets may be singular-free too
    assert rel_err(g[:, :, ok], G[:, :, ok]).max() < 1e-11
    assert rel_err(hh[:, :, ok], H[:, :, ok]).max() < 1e-10


def test_matches_library_lstsq(orc):
    """Weighted least squares through numpy's SVD-based lstsq on the same system."""
    w = workloads.random_modes(12, seed=2)
    box = orc.box_of(w)
    q = np.array([0, 17, 500, 1200], np.int64)
    off, idx = orc.neighbors(box, w.pos, w.lam, q)
    g, hh, st = orc.mls_derivs(box, w.pos, w.lam, w.U, (off, idx), q)
    ex = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
          (0, 0, 2), (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0),
          (0, 2, 1), (0, 1, 2), (0, 0, 3)]
    for a, i in enumerate(q):
        J = idx[off[a]:off[a + 1]]
        d = w.pos[:, J] - w.pos[:, [i]]
        d -= np.round(d)
        rf = 2.3 * w.lam[i]
        sw = 1.0 - (d * d).sum(0) / rf ** 2
        qq = d / w.lam[i]
        P = np.stack([np.prod(qq ** np.array(e)[:, None], axis=0) for e in ex], axis=1)
        R = (w.U[:, J] - w.U[:, [i]]).T
        c = np.linalg.lstsq(sw[:, None] * P, sw[:, None] * R, rcond=None)[0]
        li = w.lam[i]
        np.testing.assert_allclose(g[:, :, a], (c[0:3] / li).T, rtol=1e-9, atol=1e-12)
        hexp = np.stack([2 * c[3], c[4], c[5], 2 * c[6], c[7], 2 * c[8]]) / li ** 2
        np.testing.assert_allclose(hh[:, :, a], hexp.T, rtol=1e-8, atol=1e-10)


def test_exactly_19_neighbours_interpolate(orc):
    """With 19 neighbours in general position the cubic interpolates them: the
    solution is unique and independent of the weights."""
    rng = np.random.default_rng(7)
    n = 20
    pos = np.ascontiguousarray(0.5 + rng.uniform(-0.08, 0.08, size=(3, n)))
    pos[:, 0] = 0.5
    lam = np.full(n, 0.1)
    box = orc.make_box((0, 0, 0), (1, 1, 1), (0, 0, 0))
    U = rng.standard_normal((8, n))
    q = np.array([0], np.int64)
    nb = orc.neighbors(box, pos, lam, q)
    assert nb[0][1] == 19
    g0, h0, s0 = orc.mls_derivs(box, pos, lam, U, nb, q, weight_kind=0)
    g1, h1, s1 = orc.mls_derivs(box, pos, lam, U, nb, q, weight_kind=1)
    assert s0[0] == 0 and s1[0] == 0
    np.testing.assert_allclose(g0, g1, rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(h0, h1, rtol=1e-8, atol=1e-7)


def test_singular_fits(orc):
    rng = np.random.default_rng(8)
    # (a) fewer than 19 neighbours
    n = 15
    pos = np.ascontiguousarray(0.5 + rng.uniform(-0.05, 0.05, size=(3, n)))
    lam = np.full(n, 0.1)
    box = orc.make_box((0, 0, 0), (1, 1, 1), (0, 0, 0))
    U = rng.standard_normal((8, n))
    nb = orc.neighbors(box, pos, lam)
    g, h, st = orc.mls_derivs(box, pos, lam, U, nb)
    assert (st == 1).all() and not g.any() and not h.any()
    out, st2 = orc.mhd_rhs(box, pos, lam, U, nb)
    assert (st2 == 1).all() and not out.any()
    # (b) coplanar neighbours: z-monomials vanish, the fit is rank deficient
    n = 60
    pos = np.ascontiguousarray(0.5 + rng.uniform(-0.05, 0.05, size=(3, n)))
    pos[2] = 0.5
    U = rng.standard_normal((8, n))
    nb = orc.neighbors(box, pos, np.full(n, 0.1))
    g, h, st = orc.mls_derivs(box, pos, np.full(n, 0.1), U, nb)
    assert (st == 1).all()


def _rotation(seed):
    A = np.random.default_rng(seed).standard_normal((3, 3))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def test_rotation_equivariance(orc):
    """The cubic span and the radial weight are rotation invariant, so rotating
    particles and vector fields rotates V, B derivatives and the RHS."""
    w = workloads.random_modes(12, seed=4, amp=0.2)
    n = w.n
    R = _rotation(9)
    c = np.full((3, 1), 0.5)
    pos2 = np.ascontiguousarray(c + R @ (w.pos - c))
    U2 = w.U.copy()
    U2[1:4] = R @ w.U[1:4]
    U2[4:7] = R @ w.U[4:7]
    box = orc.make_box((-1, -1, -1), (3, 3, 3), (0, 0, 0))
    q = np.arange(0, n, 11, dtype=np.int64)
    nb = orc.neighbors(box, w.pos, w.lam, q)
    o1, s1 = orc.mhd_rhs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
    o2, s2 = orc.mhd_rhs(box, pos2, w.lam, U2, nb, q, gamma=w.gamma)
    np.testing.assert_array_equal(s1, s2)   # open-box corners may be singular in both
    ok = s1 == 0
    assert ok.mean() > 0.9
    exp = o1.copy()
    exp[1:4] = R @ o1[1:4]
    exp[4:7] = R @ o1[4:7]
    assert rel_err(o2[:, ok], exp[:, ok]).max() < 1e-11
    g1, h1, _ = orc.mls_derivs(box, w.pos, w.lam, w.U, nb, q)
    g2, h2, _ = orc.mls_derivs(box, pos2, w.lam, U2, nb, q)
    # scalar fields: the gradient rotates as a vector, the Hessian as R H R^T
    for f in (0, 7):
        assert rel_err(g2[f][:, ok], (R @ g1[f])[:, ok]).max() < 1e-11
        H1 = h1[f][[0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(3, 3, -1)
        H2 = h2[f][[0, 1, 2, 1, 3, 4, 2, 4, 5]].reshape(3, 3, -1)
        RHR = np.einsum("ab,bcn,dc->adn", R, H1, R)
        assert rel_err(H2[..., ok].reshape(9, -1), RHR[..., ok].reshape(9, -1)).max() < 1e-10


def test_translation_invariance(orc):
    w = workloads.random_modes(12, seed=6, amp=0.2)
    box = orc.make_box((-1, -1, -1), (3, 3, 3), (0, 0, 0))
    q = np.arange(0, w.n, 13, dtype=np.int64)
    nb = orc.neighbors(box, w.pos, w.lam, q)
    o1, s1 = orc.mhd_rhs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
    pos2 = np.ascontiguousarray(w.pos + np.array([[0.3125], [-0.25], [0.125]]))
    o2, s2 = orc.mhd_rhs(box, pos2, w.lam, w.U, nb, q, gamma=w.gamma)
    np.testing.assert_array_equal(s1, s2)
    assert rel_err(o2, o1).max() < 1e-12
