"""GPU adjoint of the fused fit + RHS (hand-written reverse mode) against the
oracle's forward-mode derivative and against central finite differences."""
import numpy as np
import pytest

import oracle
import workloads
from _gpu import need_gpu, sample, torch

pytestmark = pytest.mark.gpu


def setup(phb, w, **prm):
    plan = phb.Plan.for_workload(w)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    return plan, pos, lam, U, phb.Params(gamma=w.gamma, precision="fp64", **prm)


@pytest.mark.parametrize("with_terms", [False, True, "laws"])
def test_dot_product_against_oracle_jvp(with_terms):
    """<gbar, J v> from the oracle's dual numbers equals <J^T gbar, v> from the
    GPU adjoint (all particles, neighbour sets fixed); with input zeta / eta,
    and with the coefficient laws on top of them."""
    phb = need_gpu()
    w = workloads.random_modes(12, seed=41, amp=0.05)
    rng = np.random.default_rng(5)
    kw = {}
    zeta = eta = None
    laws = (0.0, 0.0, 0.0)
    if with_terms:
        zeta = rng.uniform(0, 0.05, w.n)
        eta = rng.uniform(0, 0.02, w.n)
        kw = dict(zeta=torch.tensor(zeta, device="cuda"), eta=torch.tensor(eta, device="cuda"))
    if with_terms == "laws":
        laws = (0.8, 2.0, 1.5)
        kw.update(c_zeta_l=laws[0], c_zeta_a=laws[1], c_eta=laws[2])
    plan, pos, lam, U, prm = setup(phb, w, **kw)
    gbar = rng.standard_normal((8, w.n))
    Ub, xb = phb.rhs_adjoint(plan, prm, pos, lam, U, torch.tensor(gbar, device="cuda"))
    Ub, xb = Ub.cpu().numpy(), xb.cpu().numpy()
    vpos = rng.standard_normal((3, w.n)) * w.lam
    vU = rng.standard_normal((8, w.n))
    box = oracle.box_of(w)
    nb = oracle.neighbors(box, w.pos, w.lam)
    _, jv = oracle.rhs_jvp(box, w.pos, w.lam, w.U, vpos, vU, nb, gamma=w.gamma, zeta=zeta, eta=eta,
                           laws=laws)
    lhs = float((gbar * jv).sum())
    rhs = float((Ub * vU).sum() + (xb * vpos).sum())
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0), (lhs, rhs)


def test_gradient_entries_against_oracle_and_central_differences():
    """L = sum_ik r_ik (dU_k/dt)_i: dL/dx and dL/dU on 64 seeded entries vs the
    oracle's exact directional derivatives (unit directions) and vs central
    differences of the GPU FP64 forward (step 1e-6)."""
    phb = need_gpu()
    w = workloads.random_modes(12, seed=42, amp=0.05)
    plan, pos, lam, U, prm = setup(phb, w)
    r = workloads.loss_weights(w.n, seed=7)
    Ub, xb = phb.rhs_adjoint(plan, prm, pos, lam, U, torch.tensor(r, device="cuda"))
    Ub, xb = Ub.cpu().numpy(), xb.cpu().numpy()
    rng = np.random.default_rng(3)
    box = oracle.box_of(w)
    nb = oracle.neighbors(box, w.pos, w.lam)
    out = torch.empty((8, w.n), dtype=torch.float64, device="cuda")
    scale = max(np.abs(Ub).max(), np.abs(xb).max() * w.lam.min())
    for k in range(64):
        which = "x" if k % 3 == 0 else "U"
        i = int(rng.integers(w.n))
        c = int(rng.integers(3 if which == "x" else 8))
        vpos = np.zeros((3, w.n))
        vU = np.zeros((8, w.n))
        (vpos if which == "x" else vU)[c, i] = 1.0
        _, jv = oracle.rhs_jvp(box, w.pos, w.lam, w.U, vpos, vU, nb, gamma=w.gamma)
        exact = float((r * jv).sum())
        got = float(xb[c, i] if which == "x" else Ub[c, i])
        assert abs(got - exact) <= 1e-9 * scale + 1e-9 * abs(exact), (which, c, i, got, exact)
        # central differences of the GPU forward (neighbour lists held fixed)
        h = 1e-6 * (w.lam[i] if which == "x" else 1.0)
        vals = []
        for sgn in (1.0, -1.0):
            p2, U2 = pos.clone(), U.clone()
            (p2 if which == "x" else U2)[c, i] += sgn * h
            phb.mhd_rhs(plan, prm, p2, lam, U2, out=out)
            vals.append(float((out.cpu().numpy() * r).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - exact) <= 1e-6 * max(abs(exact), scale * (w.lam[i] if which == "x" else 1)), \
            (which, c, i, fd, exact)


def test_autograd_function():
    phb = need_gpu()
    w = workloads.random_modes(10, seed=43, amp=0.05)
    plan, pos, lam, U, prm = setup(phb, w)
    pos_t = pos.clone().requires_grad_(True)
    U_t = U.clone().requires_grad_(True)
    r = torch.tensor(workloads.loss_weights(w.n, seed=9), device="cuda")
    loss = (phb.rhs_autograd(pos_t, U_t, lam, plan, prm) * r).sum()
    loss.backward()
    Ub, xb = phb.rhs_adjoint(plan, prm, pos, lam, U, r)
    assert torch.equal(U_t.grad, Ub) and torch.equal(pos_t.grad, xb)
    # forward of the autograd path equals the plain call
    out, _ = phb.mhd_rhs(plan, prm, pos, lam, U)
    assert torch.equal(phb.rhs_autograd(pos, U, lam, plan, prm), out)


def test_deterministic():
    phb = need_gpu()
    w = workloads.random_modes(12, seed=44)
    plan, pos, lam, U, prm = setup(phb, w)
    g = torch.tensor(np.random.default_rng(1).standard_normal((8, w.n)), device="cuda")
    a1 = phb.rhs_adjoint(plan, prm, pos, lam, U, g)
    a2 = phb.rhs_adjoint(plan, prm, pos, lam, U, g)
    assert torch.equal(a1[0], a2[0]) and torch.equal(a1[1], a2[1])


@pytest.mark.parametrize("open_box", [False, True])
def test_stored_factorisations_match_recompute(open_box):
    """The stored-factorisation adjoint (record once, then adjoint from the
    record) gives bit-identical gradients to the recomputing adjoint, including
    particles whose fit is singular (open-box corners)."""
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    w = workloads.random_modes(10, seed=45, amp=0.05)
    if open_box:
        w.periodic[:] = 0
    plan, pos, lam, U, prm = setup(phb, w)
    g = torch.tensor(np.random.default_rng(2).standard_normal((8, w.n)), device="cuda")
    Ub, xb = phb.rhs_adjoint(plan, prm, pos, lam, U, g)
    rec = phb.adjoint_record(plan, prm, pos, lam, U)
    assert rec.numel() == 343 * w.n
    Ub2, xb2 = phb.rhs_adjoint_stored(plan, prm, pos, lam, U, g, rec)
    torch.cuda.synchronize()
    assert torch.equal(Ub, Ub2) and torch.equal(xb, xb2)
    assert bool(plan.read_status() & _lib.FLAG_FIT_SINGULAR) == open_box
    # the autograd path with stored factors
    pos_t = pos.clone().requires_grad_(True)
    U_t = U.clone().requires_grad_(True)
    (phb.rhs_autograd(pos_t, U_t, lam, plan, prm, store_factors=True) * g).sum().backward()
    assert torch.equal(U_t.grad, Ub) and torch.equal(pos_t.grad, xb)


def test_stored_record_too_small_is_rejected():
    phb = need_gpu()
    w = workloads.random_modes(8, seed=46)
    plan, pos, lam, U, prm = setup(phb, w)
    rec = torch.empty(343 * w.n - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(phb.PhbError):
        phb.adjoint_record(plan, prm, pos, lam, U, record=rec)


def test_adjoint_workload_full_size():
    """The adjoint workload at its stated size: 262,144 jittered-lattice
    particles with random-mode fields, L = sum_ik r_ik (dU_k/dt)_i.
    (1) 64 seeded gradient entries (positions and fields) against central
    differences of the GPU FP64 forward (step 1e-6, neighbour sets held) at
    1e-6, and against the oracle's exact directional derivatives (dual numbers
    on the particles whose lists contain the perturbed one) at 1e-9;
    (2) the dot-product identity <r_S, (J v)_S> = <J^T r_S, v> on a
    4,096-particle subset S: the oracle's JVP at S along a random v against the
    GPU adjoint of the loss restricted to S."""
    phb = need_gpu()
    w = workloads.config("C4")
    n = w.n
    plan, pos, lam, U, prm = setup(phb, w)
    r = workloads.loss_weights(n)
    Ub, xb = phb.rhs_adjoint(plan, prm, pos, lam, U, torch.tensor(r, device="cuda"))
    Ub, xb = Ub.cpu().numpy(), xb.cpu().numpy()
    box = oracle.box_of(w)
    rng = np.random.default_rng(2024)
    out_p = torch.empty((8, n), dtype=torch.float64, device="cuda")
    out_m = torch.empty_like(out_p)
    rg = torch.tensor(r, device="cuda")
    scale_u = np.abs(Ub).max()
    scale_x = np.abs(xb).max()
    for k in range(64):
        which = "x" if k % 3 == 0 else "U"
        i = int(rng.integers(n))
        c = int(rng.integers(3 if which == "x" else 8))
        # particles whose right-hand side depends on particle i: i itself and
        # every j that lists i (|x_i - x_j| < r_f,j)
        d = w.pos - w.pos[:, i:i + 1]
        d -= w.box_len[:, None] * np.rint(d / w.box_len[:, None])
        q = np.flatnonzero(((d * d).sum(0) < (2.3 * w.lam) ** 2) | (np.arange(n) == i)).astype(np.int64)
        nb = oracle.neighbors(box, w.pos, w.lam, q)
        vpos = np.zeros((3, n))
        vU = np.zeros((8, n))
        (vpos if which == "x" else vU)[c, i] = 1.0
        _, jv = oracle.rhs_jvp(box, w.pos, w.lam, w.U, vpos, vU, nb, q, gamma=w.gamma)
        exact = float((r[:, q] * jv).sum())
        got = float(xb[c, i] if which == "x" else Ub[c, i])
        sc = scale_x if which == "x" else scale_u
        assert abs(got - exact) <= 1e-9 * sc + 1e-9 * abs(exact), (which, c, i, got, exact)
        h = 1e-6 * (w.lam[i] if which == "x" else 1.0)
        p2, U2 = pos.clone(), U.clone()
        (p2 if which == "x" else U2)[c, i] += h
        phb.mhd_rhs(plan, prm, p2, lam, U2, out=out_p)
        (p2 if which == "x" else U2)[c, i] -= 2 * h
        phb.mhd_rhs(plan, prm, p2, lam, U2, out=out_m)
        # the difference is nonzero only near i: summing it, not the two
        # losses, keeps the rounding of the 2M-term sums out of the estimate
        fd = float(((out_p - out_m) * rg).sum().item()) / (2 * h)
        assert abs(fd - exact) <= 1e-6 * max(abs(exact), sc * (w.lam[i] if which == "x" else 1.0)), \
            (which, c, i, fd, exact)
    # dot-product identity on a 4,096-particle subset
    S = sample(n, 4096, seed=11)
    rS = np.zeros_like(r)
    rS[:, S] = r[:, S]
    UbS, xbS = phb.rhs_adjoint(plan, prm, pos, lam, U, torch.tensor(rS, device="cuda"))
    vpos = rng.standard_normal((3, n)) * w.lam
    vU = rng.standard_normal((8, n)) * 1e-2
    nbS = oracle.neighbors(box, w.pos, w.lam, S)
    _, jv = oracle.rhs_jvp(box, w.pos, w.lam, w.U, vpos, vU, nbS, S, gamma=w.gamma)
    lhs = float((r[:, S] * jv).sum())
    rhs = float((UbS.cpu().numpy() * vU).sum() + (xbS.cpu().numpy() * vpos).sum())
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0), (lhs, rhs)
    del plan
    torch.cuda.empty_cache()
