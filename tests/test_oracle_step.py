"""Pins of the oracle's predictor-corrector step and its forward-mode derivative
(Paper II Sec. 2 'second order predictor-corrector', Sec. 4.2)."""
import numpy as np

import workloads
from _analytic import rel_err


def test_uniform_flow_advects_exactly(orc):
    w = workloads.linear_wave(8, amplitude=0.0)
    w.U[1:4] = np.array([[0.3], [-0.2], [0.1]])
    box = orc.box_of(w)
    dt = 0.0625
    pos, U, ns = orc.pc_step(box, w.pos, w.lam, w.U, dt, gamma=w.gamma)
    assert ns == 0
    np.testing.assert_array_equal(U, w.U)
    np.testing.assert_array_equal(pos, w.pos + dt * w.U[1:4])


def test_heun_is_second_order_in_time(orc):
    """One step against the semi-discrete solution (64 small steps): the local
    error scales as dt^3 (Euler would give dt^2)."""
    w = workloads.linear_wave(8, amplitude=1e-3)
    box = orc.box_of(w)

    def run(dt, steps):
        p, u = w.pos, w.U
        for _ in range(steps):
            p, u, _ = orc.pc_step(box, p, w.lam, u, dt, gamma=w.gamma)
        return u

    errs = []
    for dt in (0.04, 0.02):
        ref = run(dt / 64, 64)
        errs.append(np.abs(run(dt, 1) - ref).max())
    assert errs[0] / errs[1] > 6.5, errs


def test_jvp_matches_central_differences(orc):
    w = workloads.random_modes(10, seed=31, amp=0.05)
    box = orc.box_of(w)
    rng = np.random.default_rng(4)
    q = np.sort(rng.choice(w.n, 120, replace=False)).astype(np.int64)
    nb = orc.neighbors(box, w.pos, w.lam, q)
    dpos = rng.uniform(-1, 1, size=(3, w.n)) * w.lam
    dU = rng.uniform(-1, 1, size=(8, w.n))
    zeta = np.full(w.n, 0.02)
    eta = np.full(w.n, 0.01)
    out, dout = orc.rhs_jvp(box, w.pos, w.lam, w.U, dpos, dU, nb, q, gamma=w.gamma, zeta=zeta,
                            eta=eta)
    base, _ = orc.mhd_rhs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma, zeta=zeta, eta=eta)
    np.testing.assert_array_equal(out, base)
    h = 1e-6
    op, _ = orc.mhd_rhs(box, w.pos + h * dpos, w.lam, w.U + h * dU, nb, q, gamma=w.gamma,
                        zeta=zeta, eta=eta)
    om, _ = orc.mhd_rhs(box, w.pos - h * dpos, w.lam, w.U - h * dU, nb, q, gamma=w.gamma,
                        zeta=zeta, eta=eta)
    fd = (op - om) / (2 * h)
    assert rel_err(dout, fd).max() < 1e-6


def test_frozen_particles_in_uniform_flow(orc):
    """Fixed-value boundaries (the Sec. 3 annulus test keeps particles outside
    a radius range from evolving): in a uniform flow every right-hand side
    vanishes exactly, so frozen particles keep x and U bit for bit while the
    others advect by V dt exactly, although the frozen ones now lag behind."""
    w = workloads.linear_wave(8, amplitude=0.0)
    w.U[1:4] = np.array([[0.3], [-0.2], [0.1]])
    rng = np.random.default_rng(4)
    frozen = rng.random(w.n) < 0.3
    box = orc.box_of(w)
    dt = 0.0625
    pos, U, ns = orc.pc_step(box, w.pos, w.lam, w.U, dt, gamma=w.gamma, frozen=frozen)
    assert ns == 0
    np.testing.assert_array_equal(U, w.U)
    np.testing.assert_array_equal(pos[:, frozen], w.pos[:, frozen])
    np.testing.assert_array_equal(pos[:, ~frozen], w.pos[:, ~frozen] + dt * w.U[1:4, ~frozen])


def test_frozen_mask_all_zero_is_the_plain_step_and_frozen_keep_state(orc):
    w = workloads.random_modes(8, seed=9, amp=0.05)
    box = orc.box_of(w)
    dt = 0.002
    p0, u0, _ = orc.pc_step(box, w.pos, w.lam, w.U, dt, gamma=w.gamma)
    p1, u1, _ = orc.pc_step(box, w.pos, w.lam, w.U, dt, gamma=w.gamma,
                            frozen=np.zeros(w.n, bool))
    assert np.array_equal(p0, p1) and np.array_equal(u0, u1)
    frozen = np.zeros(w.n, bool)
    frozen[: w.n // 4] = True
    p2, u2, _ = orc.pc_step(box, w.pos, w.lam, w.U, dt, gamma=w.gamma, frozen=frozen)
    assert np.array_equal(p2[:, frozen], w.pos[:, frozen])
    assert np.array_equal(u2[:, frozen], w.U[:, frozen])
    assert not np.array_equal(u2[:, ~frozen], w.U[:, ~frozen])


# ---- individual power-of-two time steps (block steps)

def test_block_step_one_level_is_heun(orc):
    """Every particle on level 0: one block step is the plain Heun step; every
    particle on level 1 of max_level 1: two Heun steps of dt/2."""
    w = workloads.random_modes(8, seed=9, amp=0.05)
    box = orc.box_of(w)
    dt = 0.004
    lv0 = np.zeros(w.n, np.int64)
    pb, ub, _ = orc.block_step(box, w.pos, w.lam, w.U, lv0, dt, 0, gamma=w.gamma)
    ph, uh, _ = orc.pc_step(box, w.pos, w.lam, w.U, dt, gamma=w.gamma)
    scale = np.abs(uh - w.U).max()
    assert np.abs(ub - uh).max() <= 1e-13 * scale and np.abs(pb - ph).max() <= 1e-15
    pb, ub, _ = orc.block_step(box, w.pos, w.lam, w.U, lv0 + 1, dt, 1, gamma=w.gamma)
    p2, u2, _ = orc.pc_step(box, w.pos, w.lam, w.U, dt / 2, gamma=w.gamma)
    p2, u2, _ = orc.pc_step(box, p2, w.lam, u2, dt / 2, gamma=w.gamma)
    assert np.abs(ub - u2).max() <= 1e-13 * scale and np.abs(pb - p2).max() <= 1e-15


def test_block_step_uniform_flow_is_exact(orc):
    """A uniform flow has a vanishing right-hand side: whatever the levels,
    every particle advects by V dt exactly and U stays put."""
    w = workloads.linear_wave(8, amplitude=0.0)
    w.U[1:4] = np.array([[0.3], [-0.2], [0.1]])
    box = orc.box_of(w)
    rng = np.random.default_rng(6)
    levels = rng.integers(0, 3, w.n)
    dt = 0.0625
    pos, U, _ = orc.block_step(box, w.pos, w.lam, w.U, levels, dt, 2, gamma=w.gamma)
    assert np.abs(U - w.U).max() <= 1e-15
    assert np.abs(pos - (w.pos + dt * w.U[1:4])).max() <= 1e-15


def test_block_step_two_levels_second_order(orc):
    """A linear wave with half the particles (x < 1/2) on the finer level: the
    error of one block step against the semi-discrete solution (many small
    steps) scales as dt^3, the local error of a second-order scheme; inactive
    neighbours held at their old state instead of predicted would leave dt^2."""
    w = workloads.linear_wave(8, amplitude=1e-3)
    box = orc.box_of(w)
    levels = (w.pos[0] < 0.5).astype(np.int64)

    def ref(dt):
        p, u = w.pos, w.U
        for _ in range(64):
            p, u, _ = orc.pc_step(box, p, w.lam, u, dt / 64, gamma=w.gamma)
        return u

    errs = []
    for dt in (0.04, 0.02):
        _, u, _ = orc.block_step(box, w.pos, w.lam, w.U, levels, dt, 1, gamma=w.gamma)
        errs.append(np.abs(u - ref(dt)).max())
    assert errs[0] / errs[1] > 6.5, errs


def test_block_step_continues_from_its_anchor(orc):
    """Two block steps with the anchor carried over equal two steps where the
    second starts afresh (the anchor derivative at a synchronised time is the
    right-hand side there)."""
    w = workloads.random_modes(8, seed=12, amp=0.05)
    box = orc.box_of(w)
    levels = np.random.default_rng(2).integers(0, 2, w.n)
    dt = 0.003
    p1, u1, anc = orc.block_step(box, w.pos, w.lam, w.U, levels, dt, 1, gamma=w.gamma)
    pa, ua, _ = orc.block_step(box, p1, w.lam, u1, levels, dt, 1, anchor=anc, gamma=w.gamma)
    pb, ub, _ = orc.block_step(box, p1, w.lam, u1, levels, dt, 1, gamma=w.gamma)
    assert np.abs(ua - ub).max() <= 1e-14 * np.abs(ub - w.U).max()
    assert np.abs(pa - pb).max() <= 1e-15
