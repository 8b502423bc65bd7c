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


def test_frozen_particles_in_uniform_flow():
    """Frozen particles keep x and U bit for bit; the others still advect by V dt
    exactly (every right-hand side vanishes in a uniform state)."""
    phb = need_gpu()
    w = workloads.linear_wave(8, amplitude=0.0)
    w.U[1:4] = np.array([[0.25], [-0.125], [0.5]])
    frozen = np.random.default_rng(5).random(w.n) < 0.3
    dt = 0.015625
    plan = phb.Plan.for_workload(w, skin=0.05)
    pos, lam, U = phb.tensors_of(w)
    prm = phb.Params(gamma=w.gamma, frozen=torch.from_numpy(frozen).cuda())
    phb.pc_step(plan, prm, pos, lam, U, dt)
    assert plan.read_status() == 0
    pos, U = pos.cpu().numpy(), U.cpu().numpy()
    np.testing.assert_array_equal(U, w.U)
    np.testing.assert_array_equal(pos[:, frozen], w.pos[:, frozen])
    np.testing.assert_array_equal(pos[:, ~frozen], w.pos[:, ~frozen] + dt * w.U[1:4, ~frozen])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_frozen_mask_matches_oracle(prec, tol):
    """A frozen shell around a moving interior (the fixed-value boundary of the
    Sec. 3 tests): frozen particles keep their state exactly, the interior
    matches the oracle's masked step, also when replayed from a CUDA graph."""
    phb = need_gpu()
    w = workloads.random_modes(10, seed=24, amp=0.05)
    c = w.box_lo + 0.5 * w.box_len
    r = np.sqrt(((w.pos - c[:, None]) ** 2).sum(0))
    frozen = r > 0.4 * w.box_len.min()
    dt, skin = 0.002, 0.01
    box = oracle.box_of(w)
    op, oU, ns = oracle.pc_step(box, w.pos, w.lam, w.U, dt, gamma=w.gamma, frozen=frozen)
    assert ns == 0
    g, h, _ = oracle.mls_derivs(box, w.pos, w.lam, w.U, oracle.neighbors(box, w.pos, w.lam),
                                gamma=w.gamma)
    sc = dt * rhs_term_scales(w.U, g, h, w.gamma)
    mask = torch.from_numpy(frozen.astype(np.uint8)).cuda()
    prm = phb.Params(gamma=w.gamma, precision=prec, frozen=mask)
    for graph in (False, True):
        plan = phb.Plan.for_workload(w, skin=skin)
        pos, lam, U = phb.tensors_of(w)
        if graph:
            phb.build_neighbors(plan, pos, lam)
            phb.StepGraph(plan, prm, pos, lam, U, dt, steps=1).replay()
        else:
            phb.pc_step(plan, prm, pos, lam, U, dt)
        assert plan.read_status() == 0
        pos, U = pos.cpu().numpy(), U.cpu().numpy()
        assert np.array_equal(pos[:, frozen], w.pos[:, frozen])
        assert np.array_equal(U[:, frozen], w.U[:, frozen])
        m = ~frozen
        assert rhs_err((U - w.U)[:, m], (oU - w.U)[:, m], sc).max() < tol
        assert kind_err((pos - w.pos)[:, m], (op - w.pos)[:, m]).max() < tol


def test_skin_violation_is_flagged():
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    w = workloads.random_modes(8, seed=22, amp=0.05)
    w.U[1] += 1.0
    pos, U, plan = run_pc(phb, w, 0.01, "fp64", skin=0.005)
    assert plan.read_status() & _lib.FLAG_SKIN


@pytest.mark.parametrize("schedule", [0, 1])
def test_step_graph_matches_eager_steps(schedule):
    """Two steps replayed from a captured CUDA graph give bit-identical states to
    two eagerly launched steps (same kernels, no order-dependent sums)."""
    phb = need_gpu()
    w = workloads.random_modes(12, seed=23, amp=0.05)
    dt, skin = 0.002, 0.02
    prm = phb.Params(gamma=w.gamma)
    ref = phb.Plan.for_workload(w, skin=skin, schedule=schedule)
    pos_e, lam, U_e = phb.tensors_of(w)
    phb.build_neighbors(ref, pos_e, lam)
    for _ in range(2):
        phb.pc_step(ref, prm, pos_e, lam, U_e, dt)
    plan = phb.Plan.for_workload(w, skin=skin, schedule=schedule)
    pos_g, _, U_g = phb.tensors_of(w)
    phb.build_neighbors(plan, pos_g, lam)
    g = phb.StepGraph(plan, prm, pos_g, lam, U_g, dt, steps=2)
    g.replay()
    torch.cuda.synchronize()
    assert ref.read_status() == 0 and plan.read_status() == 0
    assert torch.equal(pos_g, pos_e) and torch.equal(U_g, U_e)
    # a second replay continues from the advanced state
    pos0, U0 = pos_g.clone(), U_g.clone()
    g.replay()
    for _ in range(2):
        phb.pc_step(ref, prm, pos_e, lam, U_e, dt)
    torch.cuda.synchronize()
    assert not torch.equal(pos_g, pos0)
    assert torch.equal(pos_g, pos_e) and torch.equal(U_g, U_e)


def test_autotune_returns_a_timed_candidate(tmp_path, monkeypatch):
    phb = need_gpu()
    from paper_1110_0836_gb300 import tune
    monkeypatch.setenv("PHB_TUNE_CACHE", str(tmp_path / "tune.json"))
    w = workloads.shock_tube(20000, seed=3)
    cands = [dict(tile=128, schedule=0, cell_frac=0.5), dict(tile=64, schedule=1, cell_frac=0.5)]
    res = tune.autotune(w, skin=0.0, reps=2, candidates=cands)
    assert {k: res[k] for k in ("tile", "schedule", "cell_frac")} in cands
    assert all(t["ms"] is not None and t["ms"] > 0 for t in res["table"])
    again = tune.autotune(w, skin=0.0, reps=2, candidates=cands)
    assert again == res   # served from the cache file


# Sec. 3.1 setups (rho = 1, P = 1 / gamma, gamma = 5/3, propagation along x)
# and the oblique fast wave of the workload generator.
WAVES = {
    "magnetoacoustic": dict(mode="fast", B0=(0.0, 0.0, np.sqrt(3.0)), P0=0.6),
    "alfven": dict(mode="alfven", B0=(1.0, 0.0, 0.0), P0=0.6),
    "sound": dict(mode="fast", B0=(0.0, 0.0, 0.0), P0=0.6),
    "oblique_fast": dict(mode="fast"),
}


def _evolve_wave(phb, n_side, prec, wave, cfl=0.05, jitter=0.1):
    """One period of an App. A eigenmode (amplitude 1e-6) with the
    predictor-corrector step; mean |U - U_exact| / amplitude summed over the
    eight fields (the relative L1 error of Sec. 3.1), against the travelling
    eigenmode sin(k x - omega t)."""
    w = workloads.linear_wave(n_side, jitter=jitter, **WAVES[wave])
    m = w.meta
    om, k, A, vhat = m["omega"], m["k"], m["amplitude"], m["vhat"]
    T = 2 * np.pi / om
    nsteps = int(np.ceil(T / (cfl * m["h"] * k / om)))
    dt = T / nsteps
    plan = phb.Plan.for_workload(w, skin=0.05 * 2.3 * m["h"])
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    g = phb.StepGraph(plan, phb.Params(gamma=w.gamma, precision=prec), pos, lam, U, dt)
    for _ in range(nsteps):
        g.replay()
    torch.cuda.synchronize()
    assert plan.read_status() == 0
    x = pos[0].cpu().numpy()
    s = A * np.sin(k * x - om * T)
    kv = k * vhat[0]
    ex = workloads.background(w.n, B0=m["B0"], P0=m["P0"], gamma=w.gamma)
    ex[0] += m["rho0"] * kv / om * s
    ex[1:4] += vhat[:, None] * s
    ex[4:7] += ((kv * m["B0"][:, None] - k * m["B0"][0] * vhat[:, None]) / om) * s
    ex[7] += w.gamma * m["P0"] * kv / om * s / (w.gamma - 1)
    return float((np.abs(U.cpu().numpy() - ex).mean(axis=1) / A).sum())


@pytest.mark.parametrize("wave", sorted(WAVES))
def test_linear_wave_convergence_and_mixed_precision(wave):
    """Time-evolved linear waves (Sec. 3.1, App. A): after one period the
    relative L1 error falls at least second order from 16^3 to 32^3 jittered
    lattices (CFL 0.05, so that the spatial error dominates), and the
    FP32-mixed path tracks the FP64 path on the 1e-6 signal."""
    phb = need_gpu()
    e16 = _evolve_wave(phb, 16, "fp64", wave)
    e32 = _evolve_wave(phb, 32, "fp64", wave)
    order = np.log2(e16 / e32)
    assert order >= 2.0, (e16, e32, order)
    m32 = _evolve_wave(phb, 32, "fp32_mixed", wave)
    assert abs(m32 - e32) <= 0.02 * e32, (m32, e32)


def test_host_buffer_step_matches_device_step():
    """phb_pc_step_host on pinned host arrays (eager, and replayed from a graph that
    holds the copies) gives bit-identical states to phb_pc_step on device arrays."""
    phb = need_gpu()
    w = workloads.random_modes(12, seed=24, amp=0.05)
    dt, skin = 0.002, 0.02
    prm = phb.Params(gamma=w.gamma)
    plan = phb.Plan.for_workload(w, skin=skin)
    pos_d, lam_d, U_d = phb.tensors_of(w)
    phb.pc_step(plan, prm, pos_d, lam_d, U_d, dt)
    hpos = torch.as_tensor(w.pos).clone().pin_memory()
    hlam = torch.as_tensor(w.lam).clone().pin_memory()
    hU = torch.as_tensor(w.U).clone().pin_memory()
    opos, oU = torch.empty_like(hpos).pin_memory(), torch.empty_like(hU).pin_memory()
    phb.pc_step_host(plan, prm, hpos, hlam, hU, dt, opos, oU)
    torch.cuda.synchronize()
    assert plan.read_status() == 0
    assert torch.equal(opos, pos_d.cpu()) and torch.equal(oU, U_d.cpu())
    # inputs untouched; in place on the host (outputs = inputs) as well
    assert torch.equal(hpos, torch.as_tensor(w.pos)) and torch.equal(hU, torch.as_tensor(w.U))
    g = phb.HostStepGraph(plan, prm, hpos, hlam, hU, dt, opos, oU)
    opos.zero_(), oU.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(opos, pos_d.cpu()) and torch.equal(oU, U_d.cpu())
    phb.pc_step_host(plan, prm, hpos, hlam, hU, dt)
    torch.cuda.synchronize()
    assert torch.equal(hpos, pos_d.cpu()) and torch.equal(hU, U_d.cpu())
    with pytest.raises(ValueError):
        phb.pc_step_host(plan, prm, pos_d, lam_d, U_d, dt)


def _corrector_marks(phb, plan):
    """Per slot: 1 where the corrector's fit of the last host-buffer step wrote
    U^{n+1} to the host itself (the step part of the workspace ends with these
    n bytes, 256-byte aligned)."""
    from paper_1110_0836_gb300 import _lib
    _, end = _lib.workspace_part(plan.c, _lib.PART_STEP)
    n = plan.n
    b = end - ((n + 255) // 256) * 256
    return plan.ws[b:b + n].cpu().numpy()


@pytest.mark.parametrize("order", ["storage", "generator"])
def test_host_step_direct_write_matches_device_step(order):
    """phb_pc_step_host with page-locked outputs: the corrector's fit writes
    U^{n+1} straight to the host wherever a warp's slots have nearby caller
    indices (most particles in the library's storage order, few in the
    generator's) and the step copies the rest; with frozen particles, fits
    routed to FP64 and fits queued for the corrected step, the outputs equal
    phb_pc_step's bit for bit, and so do pageable outputs (one copy)."""
    phb = need_gpu()
    w = workloads.shear_layer(20_000, seed=12)
    vmax = float(np.sqrt((w.U[1:4] ** 2).sum(0)).max())
    dt = 0.05 * float(w.lam.min()) / max(vmax, 1.0)
    skin = max(4.0 * dt * vmax, 0.02 * 2.3 * float(w.lam.min()))
    plan = phb.Plan.for_workload(w, skin=skin)
    pos_d, lam_d, U_d = phb.tensors_of(w)
    frozen = np.random.default_rng(3).random(w.n) < 0.1
    if order == "storage":
        phb.build_neighbors(plan, pos_d, lam_d)
        perm = phb.reorder(plan, pos_d, lam_d, U_d)
        frozen = frozen[perm.cpu().numpy()]
    prm = phb.Params(gamma=w.gamma, refine="on", cond_threshold=300.0,
                     frozen=torch.from_numpy(frozen).cuda())
    hpos, hlam, hU = (t.cpu().pin_memory() for t in (pos_d, lam_d, U_d))
    opos, oU = torch.empty_like(hpos).pin_memory(), torch.empty_like(hU).pin_memory()
    phb.pc_step_host(plan, prm, hpos, hlam, hU, dt, opos, oU)
    torch.cuda.synchronize()
    host_status = plan.read_status()
    marks = _corrector_marks(phb, plan)
    st = plan.stats()
    assert st["routed_to_fp64"] > 0 and st["refined_tiles"] == st["tiles"]
    plan.reset_status()
    phb.pc_step(plan, prm, pos_d, lam_d, U_d, dt)
    torch.cuda.synchronize()
    assert plan.read_status() == host_status
    assert torch.equal(opos, pos_d.cpu()) and torch.equal(oU, U_d.cpu())
    assert np.array_equal(oU.numpy()[:, frozen], hU.numpy()[:, frozen])
    # every solved fit is queued for the corrected step here (refine "on",
    # lambda varies, the records fit in L2): tiles write only the few fits
    # they finish themselves (too few neighbours to solve)
    assert marks.mean() < 0.05
    # pageable outputs: the copy after the step
    ppos, pU = torch.empty_like(hpos), torch.empty_like(hU)
    assert not pU.is_pinned()
    phb.pc_step_host(plan, prm, hpos, hlam, hU, dt, ppos, pU)
    torch.cuda.synchronize()
    assert torch.equal(ppos, pos_d.cpu()) and torch.equal(pU, U_d.cpu())


@pytest.mark.parametrize("order", ["storage", "generator"])
def test_host_step_direct_write_plain_fits(order):
    """The same on a lattice (no refined tile, no fit routed to FP64: the
    lattice's fits are all about equally well conditioned) with some
    particles frozen: in storage order the corrector's tiles write every
    other particle's U^{n+1} to the host, in the generator's order few; the
    outputs equal phb_pc_step's bit for bit either way."""
    phb = need_gpu()
    w = workloads.random_modes(24, seed=26, amp=0.05)
    dt, skin = 0.002, 0.02
    plan = phb.Plan.for_workload(w, skin=skin)
    pos_d, lam_d, U_d = phb.tensors_of(w)
    frozen = np.random.default_rng(4).random(w.n) < 0.05
    if order == "storage":
        phb.build_neighbors(plan, pos_d, lam_d)
        perm = phb.reorder(plan, pos_d, lam_d, U_d)
        frozen = frozen[perm.cpu().numpy()]
    hpos, hlam, hU = (t.cpu().pin_memory() for t in (pos_d, lam_d, U_d))
    opos, oU = torch.empty_like(hpos).pin_memory(), torch.empty_like(hU).pin_memory()
    prm = phb.Params(gamma=w.gamma, refine="off", frozen=torch.from_numpy(frozen).cuda())
    phb.pc_step_host(plan, prm, hpos, hlam, hU, dt, opos, oU)
    torch.cuda.synchronize()
    assert plan.stats()["routed_to_fp64"] == 0
    host_status = plan.read_status()
    marks = _corrector_marks(phb, plan)
    plan.reset_status()
    phb.pc_step(plan, prm, pos_d, lam_d, U_d, dt)
    torch.cuda.synchronize()
    assert plan.read_status() == host_status
    assert torch.equal(opos, pos_d.cpu()) and torch.equal(oU, U_d.cpu())
    if order == "storage":
        assert marks.sum() == w.n - frozen.sum()
    else:
        assert marks.mean() < 0.5
        assert marks.sum() <= w.n - frozen.sum()


def _split_fp64(v):
    """FP32 hi/lo split by its definition: h = fl32(v), l = fl32(v - h)."""
    h = v.astype(np.float32)
    return h, (v - h.astype(np.float64)).astype(np.float32)


def test_records_are_the_fp64_hilo_split_bit_for_bit():
    """The FP32 hi/lo records the fits read (split on the integer pipe) equal
    h = fl32(v), l = fl32(v - h) bit for bit, for ordinary values and for
    zeros, tiny, huge, exactly representable and tie-rounding ones."""
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    import ctypes as C
    w = workloads.random_modes(16, seed=41)
    rng = np.random.default_rng(3)
    n = w.n
    U = w.U.copy()
    special = np.array([0.0, -0.0, 1e-30, -3e-25, 7.5e-23, 2.0**-74, 2.0**-75, 1e30, -2.5e37,
                        2.0**126 * 1.9, 1.0, -2.0, (2.0**24 + 1.0) * 2.0**-24,
                        (2.0**23 + 0.5) * 2.0**-20, (2.0**23 + 1.5) * 2.0**-20,
                        1.0 + 2.0**-24, 1.0 + 3 * 2.0**-25])
    idx = rng.choice(n, size=(4, special.size), replace=False)
    for f, row in zip((4, 5, 6, 7), idx):
        U[f, row] = special
    plan = phb.Plan.for_workload(w)
    pos, lam, Ud = phb.tensors_of(w)
    Ud.copy_(torch.as_tensor(U))
    phb.build_neighbors(plan, pos, lam)
    perm = phb.reorder(plan, pos, lam, Ud).cpu().numpy()   # arrays now in slot order
    phb.build_neighbors(plan, pos, lam)
    phb.mhd_rhs(plan, phb.Params(gamma=w.gamma, precision="fp64"), pos, lam, Ud)
    torch.cuda.synchronize()
    off, nbytes = C.c_size_t(), C.c_size_t()
    assert _lib.lib().phb_record_region(C.byref(plan.c), C.byref(off), C.byref(nbytes)) == 0
    assert nbytes.value == n * 24 * 4
    rec = plan.ws[off.value:off.value + nbytes.value].view(torch.float32).cpu().numpy()
    rec = rec.reshape(n, 24)
    P, Us = pos.cpu().numpy(), Ud.cpu().numpy()
    assert np.array_equal(Us, U[:, perm])
    xh, xl = _split_fp64(P)
    uh, ul = _split_fp64(Us)
    layout = {0: xh[0], 1: xh[1], 2: xh[2], 4: xl[0], 5: xl[1], 6: xl[2],
              8: uh[0], 9: uh[7], 10: uh[1], 11: uh[2], 12: ul[0], 13: ul[7], 14: ul[1],
              15: ul[2], 16: uh[3], 17: uh[4], 18: uh[5], 19: uh[6], 20: ul[3], 21: ul[4],
              22: ul[5], 23: ul[6]}
    for col, want in layout.items():
        got = rec[:, col]
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), col
