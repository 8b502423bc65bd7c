"""GPU fused fit + RHS vs the FP64 oracle (Paper II Sec. 2; App. A).

Bars (per field and per derivative kind: max_i |a - o| / max_i |o|; time
derivatives per field against the scale of that equation's terms): FP64 path
1e-12, FP32-mixed path 1e-5 on every workload."""
import numpy as np
import pytest

import oracle
import workloads
from _gpu import kind_err, need_gpu, rhs_err, rhs_term_scales, sample, torch

pytestmark = pytest.mark.gpu


def gpu_run(phb, w, params, mode="rhs", skin=0.0, plan=None):
    plan = plan or phb.Plan.for_workload(w, skin=skin)
    pos, lam, U = phb.tensors_of(w)
    phb.build_neighbors(plan, pos, lam)
    st = torch.full((w.n,), -1, dtype=torch.int32, device="cuda")
    if mode == "rhs":
        out, _ = phb.mhd_rhs(plan, params, pos, lam, U, fit_status=st)
        res = out.cpu().numpy()
    else:
        g, h, _ = phb.mls_derivs(plan, params, pos, lam, U, out=None)
        st = _
        res = (g.cpu().numpy(), h.cpu().numpy())
    torch.cuda.synchronize()
    return res, st.cpu().numpy(), plan


def oracle_run(w, mode="rhs", query=None, **kw):
    box = oracle.box_of(w)
    nb = oracle.neighbors(box, w.pos, w.lam, query)
    if mode == "rhs":
        return oracle.mhd_rhs(box, w.pos, w.lam, w.U, nb, query, gamma=w.gamma, **kw)
    g, h, st = oracle.mls_derivs(box, w.pos, w.lam, w.U, nb, query, gamma=w.gamma, **kw)
    return (g, h), st


def term_scales(w, query=None, zeta=None, eta=None, **kw):
    """Scale of each RHS equation's terms at the (query) particles, from oracle derivatives."""
    (g, h), _ = oracle_run(w, "derivs", query, **kw)
    q = slice(None) if query is None else query
    return rhs_term_scales(w.U[:, q], g, h, w.gamma,
                           None if zeta is None else zeta[q], None if eta is None else eta[q])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_derivs_small_lattice(prec, tol):
    phb = need_gpu()
    w = workloads.random_modes(16, seed=2)
    (g, h), st, plan = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision=prec), mode="derivs")
    (go, ho), sto = oracle_run(w, "derivs")
    assert not sto.any() and not st.any()
    assert kind_err(g, go).max() < tol, kind_err(g, go)
    assert kind_err(h, ho).max() < tol, kind_err(h, ho)
    plan.raise_status()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
@pytest.mark.parametrize("which", ["modes", "wave"])
def test_rhs_small(prec, tol, which):
    phb = need_gpu()
    w = workloads.random_modes(16, seed=3) if which == "modes" else workloads.linear_wave(16)
    out, st, plan = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision=prec))
    exp, sto = oracle_run(w)
    assert (st == 0).all()
    e = rhs_err(out, exp, term_scales(w))
    assert e.max() < tol, e


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("name,nq", [("C2", 600), ("C3", 300), ("C5", 1024)])
def test_rhs_full_size_sampled(prec, name, nq):
    """Full-size sets in the benchmark's launch configuration, sampled particles:
    64^3 lattice, 1,048,576-particle shock tube, 8,000,000-particle shear layer.
    Time derivatives (term-scaled) and the gradients and Hessians of all eight
    fields (scaled by the sample's largest value of each kind) meet 1e-12 in
    FP64 and 1e-5 in FP32-mixed; the term scales are maxima over the sample,
    so the sample must be large enough to see the equation's largest terms."""
    tol = 1e-12 if prec == "fp64" else 1e-5
    phb = need_gpu()
    w = workloads.config(name)
    prm = phb.Params(gamma=w.gamma, precision=prec)
    out, st, plan = gpu_run(phb, w, prm)
    q = sample(w.n, nq, seed=7)
    exp, sto = oracle_run(w, query=q)
    (go, ho), _ = oracle_run(w, "derivs", query=q)
    sc = rhs_term_scales(w.U[:, q], go, ho, w.gamma)
    e = rhs_err(out[:, q], exp, sc)
    print(name, prec, "max term-scaled error", e.max(), "refined tiles", plan.stats()["refined_tiles"])
    assert e.max() < tol, e
    assert (st[q] == sto).all() or prec == "fp32_mixed"
    (g, h), _, _ = gpu_run(phb, w, prm, mode="derivs", plan=plan)
    eg, eh = kind_err(g[:, :, q], go), kind_err(h[:, :, q], ho)
    print(name, prec, "gradients", eg.max(), "Hessians", eh.max())
    assert eg.max() < tol, eg
    assert eh.max() < tol, eh
    del plan
    torch.cuda.empty_cache()


def test_viscosity_and_divb_terms_fp64():
    phb = need_gpu()
    w = workloads.random_modes(14, seed=5, amp=0.05)
    rng = np.random.default_rng(1)
    zeta = rng.uniform(0.0, 0.05, w.n)
    eta = rng.uniform(0.0, 0.02, w.n)
    prm = phb.Params(gamma=w.gamma, precision="fp64", zeta=torch.tensor(zeta, device="cuda"),
                     eta=torch.tensor(eta, device="cuda"))
    out, st, _ = gpu_run(phb, w, prm)
    exp, _ = oracle_run(w, zeta=zeta, eta=eta)
    sc = term_scales(w, zeta=zeta, eta=eta)
    assert rhs_err(out, exp, sc).max() < 1e-12
    prm.precision = "fp32_mixed"
    out, st, _ = gpu_run(phb, w, prm)
    assert rhs_err(out, exp, sc).max() < 1e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_mixed", 1e-5)])
def test_coefficient_laws(prec, tol):
    """zeta += C_l lambda c + C_a lambda^2 max(0, -div V), eta += C_eta lambda c on
    top of input coefficients, against the oracle; term scales with each
    particle's resulting coefficients."""
    phb = need_gpu()
    w = workloads.random_modes(14, seed=7, amp=0.05)
    rng = np.random.default_rng(3)
    zeta = rng.uniform(0.0, 0.02, w.n)
    eta = rng.uniform(0.0, 0.01, w.n)
    laws = (0.8, 2.0, 1.5)
    prm = phb.Params(gamma=w.gamma, precision=prec, zeta=torch.tensor(zeta, device="cuda"),
                     eta=torch.tensor(eta, device="cuda"), c_zeta_l=laws[0], c_zeta_a=laws[1],
                     c_eta=laws[2])
    out, st, _ = gpu_run(phb, w, prm)
    exp, _ = oracle_run(w, zeta=zeta, eta=eta, laws=laws)
    base, _ = oracle_run(w, zeta=zeta, eta=eta)
    (g, h), _ = oracle_run(w, "derivs")
    divV = g[1, 0] + g[2, 1] + g[3, 2]
    P = (w.gamma - 1.0) * w.U[7]
    c = np.sqrt((w.gamma * P + (w.U[4:7] ** 2).sum(0)) / w.U[0])
    zt = zeta + laws[0] * w.lam * c + laws[1] * w.lam ** 2 * np.maximum(0.0, -divV)
    et = eta + laws[2] * w.lam * c
    assert (divV < 0).any() and (divV > 0).any()
    sc = term_scales(w, zeta=zt, eta=et)
    assert rhs_err(out, exp, sc).max() < tol
    assert rhs_err(base, exp, sc).max() > 100 * tol     # the laws change the result


def test_unweighted_fit():
    phb = need_gpu()
    w = workloads.random_modes(14, seed=6)
    out, st, _ = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision="fp64", weight_kind=1))
    exp, _ = oracle_run(w, weight_kind=1)
    assert rhs_err(out, exp, term_scales(w, weight_kind=1)).max() < 1e-12


def test_singular_fits_open_box():
    """Open-box corner particles have fewer than 19 neighbours: status 1 and
    zero derivatives on both sides."""
    phb = need_gpu()
    w = workloads.random_modes(10, seed=8)
    w.periodic[:] = 0
    from paper_1110_0836_gb300 import _lib
    for prec in ("fp64", "fp32_mixed"):
        (g, h), st, plan = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision=prec), "derivs")
        (go, ho), sto = oracle_run(w, "derivs")
        assert sto.any()
        sing = sto == 1
        assert (st[sing] == 1).all()
        assert not g[:, :, sing].any() and not h[:, :, sing].any()
        ok = ~sing & (st != 1)
        # interior particles (full neighbour spheres) meet the bars; fits at the
        # open faces are one-sided and so ill-conditioned that the least-squares
        # solution itself moves at ~1e-10 under FP64 rounding (QR or not)
        rf = 2.3 * w.lam.max()
        inner = ok & np.all((w.pos > rf) & (w.pos < 1 - rf), axis=0)
        edge = ok & ~inner
        tol_in, tol_edge = (1e-12, 1e-8) if prec == "fp64" else (1e-5, 1e-3)
        scale = np.abs(go[:, :, ok]).max(axis=(1, 2))
        assert (np.abs(g[:, :, inner] - go[:, :, inner]).max(axis=(1, 2)) / scale).max() < tol_in
        assert (np.abs(g[:, :, edge] - go[:, :, edge]).max(axis=(1, 2)) / scale).max() < tol_edge
        assert plan.read_status() & _lib.FLAG_FIT_SINGULAR


def test_forced_fp64_routing():
    """cond_threshold = 1 routes every fit of the mixed path to the FP64 kernel."""
    phb = need_gpu()
    w = workloads.random_modes(12, seed=10)
    out, st, _ = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision="fp32_mixed",
                                           cond_threshold=1.0))
    exp, _ = oracle_run(w)
    assert (st == 2).all()
    assert rhs_err(out, exp, term_scales(w)).max() < 1e-12


def test_shock_tube_variable_lambda():
    """Density-sampled 8x1x1 shock-tube set (variable lambda, 24-86 neighbours)."""
    phb = need_gpu()
    w = workloads.shock_tube(60000, seed=12)
    q = sample(w.n, 1500, seed=2)
    exp, sto = oracle_run(w, query=q)
    sc = term_scales(w, q)
    out64, st64, _ = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision="fp64"))
    assert rhs_err(out64[:, q], exp, sc).max() < 1e-12
    out32, st32, _ = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision="fp32_mixed"))
    assert rhs_err(out32[:, q], exp, sc).max() < 1e-5
    assert (st32 == 2).mean() < 0.01


@pytest.mark.parametrize("which", ["shear", "lattice"])
def test_corrected_step_modes(which):
    """phb_params.refine: "auto" refines every tile of a density-sampled set
    and none of a jittered lattice; "on" refines every tile; the refined and
    the auto results meet 1e-5 on gradients and Hessians of every field."""
    phb = need_gpu()
    w = workloads.shear_layer(200_000, seed=21) if which == "shear" else workloads.random_modes(24, seed=22)
    q = sample(w.n, 1200, seed=4)
    (go, ho), _ = oracle_run(w, "derivs", query=q)
    plan = phb.Plan.for_workload(w)
    errs = {}
    for mode in ("off", "auto", "on"):
        (g, h), st, plan = gpu_run(phb, w, phb.Params(gamma=w.gamma, refine=mode), "derivs", plan=plan)
        stats = plan.stats()
        errs[mode] = max(kind_err(g[:, :, q], go).max(), kind_err(h[:, :, q], ho).max())
        print(which, mode, errs[mode], stats["refined_tiles"], "of", stats["tiles"])
        if mode == "off":
            assert stats["refined_tiles"] == 0
        elif mode == "on" or which == "shear":
            assert stats["refined_tiles"] == stats["tiles"]
        else:
            assert stats["refined_tiles"] == 0
    assert errs["on"] < 1e-5 and errs["auto"] < 1e-5
    if which == "shear":
        # the corrected step is what meets the bar at the steep layers
        assert errs["off"] > 3 * errs["on"]


def test_nonfinite_input_is_flagged():
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    w = workloads.random_modes(10, seed=13)
    w.U[3, 17] = np.nan
    out, st, plan = gpu_run(phb, w, phb.Params(gamma=w.gamma))
    assert plan.read_status() & _lib.FLAG_NONFINITE


@pytest.mark.parametrize("tile,stage_cap,schedule", [(64, 0, 0), (128, 0, 0), (128, 64, 0),
                                                     (64, 64, 0), (128, 0, 1), (64, 0, 1),
                                                     (128, 64, 1)])
def test_tile_shapes_and_global_fallback(tile, stage_cap, schedule):
    """Both tile sizes, both tile schedules (tiles in cell order, or in
    descending cost order), and a staging capacity so small that
    every tile reads its neighbours from global memory, give the same answers
    within the bars."""
    phb = need_gpu()
    w = workloads.random_modes(16, seed=31)
    # cell edge of half the radius: on this 16^3 box the default cell (one
    # radius, 6 cells per axis) makes most tiles' neighbourhoods span the box
    plan = phb.Plan.for_workload(w, tile=tile, stage_cap=stage_cap, schedule=schedule,
                                 cell_frac=0.5)
    exp, _ = oracle_run(w)
    sc = term_scales(w)
    for prec, tol in (("fp32_mixed", 1e-5), ("fp64", 1e-12)):
        out, st, plan = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision=prec), plan=plan)
        assert rhs_err(out, exp, sc).max() < tol
    stats = plan.stats()
    if stage_cap == 64:
        assert stats["fit_fallback_tiles"] == stats["tiles"] == plan.c.ntiles
    elif tile == 128:
        assert stats["fit_fallback_tiles"] < 0.1 * stats["tiles"]


@pytest.mark.parametrize("n", [1, 2, 5])
def test_tiny_sets_are_singular_everywhere(n):
    """Fewer particles than basis terms: every fit is singular on both sides,
    every derivative and time derivative is zero, the status flag is raised,
    and a predictor-corrector step just advects with V."""
    phb = need_gpu()
    from paper_1110_0836_gb300 import _lib
    rng = np.random.default_rng(n)
    pos = rng.uniform(0.2, 0.8, size=(3, n))
    lam = np.full(n, 0.05)
    U = np.zeros((8, n))
    U[0], U[7] = 1.0, 1.5
    U[1:4] = rng.uniform(-0.1, 0.1, size=(3, n))
    U[4:7] = rng.uniform(-1, 1, size=(3, n))
    w = workloads.Workload("tiny", np.zeros(3), np.ones(3), np.ones(3, np.int32), pos, lam, U,
                           5.0 / 3.0)
    for prec in ("fp64", "fp32_mixed"):
        out, st, plan = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision=prec))
        exp, sto = oracle_run(w)
        assert (sto == 1).all() and (st == 1).all()
        assert not out.any() and not exp.any()
        assert plan.read_status() & _lib.FLAG_FIT_SINGULAR
        plan2 = phb.Plan.for_workload(w, skin=0.01)
        p, l, u = phb.tensors_of(w)
        phb.pc_step(plan2, phb.Params(gamma=w.gamma, precision=prec), p, l, u, 0.01)
        assert np.array_equal(u.cpu().numpy(), U)
        assert np.allclose(p.cpu().numpy(), pos + 0.01 * U[1:4], rtol=0, atol=1e-15)


def test_planar_set_all_fits_singular():
    """A set on one z plane: every monomial with z vanishes, so the normal
    matrix is singular for every particle - status 1 and zero derivatives on
    both sides (the FP32-mixed path routes the failed factorisations to FP64,
    which declares them singular)."""
    phb = need_gpu()
    n_side = 12
    h = 1.0 / n_side
    idx = np.arange(n_side) + 0.5
    X, Y = np.meshgrid(idx * h, idx * h, indexing="ij")
    rng = np.random.default_rng(3)
    pos = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 0.5)])
    pos[:2] += rng.uniform(-0.1 * h, 0.1 * h, size=(2, X.size))
    n = pos.shape[1]
    U = np.zeros((8, n))
    U[0], U[7], U[4] = 1.0, 1.5, 1.0
    U[1] = 0.01 * np.sin(2 * np.pi * pos[0])
    # lambda = 1.5 h: ~37 neighbours in the plane, more than the 19 basis
    # terms, so the singular normal matrix and not the count decides
    w = workloads.Workload("planar", np.zeros(3), np.ones(3), np.array([1, 1, 0], np.int32), pos,
                           np.full(n, 1.5 * h), U, 5.0 / 3.0)
    for prec in ("fp64", "fp32_mixed"):
        (g, hs), st, plan = gpu_run(phb, w, phb.Params(gamma=w.gamma, precision=prec), "derivs")
        (go, ho), sto = oracle_run(w, "derivs")
        assert (sto == 1).all() and (st == 1).all()
        assert not g.any() and not hs.any()
        assert plan.neighbor_total() >= 19 * n


def test_corrected_step_schedules_agree():
    """The corrected step of refined tiles run by the queue kernel and inside the
    tiles gives bit-identical time derivatives and derivatives (same arithmetic,
    the first solves and moments kept in global memory or in shared memory),
    and both meet 1e-5 against the oracle on a density-sampled set."""
    phb = need_gpu()
    w = workloads.shear_layer(150_000, seed=31)
    q = sample(w.n, 600, seed=8)
    exp, _ = oracle_run(w, query=q)
    (go, ho), _ = oracle_run(w, "derivs", query=q)
    sc = rhs_term_scales(w.U[:, q], go, ho, w.gamma)
    plan = phb.Plan.for_workload(w)
    res = {}
    for sched in ("queue", "tile"):
        prm = phb.Params(gamma=w.gamma, refine="on", refine_schedule=sched)
        out, st, plan = gpu_run(phb, w, prm, plan=plan)
        (g, h), _, _ = gpu_run(phb, w, prm, mode="derivs", plan=plan)
        assert plan.stats()["refined_tiles"] == plan.stats()["tiles"]
        res[sched] = (out, g, h)
        assert rhs_err(out[:, q], exp, sc).max() < 1e-5
        assert max(kind_err(g[:, :, q], go).max(), kind_err(h[:, :, q], ho).max()) < 1e-5
    for a, b in zip(res["queue"], res["tile"]):
        assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        phb.Params(gamma=w.gamma, refine_schedule="later").c()


@pytest.mark.parametrize("tile", [64, 128])
def test_corrected_step_under_both_tile_schedules(tile):
    """The corrected step (every tile refined, in both of its schedules) with
    the tiles run in descending cost order gives the time derivatives of the
    cell order bit for bit (the same tiles, staged relative to the same particles),
    and both tile sizes meet 1e-5 against the oracle."""
    phb = need_gpu()
    w = workloads.shear_layer(60_000, seed=33)
    q = sample(w.n, 400, seed=10)
    exp, _ = oracle_run(w, query=q)
    (go, ho), _ = oracle_run(w, "derivs", query=q)
    sc = rhs_term_scales(w.U[:, q], go, ho, w.gamma)
    ref_plan = phb.Plan.for_workload(w, tile=tile, schedule=0)
    plan = phb.Plan.for_workload(w, tile=tile, schedule=1)
    for sched in ("queue", "tile"):
        prm = phb.Params(gamma=w.gamma, refine="on", refine_schedule=sched)
        ref, _, _ = gpu_run(phb, w, prm, plan=ref_plan)
        out, _, _ = gpu_run(phb, w, prm, plan=plan)
        assert np.array_equal(out, ref), sched
        assert plan.stats()["refined_tiles"] == plan.stats()["tiles"]
        assert rhs_err(out[:, q], exp, sc).max() < 1e-5
