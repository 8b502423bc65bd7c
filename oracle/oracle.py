"""ctypes front end of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: the slow reference that the CUDA library is checked
against.  Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline
leg and its ``--impl reference`` arm) may import this module.  It imports
nothing from the CUDA package.

Array conventions follow the library: pos [3][n], U [8][n] float64, fields
(rho, Vx, Vy, Vz, Bx, By, Bz, sigma).  Neighbour lists are CSR over a query
list of particle indices, with neighbour indices in increasing order.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")


class Box(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("len", C.c_double * 3), ("periodic", C.c_int32 * 3)]


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("rf_factor", C.c_double), ("weight_kind", C.c_int32),
                ("pad", C.c_int32), ("zeta", C.c_void_p), ("eta", C.c_void_p),
                ("frozen", C.c_void_p), ("c_zeta_l", C.c_double), ("c_zeta_a", C.c_double),
                ("c_eta", C.c_double)]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load(_build.build())
    return _LIB


def load(path: str):
    """Open an oracle shared library at ``path`` and declare its signatures."""
    L = C.CDLL(path)
    L.orc_neighbors.argtypes = [C.POINTER(Box), C.c_int64, _f64p, _f64p, C.c_double, C.c_double,
                                C.c_int64, _i64p, _i64p, C.c_void_p, C.c_int64]
    L.orc_mls_derivs.argtypes = [C.POINTER(Box), C.c_int64, _f64p, _f64p, _f64p, C.POINTER(Params),
                                 C.c_int64, _i64p, _i64p, _i64p, _f64p, C.c_void_p, _i32p]
    L.orc_mhd_rhs.argtypes = [C.POINTER(Box), C.c_int64, _f64p, _f64p, _f64p, C.POINTER(Params),
                              C.c_int64, _i64p, _i64p, _i64p, _f64p, _i32p]
    L.orc_rhs_jvp.argtypes = [C.POINTER(Box), C.c_int64, _f64p, _f64p, _f64p, C.c_void_p,
                              C.c_void_p, C.POINTER(Params), C.c_int64, _i64p, _i64p, _i64p,
                              _f64p, _f64p]
    L.orc_pc_step.argtypes = [C.POINTER(Box), C.c_int64, _f64p, _f64p, _f64p, C.c_double,
                              C.POINTER(Params)]
    L.orc_timestep_levels.argtypes = [C.c_int64, _f64p, _f64p, C.c_double, C.c_double, C.c_double,
                                      C.c_int32, _i64p, _i64p, _i32p]
    L.orc_adapt_scan.argtypes = [C.POINTER(Box), C.c_int64, _f64p, _f64p, C.c_double, C.c_double,
                                 C.c_double, C.c_int64, _i64p, _i64p, _i64p, _i32p, _i32p, _f64p,
                                 _i32p]
    L.orc_adapt_scan.restype = C.c_int64
    for f in ("orc_neighbors", "orc_mls_derivs", "orc_mhd_rhs", "orc_rhs_jvp", "orc_pc_step",
              "orc_timestep_levels"):
        getattr(L, f).restype = C.c_int
    return L


class using:
    """Context manager: route every oracle call through another build of it
    (the mutation tests plant mistakes in a copy of the source)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _LIB
        self.prev = _LIB
        _LIB = load(self.path)
        return self

    def __exit__(self, *exc):
        global _LIB
        _LIB = self.prev
        return False


def make_box(lo, ln, periodic) -> Box:
    b = Box()
    for a in range(3):
        b.lo[a] = float(lo[a])
        b.len[a] = float(ln[a])
        b.periodic[a] = int(periodic[a])
    return b


def box_of(w) -> Box:
    return make_box(w.box_lo, w.box_len, w.periodic)


class _P:
    """Params plus the numpy arrays its pointers refer to (kept alive)."""

    def __init__(self, gamma, rf_factor=2.3, weight_kind=0, zeta=None, eta=None, frozen=None,
                 laws=(0.0, 0.0, 0.0)):
        self.keep = []
        self.p = Params()
        self.p.gamma = float(gamma)
        self.p.rf_factor = float(rf_factor)
        self.p.weight_kind = int(weight_kind)
        self.p.zeta = self._ptr(zeta)
        self.p.eta = self._ptr(eta)
        self.p.c_zeta_l, self.p.c_zeta_a, self.p.c_eta = (float(x) for x in laws)
        self.p.frozen = None
        if frozen is not None:
            fz = np.ascontiguousarray(np.asarray(frozen) != 0, np.uint8)
            self.keep.append(fz)
            self.p.frozen = fz.ctypes.data

    def _ptr(self, a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, np.float64)
        self.keep.append(a)
        return a.ctypes.data


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


def _query(n, query):
    return np.arange(n, dtype=np.int64) if query is None else _c(query, np.int64)


def neighbors(box: Box, pos, lam, query=None, rf_factor=2.3, skin=0.0):
    """Brute-force neighbour sets of the query particles: (off[nq+1], idx)."""
    pos, lam = _c(pos), _c(lam)
    n = lam.shape[0]
    q = _query(n, query)
    off = np.zeros(q.shape[0] + 1, np.int64)
    L = lib()
    L.orc_neighbors(C.byref(box), n, pos, lam, rf_factor, skin, q.shape[0], q, off, None, 0)
    idx = np.zeros(max(int(off[-1]), 1), np.int64)
    rc = L.orc_neighbors(C.byref(box), n, pos, lam, rf_factor, skin, q.shape[0], q, off,
                         idx.ctypes.data, idx.shape[0])
    assert rc == 0
    return off, idx[: off[-1]]


def mls_derivs(box: Box, pos, lam, U, nbrs, query=None, gamma=5.0 / 3.0, rf_factor=2.3,
               weight_kind=0):
    """grad [8][3][nq], hess [8][6][nq], status [nq] for the query particles."""
    pos, lam, U = _c(pos), _c(lam), _c(U)
    n = lam.shape[0]
    q = _query(n, query)
    off, idx = nbrs
    nq = q.shape[0]
    grad = np.zeros((8, 3, nq))
    hess = np.zeros((8, 6, nq))
    st = np.zeros(nq, np.int32)
    P = _P(gamma, rf_factor, weight_kind)
    lib().orc_mls_derivs(C.byref(box), n, pos, lam, U, C.byref(P.p), nq, q, _c(off, np.int64),
                         _c(idx, np.int64) if len(idx) else np.zeros(1, np.int64), grad,
                         hess.ctypes.data, st)
    return grad, hess, st


def mhd_rhs(box: Box, pos, lam, U, nbrs, query=None, gamma=5.0 / 3.0, rf_factor=2.3,
            weight_kind=0, zeta=None, eta=None, laws=(0.0, 0.0, 0.0)):
    """dU/dt [8][nq] and status [nq] for the query particles.  laws = (C_l, C_a,
    C_eta) of the bulk-viscosity and div B diffusivity laws (0 = off)."""
    pos, lam, U = _c(pos), _c(lam), _c(U)
    n = lam.shape[0]
    q = _query(n, query)
    off, idx = nbrs
    nq = q.shape[0]
    out = np.zeros((8, nq))
    st = np.zeros(nq, np.int32)
    P = _P(gamma, rf_factor, weight_kind, zeta, eta, laws=laws)
    lib().orc_mhd_rhs(C.byref(box), n, pos, lam, U, C.byref(P.p), nq, q, _c(off, np.int64),
                      _c(idx, np.int64) if len(idx) else np.zeros(1, np.int64), out, st)
    return out, st


def rhs_jvp(box: Box, pos, lam, U, dpos, dU, nbrs, query=None, gamma=5.0 / 3.0, rf_factor=2.3,
            weight_kind=0, zeta=None, eta=None, laws=(0.0, 0.0, 0.0)):
    """(dU/dt, its derivative along (dpos, dU)) for the query particles, sets frozen."""
    pos, lam, U = _c(pos), _c(lam), _c(U)
    n = lam.shape[0]
    q = _query(n, query)
    off, idx = nbrs
    nq = q.shape[0]
    out = np.zeros((8, nq))
    dout = np.zeros((8, nq))
    dpos = None if dpos is None else _c(dpos)
    dU = None if dU is None else _c(dU)
    P = _P(gamma, rf_factor, weight_kind, zeta, eta, laws=laws)
    lib().orc_rhs_jvp(C.byref(box), n, pos, lam, U,
                      None if dpos is None else dpos.ctypes.data,
                      None if dU is None else dU.ctypes.data, C.byref(P.p), nq, q,
                      _c(off, np.int64), _c(idx, np.int64) if len(idx) else np.zeros(1, np.int64),
                      out, dout)
    return out, dout


def pc_step(box: Box, pos, lam, U, dt, gamma=5.0 / 3.0, rf_factor=2.3, weight_kind=0, zeta=None,
            eta=None, frozen=None, laws=(0.0, 0.0, 0.0)):
    """One Heun step of all particles (O(n^2) brute force): returns new (pos, U).
    frozen: optional [n] mask of particles that keep x and U (fixed values)."""
    pos, lam, U = _c(pos).copy(), _c(lam), _c(U).copy()
    P = _P(gamma, rf_factor, weight_kind, zeta, eta, frozen, laws)
    nsing = lib().orc_pc_step(C.byref(box), lam.shape[0], pos, lam, U, float(dt), C.byref(P.p))
    return pos, U, nsing


def adapt_scan(box: Box, pos, lam, nbrs, query=None, rf_factor=2.3, void_factor=1.0,
               clump_factor=0.25):
    """Void and clump scan (see orc_adapt_scan) of the query particles; nbrs =
    their CSR lists at r_f (as from neighbors(..., query)).  Returns
    (void_count [nq], best [nq], cand [3][nq], clump [nq])."""
    pos, lam = _c(pos), _c(lam)
    n = lam.shape[0]
    q = _query(n, query)
    nq = q.shape[0]
    off, idx = nbrs
    vc = np.zeros(nq, np.int32)
    best = np.zeros(nq, np.int32)
    cand = np.zeros((3, nq))
    clump = np.zeros(nq, np.int32)
    lib().orc_adapt_scan(C.byref(box), n, pos, lam, float(rf_factor), float(void_factor),
                         float(clump_factor), nq, q, _c(off, np.int64),
                         _c(idx, np.int64) if len(idx) else np.zeros(1, np.int64), vc, best, cand,
                         clump)
    return vc, best, cand, clump


def adapt_apply(box: Box, pos, lam, U, nbrs, scan, grad, hess, rf_factor=2.3, void_factor=1.0):
    """Particle deletion and creation from an adaptivity scan (Sec. 2: particles
    are added in voids and deleted in clumps), readings where Paper I is not
    available:
      * a particle marked as a clump is deleted;
      * a surviving particle i with a void creates one particle at its best
        test point c_i if c_i lies inside the box on every open axis
        ([lo, lo + len)), unless a surviving neighbour j in N(i) with j < i
        creates one at a point closer than d_v = void_factor lambda_i to c_i;
      * the new particle takes lambda_i and the second-order Taylor value of
        i's fit at o = c_i - x_i: U_i + grad U_i . o + o^T (hess U_i) o / 2;
      * survivors keep their order, new particles follow in parent order;
        origin = old index for survivors, n + parent for new particles.
    nbrs: CSR lists of all particles at r_f; scan = (void_count, best, cand,
    clump) of all particles; grad [8][3][n], hess [8][6][n] (xx xy xz yy yz zz).
    Returns (pos [3][m], lam [m], U [8][m], origin [m])."""
    pos, lam, U = _c(pos), _c(lam), _c(U)
    n = lam.shape[0]
    off, idx = nbrs
    _, best, cand, clump = scan
    keep = clump == 0
    length = np.array(box.len[:3])
    lo = np.array(box.lo[:3])
    per = np.array(box.periodic[:3]) != 0

    def dist2(a, b):
        d = a - b
        for ax in range(3):
            if per[ax]:
                d[ax] = d[ax] - length[ax] * np.rint(d[ax] / length[ax])
        return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]

    inside = np.ones(n, bool)
    for ax in range(3):
        if not per[ax]:
            inside &= (cand[ax] >= lo[ax]) & (cand[ax] < lo[ax] + length[ax])
    wants = keep & (best >= 0) & inside
    create = np.zeros(n, bool)
    for i in range(n):
        if not wants[i]:
            continue
        dv = void_factor * lam[i]
        create[i] = True
        for j in idx[off[i]:off[i + 1]]:
            if j < i and wants[j] and dist2(cand[:, j], cand[:, i]) < dv * dv:
                create[i] = False
                break
    parents = np.nonzero(create)[0]
    o = cand[:, parents] - pos[:, parents]
    Unew = U[:, parents].copy()
    hi = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    for f in range(8):
        for a in range(3):
            Unew[f] += grad[f, a, parents] * o[a]
            for b in range(3):
                Unew[f] += 0.5 * hess[f, hi[(min(a, b), max(a, b))], parents] * o[a] * o[b]
    surv = np.nonzero(keep)[0]
    pos_out = np.concatenate([pos[:, surv], cand[:, parents]], axis=1)
    lam_out = np.concatenate([lam[surv], lam[parents]])
    U_out = np.concatenate([U[:, surv], Unew], axis=1)
    origin = np.concatenate([surv, n + parents]).astype(np.int64)
    return pos_out, lam_out, U_out, origin


def timestep_levels(lam, U, nbrs, gamma=5.0 / 3.0, cfl=0.1, dt_max=1.0, max_level=20):
    """Individual power-of-two time-step levels with the spatial limiter
    (see orc_timestep_levels); nbrs = CSR lists of all particles."""
    lam, U = _c(lam), _c(U)
    n = lam.shape[0]
    off, idx = nbrs
    out = np.zeros(n, np.int32)
    rc = lib().orc_timestep_levels(n, lam, U, float(gamma), float(cfl), float(dt_max),
                                   int(max_level), _c(off, np.int64),
                                   _c(idx, np.int64) if len(idx) else np.zeros(1, np.int64), out)
    if rc:
        raise ValueError("timestep_levels: invalid arguments or non-physical state")
    return out


def block_step(box: Box, pos, lam, U, levels, dt_max, max_level, anchor=None, gamma=5.0 / 3.0,
               rf_factor=2.3, weight_kind=0):
    """One synchronised step of length dt_max with individual power-of-two
    time steps (Sec. 2: every particle has its own step, Sec. 2.1: rounded
    down to powers of two and organised as GADGET's binary blocks), each
    particle advanced by the second-order predictor-corrector (read as Heun).
    Readings where the paper defers to GADGET:
      * the step is cut into 2^max_level substeps of delta = dt_max / 2^max_level;
        a particle of level L takes steps of m = 2^(max_level - L) substeps,
        all starting together at t = 0;
      * each particle keeps an anchor - its state Y0 = (x0, U0) and F0 =
        (V0, dU/dt(Y0)) at the start of its current step; at any substep time
        t its current state is the prediction Y0 + (t - t0) F0 (the
        predictor itself for a particle whose step ends at t);
      * at substep time t the particles whose step ends there are corrected:
        F = dU/dt at the current states of all particles (neighbour sets by
        brute force at the current positions),
        x = x0 + (Delta / 2)(V0 + V_current), U = U0 + (Delta / 2)(dU0 + F),
        Delta = m delta; then dU/dt at the corrected states (other particles
        still at their predictions) becomes the new anchor's derivative;
      * at t = 0 (every particle starts a step) the anchor derivative is dU/dt
        of the initial state, unless `anchor` = (x0, U0, F0) continues a
        previous step (all particles synchronised).
    With every particle on one level this is the plain Heun step.
    levels [n] int in 0..max_level.  Returns (pos, U, anchor) at t = dt_max."""
    pos, lam, U = _c(pos).copy(), _c(lam), _c(U).copy()
    levels = np.asarray(levels, np.int64)
    n = lam.shape[0]
    if levels.shape != (n,) or levels.min() < 0 or levels.max() > max_level:
        raise ValueError("levels must lie in 0..max_level")
    m = np.left_shift(1, max_level - levels)
    delta = dt_max / float(1 << max_level)

    def rhs(x, u, q):
        nb = neighbors(box, x, lam, q, rf_factor)
        out, _ = mhd_rhs(box, x, lam, u, nb, q, gamma=gamma, rf_factor=rf_factor,
                         weight_kind=weight_kind)
        return out

    if anchor is None:
        x0, u0 = pos.copy(), U.copy()
        f0 = rhs(x0, u0, np.arange(n, dtype=np.int64))
    else:
        x0, u0, f0 = (a.copy() for a in anchor)
    for k in range(1 << max_level):
        s = (k // m) * m                          # substep at which each current step began
        tau = ((k + 1) - s) * delta
        x = x0 + tau * u0[1:4]
        u = u0 + tau * f0
        A = np.flatnonzero((k + 1) % m == 0).astype(np.int64)
        if len(A):
            F = rhs(x, u, A)
            half = 0.5 * (m[A] * delta)
            xa = x0[:, A] + half * (u0[1:4, A] + u[1:4, A])
            ua = u0[:, A] + half * (f0[:, A] + F)
            x[:, A], u[:, A] = xa, ua
            x0[:, A], u0[:, A] = xa, ua
            f0[:, A] = rhs(x, u, A)
        pos, U = x, u
    return pos, U, (x0, u0, f0)


def kh_mode_amplitude(pos, U, k=4.0 * np.pi, y0=1.0, ly=4.0):
    """Magnitude of the unstable y-velocity mode of the Kelvin-Helmholtz test
    by a discrete convolution over the particles (Sec. 3.4):
      M = 2 [ (sum s_i / sum d_i)^2 + (sum c_i / sum d_i)^2 ]^(1/2),
      s_i = Vy_i sin(k x_i) e_i,  c_i = Vy_i cos(k x_i) e_i,  d_i = e_i^2,
      e_i = exp(-k |y~_i - y0|),  y~ = y below ly / 2, ly - y above it,
    the sums running over all particles.  The paper's set-up is k = 4 pi, a
    layer at y0 = 1 and its mirror image at ly - y0 = 3 (ly = 4).  Plain FP64,
    in particle order.  Returns (M, (sum s, sum c, sum d))."""
    pos, U = _c(pos), _c(U)
    x, y, vy = pos[0], pos[1], U[2]
    yt = np.where(y < 0.5 * ly, y, ly - y)
    e = np.exp(-k * np.abs(yt - y0))
    s = float(np.sum(vy * np.sin(k * x) * e))
    c = float(np.sum(vy * np.cos(k * x) * e))
    d = float(np.sum(e * e))
    return 2.0 * np.sqrt((s / d) ** 2 + (c / d) ** 2), (s, c, d)


def workload_rhs(w, query=None, **kw):
    """Convenience: brute-force neighbours plus dU/dt for a workloads.Workload."""
    box = box_of(w)
    nb = neighbors(box, w.pos, w.lam, query, kw.get("rf_factor", 2.3))
    return mhd_rhs(box, w.pos, w.lam, w.U, nb, query, gamma=w.gamma, **kw)


def available() -> bool:
    try:
        lib()
        return True
    except Exception:  # pragma: no cover - no compiler
        return False


__all__ = ["Box", "Params", "lib", "load", "using", "make_box", "box_of", "neighbors", "mls_derivs", "mhd_rhs", "adapt_scan", "adapt_apply",
           "rhs_jvp", "pc_step", "block_step", "timestep_levels", "kh_mode_amplitude",
           "workload_rhs",
           "available"]

if os.environ.get("PHB_ORACLE_EAGER"):
    lib()
