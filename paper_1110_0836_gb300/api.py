"""Torch-facing wrappers of the C ABI (include/phurbas.h).

PyTorch provides device memory and the current CUDA stream; every step of the
computation runs in libphurbas.  Arrays are float64 CUDA tensors in
structure-of-arrays layout: pos [3, n], lam [n], U [8, n] with fields
(rho, Vx, Vy, Vz, Bx, By, Bz, sigma).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import PHB_FP32_MIXED, PHB_FP64, PhbError, check

FIELDS = ("rho", "Vx", "Vy", "Vz", "Bx", "By", "Bz", "sigma")


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, shape, name: str, dtype=torch.float64) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name}: expected contiguous {dtype} {tuple(shape)}, got {t.dtype} "
                         f"{tuple(t.shape)} (contiguous={t.is_contiguous()})")
    return t


@dataclass
class Params:
    """Method parameters (phb_params)."""
    gamma: float = 5.0 / 3.0
    precision: str = "fp32_mixed"     # or "fp64"
    weight_kind: int = 0              # 0: (1 - s^2)^2, 1: unweighted
    cond_threshold: float = 3e4       # FP32-mixed: route fits above this conditioning estimate to FP64
    zeta: torch.Tensor | None = None  # bulk viscosity [n] (caller order) or None
    eta: torch.Tensor | None = None   # div B diffusivity [n] or None
    frozen: torch.Tensor | None = None  # pc_step: bool/uint8 [n], nonzero = keep x and U
    # coefficient laws added to zeta / eta (0 = off): zeta += c_zeta_l lambda c +
    # c_zeta_a lambda^2 max(0, -div V), eta += c_eta lambda c, c the fast-speed bound
    c_zeta_l: float = 0.0
    c_zeta_a: float = 0.0
    c_eta: float = 0.0
    # FP32-mixed: one corrected semi-normal-equations step per tile: "auto"
    # (tiles with a fit whose conditioning estimate exceeds refine_kappa),
    # "on" (every tile) or "off"; refine_schedule: where it runs, "auto" (by
    # the set's size), "queue" (a second kernel) or "tile" (inside the tile)
    refine: str = "auto"
    refine_kappa: float = 500.0
    refine_schedule: str = "auto"

    def c(self) -> _lib.Params:
        p = _lib.Params()
        p.gamma = float(self.gamma)
        p.weight_kind = int(self.weight_kind)
        p.precision = PHB_FP64 if self.precision == "fp64" else PHB_FP32_MIXED
        if self.precision not in ("fp64", "fp32_mixed"):
            raise ValueError(f"precision must be 'fp64' or 'fp32_mixed', not {self.precision!r}")
        p.cond_threshold = float(self.cond_threshold)
        p.zeta = None if self.zeta is None else self.zeta.data_ptr()
        p.eta = None if self.eta is None else self.eta.data_ptr()
        if self.frozen is not None and (self.frozen.dtype not in (torch.bool, torch.uint8)
                                        or not self.frozen.is_contiguous()):
            raise ValueError("frozen must be a contiguous bool or uint8 tensor")
        p.frozen = None if self.frozen is None else self.frozen.data_ptr()
        p.c_zeta_l, p.c_zeta_a, p.c_eta = float(self.c_zeta_l), float(self.c_zeta_a), float(self.c_eta)
        modes = {"auto": 0, "on": 1, "off": -1}
        if self.refine not in modes:
            raise ValueError(f"refine must be 'auto', 'on' or 'off', not {self.refine!r}")
        p.refine = modes[self.refine]
        p.refine_kappa = float(self.refine_kappa)
        schedules = {"auto": 0, "queue": 1, "tile": 2}
        if self.refine_schedule not in schedules:
            raise ValueError(f"refine_schedule must be 'auto', 'queue' or 'tile', not "
                             f"{self.refine_schedule!r}")
        p.refine_schedule = schedules[self.refine_schedule]
        return p


class Plan:
    """A phb_plan plus its device workspace and status word."""

    def __init__(self, box_lo, box_len, periodic, n: int, lambda_min: float, lambda_max: float,
                 rf_factor: float = 2.3, skin: float = 0.0, nbr_capacity: int | None = None,
                 cell_frac: float = 0.0, tile: int = 0, stage_cap: int = 0, schedule: int = 0,
                 ell_width: int = 0, device="cuda"):
        self.device = torch.device(device)
        self.args = dict(box_lo=tuple(map(float, box_lo)), box_len=tuple(map(float, box_len)),
                         periodic=tuple(int(bool(p)) for p in periodic), n=int(n),
                         lambda_min=float(lambda_min), lambda_max=float(lambda_max),
                         rf_factor=float(rf_factor), skin=float(skin), cell_frac=float(cell_frac),
                         tile=int(tile), stage_cap=int(stage_cap), schedule=int(schedule),
                         ell_width=int(ell_width))
        if nbr_capacity is None:
            # ~51 neighbours at r_f = 2.3 lambda and uniform density; margin for
            # density contrast and the skin shell
            grow = ((rf_factor * lambda_min + skin) / (rf_factor * lambda_min)) ** 3
            nbr_capacity = int(n * 72 * grow) + 1024
        self._init(int(nbr_capacity))
        self.status_word = torch.zeros(1, dtype=torch.int32, device=self.device)

    def _init(self, capacity: int):
        a = self.args
        p = _lib.Plan()
        for k in range(3):
            p.box.lo[k] = a["box_lo"][k]
            p.box.len[k] = a["box_len"][k]
            p.box.periodic[k] = a["periodic"][k]
        p.n = a["n"]
        p.rf_factor = a["rf_factor"]
        p.skin = a["skin"]
        p.lambda_min = a["lambda_min"]
        p.lambda_max = a["lambda_max"]
        p.nbr_capacity = capacity
        p.cell_frac = a["cell_frac"]
        p.tile = a["tile"]
        p.stage_cap = a["stage_cap"]
        p.schedule = a["schedule"]
        p.ell_width = a["ell_width"]
        check(_lib.lib().phb_plan_init(C.byref(p)), "phb_plan_init")
        self.c = p
        self.ws = torch.empty(int(p.ws_bytes), dtype=torch.uint8, device=self.device)

    @classmethod
    def for_workload(cls, w, skin: float = 0.0, nbr_capacity: int | None = None, device="cuda",
                     **kw):
        return cls(w.box_lo, w.box_len, w.periodic, w.n, float(w.lam.min()), float(w.lam.max()),
                   skin=skin, nbr_capacity=nbr_capacity, device=device, **kw)

    @property
    def n(self) -> int:
        return int(self.c.n)

    @property
    def capacity(self) -> int:
        return int(self.c.nbr_capacity)

    def reset_status(self):
        self.status_word.zero_()

    def read_status(self) -> int:
        """Synchronise and return the device status word."""
        return int(self.status_word.item())

    def raise_status(self, what: str = "", allow=(_lib.FLAG_FIT_SINGULAR,)) -> int:
        w = self.read_status()
        bad = w & ~sum(allow)
        if bad:
            raise PhbError(int(_lib.lib().phb_check(bad)), what or "device status")
        return w

    def stats(self) -> dict:
        """Diagnostic counters of the last build / fused fit (synchronises)."""
        out = (C.c_int32 * 5)()
        check(_lib.lib().phb_workspace_stats(C.byref(self.c), _ptr(self.ws), out, 5, _stream()),
              "phb_workspace_stats")
        return {"routed_to_fp64": int(out[0]), "build_fallback_tiles": int(out[1]),
                "fit_fallback_tiles": int(out[2]), "tiles": int(out[3]),
                "refined_tiles": int(out[4])}

    def neighbor_total(self) -> int:
        return int(_lib.lib().phb_neighbor_total(C.byref(self.c), _ptr(self.ws), _stream()))


def build_neighbors(plan: Plan, pos: torch.Tensor, lam: torch.Tensor, check_capacity: bool = True):
    """Neighbour lists of all particles (phb_build_neighbors).  With
    check_capacity, synchronises and grows the plan's list capacity if needed."""
    n = plan.n
    _need(pos, (3, n), "pos")
    _need(lam, (n,), "lam")
    L = _lib.lib()
    check(L.phb_build_neighbors(C.byref(plan.c), _ptr(pos), _ptr(lam), _ptr(plan.ws),
                                plan.ws.numel(), _ptr(plan.status_word), _stream()),
          "phb_build_neighbors")
    if check_capacity:
        w = plan.read_status()
        if w & _lib.FLAG_CAPACITY:
            total = plan.neighbor_total()
            plan._init(int(total * 1.05) + 1024)
            plan.reset_status()
            check(L.phb_build_neighbors(C.byref(plan.c), _ptr(pos), _ptr(lam), _ptr(plan.ws),
                                        plan.ws.numel(), _ptr(plan.status_word), _stream()),
                  "phb_build_neighbors")
            w = plan.read_status()
        if w & ~_lib.FLAG_FIT_SINGULAR:
            raise PhbError(int(L.phb_check(w)), "phb_build_neighbors")


def adapt_scan(plan: Plan, pos, lam, void_factor: float = 1.0, clump_factor: float = 0.25):
    """Particle adaptivity scan (phb_adapt_scan) with the lists of the last build:
    returns (void_count int32 [n], best int32 [n], cand float64 [3, n], clump int32 [n])."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam")
    vc = torch.empty(n, dtype=torch.int32, device=plan.device)
    best = torch.empty(n, dtype=torch.int32, device=plan.device)
    cand = torch.empty((3, n), dtype=torch.float64, device=plan.device)
    clump = torch.empty(n, dtype=torch.int32, device=plan.device)
    check(_lib.lib().phb_adapt_scan(C.byref(plan.c), _ptr(pos), _ptr(lam), float(void_factor),
                                    float(clump_factor), _ptr(plan.ws), plan.ws.numel(), _ptr(vc),
                                    _ptr(best), _ptr(cand), _ptr(clump), _ptr(plan.status_word),
                                    _stream()), "phb_adapt_scan")
    return vc, best, cand, clump


def adapt_apply(plan: Plan, pos, lam, U, scan, grad, hess, void_factor: float = 1.0,
                capacity: int | None = None):
    """Delete clump-marked particles and create one per void (phb_adapt_apply);
    returns (pos [3, m], lam [m], U [8, m], origin int64 [m]) with origin = old
    index for survivors and n + parent for new particles.  Synchronises to read m."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    _need(grad, (8, 3, n), "grad"), _need(hess, (8, 6, n), "hess")
    _, best, cand, clump = scan
    cap = 2 * n if capacity is None else int(capacity)
    dev = plan.device
    po = torch.empty((3, cap), dtype=torch.float64, device=dev)
    lo = torch.empty(cap, dtype=torch.float64, device=dev)
    Uo = torch.empty((8, cap), dtype=torch.float64, device=dev)
    org = torch.empty(cap, dtype=torch.int64, device=dev)
    m = torch.zeros(1, dtype=torch.int64, device=dev)
    check(_lib.lib().phb_adapt_apply(C.byref(plan.c), _ptr(pos), _ptr(lam), _ptr(U), _ptr(best),
                                     _ptr(cand), _ptr(clump), _ptr(grad), _ptr(hess),
                                     float(void_factor), cap, _ptr(po), _ptr(lo), _ptr(Uo), _ptr(org),
                                     _ptr(m), _ptr(plan.ws), plan.ws.numel(), _ptr(plan.status_word),
                                     _stream()), "phb_adapt_apply")
    k = int(m.item())
    if k > cap:
        raise PhbError(int(_lib.PHB_ERR_CAPACITY), f"phb_adapt_apply: {k} particles > capacity {cap}")
    return po[:, :k].contiguous(), lo[:k].clone(), Uo[:, :k].contiguous(), org[:k].clone()


def adapt(plan: Plan, params: Params, pos, lam, U, void_factor: float = 1.0,
          clump_factor: float = 0.25):
    """One adaptivity pass with the lists of the last build: scan, fit
    derivatives, deletion and creation.  Returns the new (pos, lam, U, origin)."""
    scan = adapt_scan(plan, pos, lam, void_factor, clump_factor)
    g, h, _ = mls_derivs(plan, params, pos, lam, U)
    return adapt_apply(plan, pos, lam, U, scan, g, h, void_factor)


def reorder(plan: Plan, pos, lam, U):
    """Permute pos, lam and U in place into the storage order of the last build
    (phb_reorder); returns the int32 [n] tensor of old indices, for the caller's
    other per-particle arrays (x_new = x_old[perm])."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    perm = torch.empty(n, dtype=torch.int32, device=plan.device)
    check(_lib.lib().phb_reorder(C.byref(plan.c), _ptr(pos), _ptr(lam), _ptr(U), _ptr(perm),
                                 _ptr(plan.ws), plan.ws.numel(), _ptr(plan.status_word), _stream()),
          "phb_reorder")
    return perm


def export_neighbors(plan: Plan):
    """(off int64 [n+1], idx int32 [total]) in caller numbering, ascending per list."""
    total = plan.neighbor_total()
    off = torch.empty(plan.n + 1, dtype=torch.int64, device=plan.device)
    idx = torch.empty(max(total, 1), dtype=torch.int32, device=plan.device)
    check(_lib.lib().phb_export_neighbors(C.byref(plan.c), _ptr(plan.ws), _ptr(off), _ptr(idx),
                                          idx.numel(), _stream()), "phb_export_neighbors")
    return off, idx[:total]


def mls_derivs(plan: Plan, params: Params, pos, lam, U, hess: bool = True, out=None):
    """MLS derivatives: grad [8,3,n], hess [8,6,n] (or None), fit_status [n] int32."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    if out is None:
        g = torch.empty((8, 3, n), dtype=torch.float64, device=plan.device)
        h = torch.empty((8, 6, n), dtype=torch.float64, device=plan.device) if hess else None
        st = torch.empty(n, dtype=torch.int32, device=plan.device)
    else:
        g, h, st = out
    pc = params.c()
    check(_lib.lib().phb_mls_derivs(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                    _ptr(plan.ws), plan.ws.numel(), _ptr(g), _ptr(h), _ptr(st),
                                    _ptr(plan.status_word), _stream()), "phb_mls_derivs")
    return g, h, st


def mhd_rhs(plan: Plan, params: Params, pos, lam, U, out=None, fit_status=None):
    """Lagrangian time derivatives dU/dt [8, n] (phb_mhd_rhs); returns (dudt, fit_status)."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    if out is None:
        out = torch.empty((8, n), dtype=torch.float64, device=plan.device)
    pc = params.c()
    check(_lib.lib().phb_mhd_rhs(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                 _ptr(plan.ws), plan.ws.numel(), _ptr(out), _ptr(fit_status),
                                 _ptr(plan.status_word), _stream()), "phb_mhd_rhs")
    return out, fit_status


def pc_step(plan: Plan, params: Params, pos, lam, U, dt: float):
    """One predictor-corrector step in place (phb_pc_step).  Needs plan.skin > 2 dt max|V|."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    if params.frozen is not None:
        _need(params.frozen, (n,), "frozen", params.frozen.dtype)
    pc = params.c()
    check(_lib.lib().phb_pc_step(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                 float(dt), _ptr(plan.ws), plan.ws.numel(), _ptr(plan.status_word),
                                 _stream()), "phb_pc_step")


def _need_host(t, shape, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if t.dtype != torch.float64 or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name}: expected contiguous float64 {tuple(shape)}, got {t.dtype} "
                         f"{tuple(t.shape)}")
    return t


def pc_step_host(plan: Plan, params: Params, pos, lam, U, dt: float, pos_out=None, U_out=None):
    """One predictor-corrector step on host tensors (phb_pc_step_host): pos [3, n], lam [n],
    U [8, n] on the CPU (pinned for asynchronous copies) are uploaded, stepped and the new
    pos and U written to pos_out / U_out (default: in place).  Asynchronous on the current
    stream: synchronise before reading the outputs."""
    n = plan.n
    _need_host(pos, (3, n), "pos"), _need_host(lam, (n,), "lam"), _need_host(U, (8, n), "U")
    pos_out = pos if pos_out is None else _need_host(pos_out, (3, n), "pos_out")
    U_out = U if U_out is None else _need_host(U_out, (8, n), "U_out")
    if params.frozen is not None:
        _need(params.frozen, (n,), "frozen", params.frozen.dtype)
    pc = params.c()
    check(_lib.lib().phb_pc_step_host(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                      _ptr(pos_out), _ptr(U_out), float(dt), _ptr(plan.ws),
                                      plan.ws.numel(), _ptr(plan.status_word), _stream()),
          "phb_pc_step_host")


def rhs_adjoint(plan: Plan, params: Params, pos, lam, U, gbar, Ubar=None, xbar=None):
    """dL/dU [8, n] and dL/dpos [3, n] for gbar = dL/d(dudt) (phb_rhs_adjoint), with the
    neighbour lists of the last build held fixed."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    _need(gbar, (8, n), "gbar")
    if Ubar is None:
        Ubar = torch.empty((8, n), dtype=torch.float64, device=plan.device)
    if xbar is None:
        xbar = torch.empty((3, n), dtype=torch.float64, device=plan.device)
    pc = params.c()
    check(_lib.lib().phb_rhs_adjoint(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                     _ptr(gbar), _ptr(plan.ws), plan.ws.numel(), _ptr(Ubar),
                                     _ptr(xbar), _ptr(plan.status_word), _stream()),
          "phb_rhs_adjoint")
    return Ubar, xbar


def mhd_rhs_active(plan: Plan, params: Params, pos, lam, U, active, out=None, fit_status=None):
    """dU/dt at the caller indices in `active` (int32 CUDA tensor) only
    (phb_mhd_rhs_active), with the lists of the last build.  out [8, n] is
    written at those columns; other columns are left as they are."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    if not isinstance(active, torch.Tensor) or not active.is_cuda or active.dtype != torch.int32 \
            or active.dim() != 1 or not active.is_contiguous():
        raise ValueError("active must be a contiguous 1-D int32 CUDA tensor")
    if out is None:
        out = torch.zeros((8, n), dtype=torch.float64, device=plan.device)
    _need(out, (8, n), "out")
    if fit_status is not None:
        _need(fit_status, (n,), "fit_status", torch.int32)
    pc = params.c()
    check(_lib.lib().phb_mhd_rhs_active(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                        _ptr(active), active.numel(), _ptr(plan.ws), plan.ws.numel(),
                                        _ptr(out), _ptr(fit_status), _ptr(plan.status_word),
                                        _stream()), "phb_mhd_rhs_active")
    return out


def timestep_levels(plan: Plan, params: Params, pos, lam, U, cfl: float, dt_max: float,
                    max_level: int = 20, out=None):
    """Individual power-of-two time-step levels with the spatial limiter
    (phb_timestep_levels), int32 [n] caller order, from the lists of the last
    build.  A particle of level L advances with dt_max / 2**L."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=plan.device)
    _need(out, (n,), "out", torch.int32)
    pc = params.c()
    check(_lib.lib().phb_timestep_levels(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                         float(cfl), float(dt_max), int(max_level), _ptr(plan.ws),
                                         plan.ws.numel(), _ptr(out), _ptr(plan.status_word),
                                         _stream()), "phb_timestep_levels")
    return out


def active_at(levels: torch.Tensor, substep: int, max_level: int) -> torch.Tensor:
    """Caller indices whose step ends at `substep` of the finest level
    (dt_max / 2**max_level units) in the binary block scheme: level L is
    active when substep is a multiple of 2**(max_level - L)."""
    period = torch.bitwise_left_shift(torch.ones_like(levels), max_level - levels)
    return torch.nonzero(substep % period == 0).flatten().to(torch.int32)


def adjoint_record(plan: Plan, params: Params, pos, lam, U, record=None):
    """Per-particle FP64 factorisations and coefficients for phb_rhs_adjoint_stored
    (phb_adjoint_record), with the lists of the last build.  Returns the record
    (float64 [343, n] device tensor, slot order)."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    L = _lib.lib()
    nbytes = int(L.phb_adjoint_record_bytes(C.byref(plan.c)))
    if record is None:
        record = torch.empty(nbytes // 8, dtype=torch.float64, device=plan.device)
    pc = params.c()
    check(L.phb_adjoint_record(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                               _ptr(plan.ws), plan.ws.numel(), _ptr(record),
                               record.numel() * record.element_size(), _ptr(plan.status_word),
                               _stream()), "phb_adjoint_record")
    return record


def rhs_adjoint_stored(plan: Plan, params: Params, pos, lam, U, gbar, record, Ubar=None, xbar=None):
    """rhs_adjoint starting from a record of adjoint_record (same plan, lists and inputs)."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    _need(gbar, (8, n), "gbar")
    if Ubar is None:
        Ubar = torch.empty((8, n), dtype=torch.float64, device=plan.device)
    if xbar is None:
        xbar = torch.empty((3, n), dtype=torch.float64, device=plan.device)
    pc = params.c()
    check(_lib.lib().phb_rhs_adjoint_stored(
        C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U), _ptr(gbar), _ptr(plan.ws),
        plan.ws.numel(), _ptr(record), record.numel() * record.element_size(), _ptr(Ubar),
        _ptr(xbar), _ptr(plan.status_word), _stream()), "phb_rhs_adjoint_stored")
    return Ubar, xbar


def block_step(plan: Plan, params: Params, pos, lam, U, levels, dt_max: float, max_level: int,
               anchor=None):
    """One synchronised step of dt_max with individual power-of-two steps
    (phb_block_begin when no anchor is given, then phb_block_substep for each
    of the 2^max_level substeps).  pos and U are advanced in place; returns
    the anchor ([19, n] float64) to continue with."""
    n = plan.n
    _need(pos, (3, n), "pos")
    _need(lam, (n,), "lam")
    _need(U, (8, n), "U")
    _need(levels, (n,), "levels", torch.int32)
    L = _lib.lib()
    if anchor is None:
        anchor = torch.empty((19, n), dtype=torch.float64, device=pos.device)
        pc = params.c()
        check(L.phb_block_begin(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                _ptr(anchor), _ptr(plan.ws), plan.ws.numel(),
                                _ptr(plan.status_word), _stream()), "phb_block_begin")
    else:
        _need(anchor, (19, n), "anchor")
    pc = params.c()
    for k in range(1 << int(max_level)):
        check(L.phb_block_substep(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam), _ptr(U),
                                  _ptr(anchor), _ptr(levels), k, int(max_level), float(dt_max),
                                  _ptr(plan.ws), plan.ws.numel(), _ptr(plan.status_word),
                                  _stream()), "phb_block_substep")
    return anchor


def fit_tc_experiment(plan: Plan, params: Params, pos, lam, U, gram=None, out=None):
    """Right-hand side with the fit's moments and right-hand sides formed on
    the tensor cores (phb_fit_tc_experiment, a measurement helper): returns
    (dudt [8, n], gram scratch [214, n])."""
    n = plan.n
    _need(pos, (3, n), "pos"), _need(lam, (n,), "lam"), _need(U, (8, n), "U")
    if gram is None:
        gram = torch.empty((214, n), dtype=torch.float32, device=pos.device)
    if out is None:
        out = torch.empty((8, n), dtype=torch.float64, device=pos.device)
    pc = params.c()
    check(_lib.lib().phb_fit_tc_experiment(C.byref(plan.c), C.byref(pc), _ptr(pos), _ptr(lam),
                                           _ptr(U), _ptr(plan.ws), plan.ws.numel(), _ptr(gram),
                                           gram.numel() * 4, _ptr(out), _ptr(plan.status_word),
                                           _stream()), "phb_fit_tc_experiment")
    return out, gram


def kh_mode_amplitude(plan: Plan, pos, U, k: float = 4.0 * 3.141592653589793, y0: float = 1.0,
                      ly: float = 4.0):
    """Kelvin-Helmholtz mode amplitude (phb_kh_mode_amplitude): returns a
    float64 device tensor (sum s, sum c, sum d, M)."""
    n = plan.n
    _need(pos, (3, n), "pos")
    _need(U, (8, n), "U")
    out = torch.empty(4, dtype=torch.float64, device=pos.device)
    check(_lib.lib().phb_kh_mode_amplitude(C.byref(plan.c), _ptr(pos), _ptr(U), float(k), float(y0),
                                           float(ly), _ptr(plan.ws), plan.ws.numel(), _ptr(out),
                                           _stream()), "phb_kh_mode_amplitude")
    return out


def tensors_of(w, device="cuda"):
    """(pos, lam, U) float64 CUDA tensors of a workloads.Workload."""
    dev = torch.device(device)
    return (torch.as_tensor(w.pos, device=dev).contiguous(),
            torch.as_tensor(w.lam, device=dev).contiguous(),
            torch.as_tensor(w.U, device=dev).contiguous())


def rhs(w, params: Params | None = None, skin: float = 0.0, device="cuda"):
    """Convenience: plan, neighbours and dU/dt for a workloads.Workload."""
    params = params or Params(gamma=w.gamma)
    plan = Plan.for_workload(w, skin=skin, device=device)
    pos, lam, U = tensors_of(w, device)
    build_neighbors(plan, pos, lam)
    st = torch.empty(w.n, dtype=torch.int32, device=plan.device)
    dudt, _ = mhd_rhs(plan, params, pos, lam, U, fit_status=st)
    return dudt, st, plan


class StepGraph:
    """CUDA graph of `steps` predictor-corrector steps (phb_pc_step), each with its
    neighbour rebuild, captured once and replayed on the current stream.

    The graph holds the addresses of pos, lam, U, the parameter arrays and the
    plan's workspace and the value of dt: keep those tensors alive and in place,
    and do not grow the plan (its capacity must already hold the lists; the
    status word reports FLAG_CAPACITY and FLAG_SKIN after a replay otherwise).
    """

    def __init__(self, plan: Plan, params: Params, pos, lam, U, dt: float, steps: int = 1):
        if steps < 1:
            raise ValueError("steps must be >= 1")
        self.plan, self.params, self.steps = plan, params, int(steps)
        self._keep = (pos, lam, U, params.zeta, params.eta, params.frozen, plan.ws)
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=plan.device)
        side.wait_stream(torch.cuda.current_stream(plan.device))
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                for _ in range(self.steps):
                    pc_step(plan, params, pos, lam, U, dt)
        torch.cuda.current_stream(plan.device).wait_stream(side)

    def replay(self):
        """Advance pos and U by `steps` steps in place (asynchronous)."""
        self.graph.replay()


class HostStepGraph:
    """CUDA graph of one predictor-corrector step on host tensors (phb_pc_step_host):
    the uploads of pos, lam and U (U overlapped with the neighbour build), the step and
    the downloads of the new pos and U to pos_out / U_out, captured once after one eager
    step (which also makes the library's side stream) and replayed on the current stream.
    Keep the tensors alive and in place; replay() is asynchronous: synchronise before
    reading the outputs."""

    def __init__(self, plan: Plan, params: Params, pos, lam, U, dt: float, pos_out, U_out):
        self.plan, self.params = plan, params
        self._keep = (pos, lam, U, pos_out, U_out, params.zeta, params.eta, params.frozen, plan.ws)
        pc_step_host(plan, params, pos, lam, U, dt, pos_out, U_out)
        torch.cuda.synchronize(plan.device)
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=plan.device)
        side.wait_stream(torch.cuda.current_stream(plan.device))
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                pc_step_host(plan, params, pos, lam, U, dt, pos_out, U_out)
        torch.cuda.current_stream(plan.device).wait_stream(side)

    def replay(self):
        self.graph.replay()
