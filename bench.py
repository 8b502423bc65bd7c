#!/usr/bin/env python
"""Benchmark of the Phurbas particle right-hand-side hot path on one GB300.

One step = one second-order predictor-corrector step (Paper II Sec. 2) of the
whole particle set: cell binning, neighbour lists with a skin, two fused MLS
fit + MHD right-hand-side evaluations and the Heun update.  The metric counts
particle-RHS evaluations (two per particle per step).  Workload: the 64^3
jittered lattice with random Fourier modes (262,144 particles, constant
lambda), inputs resident in HBM; the L2 is flushed (256 MiB write) before
every timed step and the state is reset so every step does the same work.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs an independent replica (weak scaling; the path
needs no collective between replicas) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-RHS evals/s (MLS fit + MHD RHS), FP32-mixed vs FP64 on 1 GB300, err vs oracle"
UNIT = "particle-RHS/s"
WORKLOAD = "C2"
FP32_LANES = 128   # FP32 FMA lanes per SM (4 partitions x 32)
# Algorithmic work of one particle-RHS, the method's count (Sec. 2 fit + RHS),
# per neighbour inside r_f and per particle:
#   per neighbour: 80 moment FMAs + 8 fields x 19 right-hand-side FMAs = 464
#   flop, plus ~110 flop of offsets, hi/lo centring, weight and the degree 2..6
#   monomial products = 575 flop;
#   per particle: Jacobi scaling ~0.4 k, 19x19 Cholesky ~2.3 k, 8 full
#   forward + back solves ~5.8 k, right-hand side ~0.2 k = 8.7 kflop;
# about 38 kflop at 51 neighbours.
FLOP_PER_NEIGHBOUR = 575
FLOP_PER_PARTICLE = 8700
# The fused kernel's own arithmetic, printed beside it: 7 fitted fields (the
# right-hand side needs no density fit), 213 FMA per neighbour; per particle
# Cholesky 1140 FMA + 7 forward solves (171 FMA) + 7 partial back solves (36
# FMA) + ~100 flop; the corrected step of refined tiles adds ~2x this.
KERNEL_FLOP_PER_NEIGHBOUR = 2 * (80 + 7 * 19)
KERNEL_FLOP_PER_PARTICLE = 2 * (1140 + 7 * 171 + 7 * 36) + 100
# DRAM bytes (read + write) per launch of the fused fit from one-kernel ncu
# captures of the kernel as it is built now (profiles/fit_mixed_traffic.md):
# workload name -> (bytes per launch, how).  Workloads too large to capture
# under the size rule are captured on a smaller set of the same recipe and
# scaled by the particles processed.  Absent = null.
FIT_TRAFFIC = {
    "random_modes_64^3": (68648704 + 2796288, "ncu, this workload, one launch"),
    "shock_tube_1048576": (287636736 + 836296448 + 1261650432 + 78091264,
                           "ncu, this workload, one launch of each of the two fit kernels"),
    "shear_layer_8000000": (8 * (473713408 + 285548288),
                            "ncu on the 1,000,000-particle set of the same recipe with the "
                            "corrected step in the tiles (the 8M set's schedule), x 8 "
                            "(particles processed)"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--sample", type=int, default=8192, help="oracle sample size")
    ap.add_argument("--profile", choices=["none", "fit", "step"], default="none",
                    help="minimal run for an ncu capture: 'fit' = two RHS evaluations with "
                         "prebuilt lists, 'step' = two predictor-corrector steps")
    ap.add_argument("--precision", choices=["fp32_mixed", "fp64"], default="fp32_mixed",
                    help="precision of the --profile run")
    ap.add_argument("--particles", type=int, default=0,
                    help="--profile only: the workload's recipe at this particle count (a smaller "
                         "set of the same recipe for captures that must stay small; 0 = as named)")
    ap.add_argument("--tile", type=int, default=0, help="fit tile (64 or 128; 0 = library default)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="0 = one CTA per tile in cell order, 1 = one CTA per tile in descending-cost order")
    ap.add_argument("--cell-frac", type=float, default=0.0, help="cell edge / min radius (0 = default)")
    ap.add_argument("--particle-order", choices=["storage", "generator"], default="storage",
                    help="storage: arrays put once into the library's storage order (phb_reorder) "
                         "before timing; generator: the workload generator's order")
    ap.add_argument("--tune", action="store_true",
                    help="choose tile, schedule and cell size with the autotuner (overrides the three)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the timed steps eagerly instead of replaying a captured CUDA graph")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed FP64 steps (0 = skip)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing")
    ap.add_argument("--refine-schedule", choices=["auto", "queue", "tile"], default="auto",
                    help="--profile only: where the corrected step of refined tiles runs "
                         "(phb_params.refine_schedule)")
    ap.add_argument("--tc-experiment", action="store_true",
                    help="also time the tensor-core form of the fit's accumulation (mma.sync, "
                         "3xTF32) against the FP32 CUDA-core kernel on the workload")
    return ap.parse_args()


# one-line descriptions of the synthetic workloads used in the JSON line
WORKLOAD_TEXT = {
    "C1": "16^3 = 4,096 jittered-lattice particles, periodic unit box, constant lambda = 1/16, "
          "uniform background + 1e-6 fast magnetosonic wave along x",
    "C2": "64^3 = 262,144 jittered-lattice particles in the periodic unit box, constant "
          "lambda = 1/64, fields = background + 8 random Fourier modes (k <= 4, amplitude 1e-2)",
    "C3": "1,048,576 particles density-sampled (1/lambda^3) in an 8x1x1 box across a smoothed "
          "magnetised shock-tube profile along x, lambda varying 2x, 24-86 neighbours",
    "C4": "64^3 = 262,144 jittered-lattice particles with random-mode fields (adjoint workload)",
    "C5": "8,000,000 particles density-sampled in the periodic unit box around a Kelvin-Helmholtz "
          "shear layer (Vx = +-0.5, tanh width 0.05, Bx = 0.1, 1e-2 Vy seed), lambda refined 2x "
          "within 0.1 of the layer",
}


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def aggregate_max(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class Clocks:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.remove(self.path)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cfl_dt(w, cfl=0.1):
    rho = w.U[0]
    P = (w.gamma - 1.0) * w.U[7]
    b2 = (w.U[4:7] ** 2).sum(0)
    cf = np.sqrt(w.gamma * P / rho + b2 / rho)
    return cfl * float(w.lam.min()) / float(cf.max())


def kind_err(a, o, floor_frac=1e-2):
    num = np.abs(a - o).max(axis=1)
    den = np.abs(o).max(axis=1)
    den = np.maximum(den, floor_frac * den.max())
    return num / den


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def sm_max_mhz(index: int, sampled: dict | None) -> float:
    """Maximum SM clock of the GPU: from the clock samples of the timed region,
    else one nvidia-smi query, else the GB300's documented 2070 MHz."""
    if sampled and sampled.get("sm_max_mhz", 0) > 0:
        return float(sampled["sm_max_mhz"])
    try:
        out = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20).stdout.strip()
        return float(out.splitlines()[0])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return 2070.0


def fma_peak_tflops(L, dev, precision: int, sm_count: int) -> float:
    """Best of 6 launches of the library's FMA probe (precision 1 = FP32, 0 = FP64)."""
    import ctypes as C
    import torch
    blocks = sm_count * 8
    iters = 20000 if precision == 1 else 1000
    sink = torch.empty(blocks * 256, dtype=torch.float32 if precision == 1 else torch.float64,
                       device=dev)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    best = float("inf")
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if L.phb_fma_peak(precision, blocks, iters, C.c_void_p(sink.data_ptr()), st) != 0:
            raise RuntimeError("phb_fma_peak failed")
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return blocks * 256 * iters * 16 * 2 / (best * 1e-3) / 1e12


def oracle_leg(w, sample: int, seed: int = 0):
    """Time the FP64 CPU oracle (fit + RHS with brute-force neighbour lists
    precomputed, untimed) on a sample of particles; return (rate, info, q, dudt)."""
    import oracle
    rng = np.random.default_rng(seed)
    q = np.sort(rng.choice(w.n, min(sample, w.n), replace=False)).astype(np.int64)
    box = oracle.box_of(w)
    nb = oracle.neighbors(box, w.pos, w.lam, q)
    oracle.mhd_rhs(box, w.pos, w.lam, w.U, nb, q[:64], gamma=w.gamma)  # warm
    reps, t0 = 0, time.perf_counter()
    while True:
        out, st = oracle.mhd_rhs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
        reps += 1
        el = time.perf_counter() - t0
        if el > 12.0 or reps >= 20000:
            break
    rate = reps * len(q) / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    info = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{len(q)} particles of {w.name} x {reps} repetitions ({el:.1f} s): FP64 "
                      "Householder-QR fit + RHS, OpenMP over particles, brute-force neighbour "
                      "lists precomputed outside the timing"}
    return rate, info, q, out, nb


def rhs_term_scales(U, grad, hess, gamma):
    """Per field, the largest magnitude over the sample of the terms combined in
    that field's equation (ideal MHD, no zeta / eta): the scale against which
    rounding errors of the right-hand side are measured, so that a field whose
    terms cancel is measured on its terms' size.  U [8][m], grad [8][3][m],
    hess [8][6][m] (oracle values)."""
    rho, sig, B = np.abs(U[0]), np.abs(U[7]), np.abs(U[4:7])
    gV, gB = np.abs(grad[1:4]), np.abs(grad[4:7])
    divabs = gV[0, 0] + gV[1, 1] + gV[2, 2]
    J = gB.sum(axis=(0, 1))
    sc = np.zeros(8)
    sc[0] = (rho * divabs).max()
    sc[1:4] = (((gamma - 1) * np.abs(grad[7]).max(axis=0) + J * B.max(axis=0)) / rho).max()
    for a in range(3):
        sc[4 + a] = ((B * gV[a]).sum(axis=0) + B[a] * divabs).max()
    sc[7] = (gamma * sig * divabs).max()
    return sc


def deriv_err(a, o, floor_frac=1e-2):
    """Per field: max over sample and components of |a - o| over the field's
    largest |o| (floored at floor_frac of the largest field's), a, o [8][k][m]."""
    num = np.abs(a - o).max(axis=(1, 2))
    den = np.abs(o).max(axis=(1, 2))
    den = np.maximum(den, floor_frac * den.max())
    return num / np.where(den > 0, den, 1.0)


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import workloads
    w = workloads.config(args.workload)
    import oracle
    rng = np.random.default_rng(1)
    q = np.sort(rng.choice(w.n, min(args.sample, w.n), replace=False)).astype(np.int64)
    box = oracle.box_of(w)
    nb = oracle.neighbors(box, w.pos, w.lam, q)
    for _ in range(args.warmup):
        oracle.mhd_rhs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.mhd_rhs(box, w.pos, w.lam, w.U, nb, q, gamma=w.gamma)
    el = time.perf_counter() - t0
    rate = args.steps * len(q) / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{w.name}: {WORKLOAD_TEXT.get(args.workload, w.name)}",
                       "particles": w.n, "sample_per_step": int(len(q))},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": f"{len(q)} particles per step, FP64 QR fit + RHS, "
                                       "neighbour lists precomputed"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile(args):
    """Few launches on the benchmark workload, for ncu (no timing, no oracle)."""
    import torch
    import workloads
    import paper_1110_0836_gb300 as phb
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    phb.build()
    if args.particles > 0:
        recipe = {"C3": workloads.shock_tube, "C5": workloads.shear_layer}
        if args.workload not in recipe:
            raise SystemExit("--particles applies to the density-sampled workloads C3 and C5")
        w = recipe[args.workload](args.particles)
    else:
        w = workloads.config(args.workload)
    dt = cfl_dt(w)
    vmax = float(np.sqrt((w.U[1:4] ** 2).sum(0)).max())
    skin = max(4.0 * dt * vmax, 0.02 * 2.3 * float(w.lam.min()))
    pos, lam, U = phb.tensors_of(w, dev)
    prm = phb.Params(gamma=w.gamma, precision=args.precision, refine_schedule=args.refine_schedule)
    shape = {"tile": args.tile, "schedule": args.schedule, "cell_frac": args.cell_frac}
    if args.profile == "fit":
        plan = phb.Plan.for_workload(w, device=dev, **shape)
        phb.build_neighbors(plan, pos, lam)
        if args.particle_order == "storage":
            phb.reorder(plan, pos, lam, U)
        out = torch.empty((8, w.n), dtype=torch.float64, device=dev)
        for _ in range(2):
            if args.tc_experiment:
                phb.fit_tc_experiment(plan, phb.Params(gamma=w.gamma, refine="off"), pos, lam, U,
                                      out=out)
            else:
                phb.mhd_rhs(plan, prm, pos, lam, U, out=out)
    else:
        plan = phb.Plan.for_workload(w, skin=skin, device=dev, **shape)
        phb.build_neighbors(plan, pos, lam)
        if args.particle_order == "storage":
            phb.reorder(plan, pos, lam, U)
        for _ in range(2):
            phb.pc_step(plan, prm, pos, lam, U, dt)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "status": plan.read_status(), "n": w.n}))


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import ctypes as C
    import workloads
    import paper_1110_0836_gb300 as phb
    from paper_1110_0836_gb300 import _lib
    phb.build()
    L = _lib.lib()

    w = workloads.config(args.workload)
    n = w.n
    dt = cfl_dt(w)
    vmax = float(np.sqrt((w.U[1:4] ** 2).sum(0)).max())
    rf_min = 2.3 * float(w.lam.min())
    skin = max(4.0 * dt * vmax, 0.02 * rf_min)
    pos0, lam, U0 = phb.tensors_of(w, dev)
    mixed = phb.Params(gamma=w.gamma, precision="fp32_mixed")
    fp64 = phb.Params(gamma=w.gamma, precision="fp64")

    # exact neighbour count inside r_f (for the algorithmic flop count)
    plan0 = phb.Plan.for_workload(w, device=dev)
    phb.build_neighbors(plan0, pos0, lam)
    nbr_inside = plan0.neighbor_total()
    if args.particle_order == "storage":
        # the particle arrays in the library's storage order (Hilbert-ordered
        # cells), as a tree code keeps its particles; once, before any timing
        perm = phb.reorder(plan0, pos0, lam, U0).cpu().numpy().astype(np.int64)
        w.pos = np.ascontiguousarray(w.pos[:, perm])
        w.lam = np.ascontiguousarray(w.lam[perm])
        w.U = np.ascontiguousarray(w.U[:, perm])
    del plan0
    pos, U = pos0.clone(), U0.clone()

    shape = {"tile": args.tile, "schedule": args.schedule, "cell_frac": args.cell_frac}
    tuned = None
    if args.tune:
        from paper_1110_0836_gb300.tune import autotune
        tuned = autotune(w, mixed, skin=skin, device=dev)
        shape = {k: tuned[k] for k in ("tile", "schedule", "cell_frac")}
    plan = phb.Plan.for_workload(w, skin=skin, device=dev, **shape)
    phb.build_neighbors(plan, pos0, lam)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def reset():
        pos.copy_(pos0)
        U.copy_(U0)
        flush.zero_()

    plan.reset_status()
    for _ in range(args.warmup):
        reset()
        phb.pc_step(plan, mixed, pos, lam, U, dt)
    torch.cuda.synchronize()
    status = plan.read_status()
    if status & ~_lib.FLAG_FIT_SINGULAR:
        raise RuntimeError(f"warm-up status word {status:#x}")

    graph = None
    if not args.no_graph:
        reset()
        torch.cuda.synchronize()
        launches0 = int(L.phb_launch_count())
        graph = phb.StepGraph(plan, mixed, pos, lam, U, dt)
        torch.cuda.synchronize()
        per_step_launches = int(L.phb_launch_count()) - launches0

    def step():
        if graph is not None:
            graph.replay()
        else:
            phb.pc_step(plan, mixed, pos, lam, U, dt)

    # ---------------- timed region (FP32-mixed)
    # Graph replays cannot carry the library's per-launch event trace, so with a
    # graph the fused-fit launches are timed on an eager pass over the same
    # steps right after the timed region (same kernels, same inputs).
    cap = 8 * args.steps + 16
    tr_ms = (C.c_float * cap)()
    tr_id = (C.c_int32 * cap)()
    ms = []
    if graph is None:
        L.phb_trace_start(cap)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = int(L.phb_launch_count())
    with Clocks(local) as clk:
        for _ in range(args.steps):
            reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    if graph is not None:
        launches = per_step_launches * args.steps
        eager_ms = []
        L.phb_trace_start(cap)
        for _ in range(args.steps):
            reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            phb.pc_step(plan, mixed, pos, lam, U, dt)
            e1.record()
            e1.synchronize()
            eager_ms.append(e0.elapsed_time(e1))
    else:
        launches = int(L.phb_launch_count()) - launches0
        eager_ms = ms
    ntr = L.phb_trace_stop(tr_ms, tr_id, cap)
    fit_ms = [tr_ms[k] for k in range(max(ntr, 0)) if tr_id[k] == 1]
    refine_ms = [tr_ms[k] for k in range(max(ntr, 0)) if tr_id[k] == 8]
    search_ms = [tr_ms[k] for k in range(max(ntr, 0)) if tr_id[k] == 4]
    compact_ms = [tr_ms[k] for k in range(max(ntr, 0)) if tr_id[k] == 5]
    clocks = clk.summary()
    status = plan.read_status()
    if status & ~_lib.FLAG_FIT_SINGULAR:
        raise RuntimeError(f"timed-region status word {status:#x} ({_lib.status_string(L.phb_check(status))})")
    step_ms = float(np.mean(ms))
    step_ms_max = aggregate_max(step_ms, world, dev)
    value = world * 2 * n / (step_ms_max * 1e-3)

    # the fit is two kernels: the fused fit and the corrected step of the fits
    # of refined tiles (an empty queue on a lattice)
    mixed_avg = float(np.mean(fit_ms)) if fit_ms else float("nan")
    refine_avg = float(np.sum(refine_ms)) / len(fit_ms) if (refine_ms and fit_ms) else 0.0
    fit_avg = mixed_avg + refine_avg
    sm_count = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    mhz = sm_max_mhz(local, clocks)
    flops = FLOP_PER_NEIGHBOUR * nbr_inside + FLOP_PER_PARTICLE * n
    kflops = KERNEL_FLOP_PER_NEIGHBOUR * nbr_inside + KERNEL_FLOP_PER_PARTICLE * n
    peak = sm_count * FP32_LANES * 2 * mhz * 1e6 / 1e12
    achieved = flops / (fit_avg * 1e-3) / 1e12
    kname = "k_fit_mixed"
    # the captured traffic is of the default shape: 128-particle tiles in cell order
    tr = FIT_TRAFFIC.get(w.name) if (int(plan.c.schedule) == 0 and int(plan.c.tile) == 128) else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None if tr is None else tr[0],
                "traffic_unit": "DRAM bytes read + written per launch (ncu, profiles/)",
                "traffic_how": None if tr is None else tr[1],
                "kernel": f"{kname}<kRHS, {int(plan.c.tile)}> + k_fit_refine<kRHS, {int(plan.c.tile)}> "
                          "(fused FP32 MLS fit + MHD RHS, then the corrected step of the fits of "
                          "refined tiles)",
                "launch_ms": fit_avg, "launches": len(fit_ms),
                "launch_ms_parts": {kname: mixed_avg, "k_fit_refine": refine_avg},
                "timed_on": "eager pass over the timed steps (CUDA events on the launching stream)"
                            if graph is not None else "the timed steps (CUDA events on the launching stream)",
                "algorithmic_flop_per_launch": flops,
                "flop_count": f"{FLOP_PER_NEIGHBOUR} flop per neighbour inside r_f + "
                              f"{FLOP_PER_PARTICLE} per particle (the method's count)",
                "kernel_flop_per_launch": kflops,
                "kernel_count_achieved": kflops / (fit_avg * 1e-3) / 1e12,
                "peak_basis": f"{sm_count} SMs x {FP32_LANES} FP32 lanes x 2 flop x {mhz:.0f} MHz "
                              "(SM count from the device, max SM clock from nvidia-smi)"}
    del graph

    # ---------------- FP64 path, same step (fewer steps: ~25x slower)
    value64 = ms64 = None
    if args.fp64_steps > 0:
        t64 = []
        for _ in range(args.fp64_steps):
            reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            phb.pc_step(plan, fp64, pos, lam, U, dt)
            e1.record()
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        ms64 = float(np.mean(t64))
        value64 = 2 * n / (ms64 * 1e-3)

    # ---------------- single RHS evaluation (lists prebuilt) in both precisions
    def rhs_ms(params, reps):
        out = torch.empty((8, n), dtype=torch.float64, device=dev)
        phb.mhd_rhs(plan, params, pos0, lam, U0, out=out)
        t = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            phb.mhd_rhs(plan, params, pos0, lam, U0, out=out)
            e1.record()
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        return float(np.mean(t)), out

    phb.build_neighbors(plan, pos0, lam)
    rhs32_ms, d32 = rhs_ms(mixed, 10)
    rhs64_ms, d64 = rhs_ms(fp64, 2 if n <= 2_000_000 else 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    phb.build_neighbors(plan, pos0, lam, check_capacity=False)
    e1.record()
    e1.synchronize()
    build_ms = e0.elapsed_time(e1)

    # ---------------- tensor-core experiment: the accumulation as per-particle
    # Gram matrices on mma.sync (3xTF32), against the CUDA-core kernel with
    # the corrected step off (the experiment has none)
    tc = None
    if args.tc_experiment:
        cc_prm = phb.Params(gamma=w.gamma, precision="fp32_mixed", refine="off")
        cc_out = torch.empty((8, n), dtype=torch.float64, device=dev)
        phb.mhd_rhs(plan, cc_prm, pos0, lam, U0, out=cc_out)
        tc_out, gram = phb.fit_tc_experiment(plan, cc_prm, pos0, lam, U0)
        reps = 10
        capn = 8 * reps + 8
        tms, tid = (C.c_float * capn)(), (C.c_int32 * capn)()
        L.phb_trace_start(capn)
        for _ in range(reps):
            flush.zero_()
            phb.mhd_rhs(plan, cc_prm, pos0, lam, U0, out=cc_out)
            flush.zero_()
            phb.fit_tc_experiment(plan, cc_prm, pos0, lam, U0, gram=gram, out=tc_out)
        ntc = L.phb_trace_stop(tms, tid, capn)
        by = {k: [tms[i] for i in range(max(ntc, 0)) if tid[i] == k] for k in (1, 6, 7)}
        diff = (tc_out - cc_out).abs().amax(dim=1) / cc_out.abs().amax(dim=1).clamp_min(1e-300)
        tc = {"cuda_core_fit_ms": float(np.mean(by[1])) if by[1] else None,
              "tensor_gram_ms": float(np.mean(by[6])) if by[6] else None,
              "solve_from_gram_ms": float(np.mean(by[7])) if by[7] else None,
              "max_rel_diff_vs_cuda_core": float(diff.max().item()),
              "how": "mma.sync m16n8k8 TF32, operands split hi + lo, 3 products per tile, "
                     "5 output tiles (lower triangle), one warp per particle in turn; "
                     "events around each launch, L2 flushed before each call"}
        del gram, tc_out, cc_out

    # ---------------- adjoint (FP64 reverse mode, factorisations recomputed)
    adjoint = None
    if not args.no_adjoint:
        gb = torch.as_tensor(workloads.loss_weights(n), device=dev)
        Ub = torch.empty((8, n), dtype=torch.float64, device=dev)
        xb = torch.empty((3, n), dtype=torch.float64, device=dev)
        phb.rhs_adjoint(plan, fp64, pos0, lam, U0, gb, Ub, xb)
        ta = []
        for _ in range(2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            phb.rhs_adjoint(plan, fp64, pos0, lam, U0, gb, Ub, xb)
            e1.record()
            e1.synchronize()
            ta.append(e0.elapsed_time(e1))
        adj_ms = float(np.mean(ta))

        def timed(fn, reps=2):
            t = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                r = fn()
                e1.record()
                e1.synchronize()
                t.append(e0.elapsed_time(e1))
            return float(np.mean(t)), r

        rec_ms, rec = timed(lambda: phb.adjoint_record(plan, fp64, pos0, lam, U0))
        Ub2 = torch.empty_like(Ub)
        xb2 = torch.empty_like(xb)
        st_ms, _ = timed(lambda: phb.rhs_adjoint_stored(plan, fp64, pos0, lam, U0, gb, rec, Ub2, xb2))
        b_adj, e_adj = _lib.workspace_part(plan.c, _lib.PART_ADJOINT)
        ws_adj = e_adj - b_adj                               # adjoint part of the workspace
        adjoint = {"ms": adj_ms, "value": n / (adj_ms * 1e-3), "unit": "particle-gradients/s",
                   "precision": "fp64", "factorisations": "recomputed",
                   "stored": {"record_ms": rec_ms, "adjoint_ms": st_ms,
                              "record_bytes": int(rec.numel() * 8),
                              "bit_identical": bool(torch.equal(Ub, Ub2) and torch.equal(xb, xb2))},
                   "adjoint_workspace_bytes": ws_adj}
        del gb, Ub, xb, Ub2, xb2, rec

    # ---------------- particle adaptivity pass (outside the step: scan, FP32-mixed
    # fit derivatives, deletion and creation), with the step's lists
    def timed_once(fn, reps=3):
        t = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        return float(np.median(t)), r

    scan_ms, scan = timed_once(lambda: phb.adapt_scan(plan, pos0, lam))
    gder, hder, _ = phb.mls_derivs(plan, mixed, pos0, lam, U0)
    apply_ms, applied = timed_once(lambda: phb.adapt_apply(plan, pos0, lam, U0, scan, gder, hder))
    adapt = {"scan_ms": scan_ms, "apply_ms": apply_ms,
             "scan_value": n / (scan_ms * 1e-3), "unit": "particles/s",
             "particles_with_void": int((scan[0] > 0).sum()), "clump_marks": int(scan[3].sum()),
             "created": int((applied[3] >= n).sum()), "after": int(applied[3].numel()),
             "readings": "9^3 test grid, d_v = lambda, clumps closer than lambda/4"}
    del scan, gder, hder, applied

    # ---------------- end to end through the API with host buffers: phb_pc_step_host
    # uploads pos and lambda, then U on a side stream while the lists are built,
    # steps, and downloads the new pos and U (all inside the timed region)
    hpos = pos0.cpu().pin_memory()
    hlam = lam.cpu().pin_memory()
    hU = U0.cpu().pin_memory()
    opos = torch.empty_like(hpos).pin_memory()
    oU = torch.empty_like(hU).pin_memory()
    e2e_graph = None
    if not args.no_graph:
        e2e_graph = phb.HostStepGraph(plan, mixed, hpos, hlam, hU, dt, opos, oU)
    k_e2e = max(3, min(args.steps, 10))
    te = []
    for _ in range(k_e2e):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if e2e_graph is not None:
            e2e_graph.replay()
        else:
            phb.pc_step_host(plan, mixed, hpos, hlam, hU, dt, opos, oU)
        torch.cuda.synchronize()
        te.append(time.perf_counter() - t0)
    status = plan.read_status()
    if status & ~_lib.FLAG_FIT_SINGULAR:
        raise RuntimeError(f"end-to-end status word {status:#x}")
    del e2e_graph
    e2e_s = aggregate_max(float(np.mean(te)), world, dev)
    e2e = {"value": world * 2 * n / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(hpos.numel() + hlam.numel() + hU.numel()) * 8,
           "d2h_bytes_per_step": int(opos.numel() + oU.numel()) * 8,
           "path": "phb_pc_step_host on pinned host arrays: pos and lambda uploaded, U uploaded "
                   "on a side stream during the neighbour build, the predictor-corrector step, "
                   "the new pos downloaded beside the second right-hand side and the new U "
                   "written to the host by the corrector's fit (the rest after the step) "
                   "(HostStepGraph replay, or the eager call with --no-graph); host wall clock "
                   "around each step with a synchronize on both sides"}

    # ---------------- measured FMA peaks (project probe) and the FP64 path's roofline
    p32 = fma_peak_tflops(L, dev, 1, sm_count)
    p64 = fma_peak_tflops(L, dev, 0, sm_count)
    roofline["measured_fma_peak"] = p32
    roofline["frac_of_measured_fma"] = achieved / p32
    ach64 = flops / (rhs64_ms * 1e-3) / 1e12
    roofline_fp64 = {"bound": "alu", "achieved": ach64, "peak": 1.25, "unit": "TFLOP/s",
                     "frac": ach64 / 1.25, "frac_of_measured_fma": ach64 / p64,
                     "kernel": "k_fit_fp64<kRHS> (fused FP64 MLS fit + MHD RHS), whole RHS call",
                     "peak_basis": "nominal GB300 FP64 rate"}
    measured = {"fp32_fma_tflops": p32, "fp64_fma_tflops": p64,
                "how": f"phb_fma_peak: {sm_count * 8} CTAs x 256 threads x 16 independent FMA "
                       "chains, best of 6"}

    # ---------------- CPU oracle and accuracy (rank 0, one GPU)
    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_oracle:
        rate, cpu, q, o, nbq = oracle_leg(w, args.sample)
        import oracle
        go, ho, _ = oracle.mls_derivs(oracle.box_of(w), w.pos, w.lam, w.U, nbq, q, gamma=w.gamma)
        sc = rhs_term_scales(w.U[:, q], go, ho, w.gamma)
        err = {"metric": "time derivatives: per field max_i|a-o| over the field's term scale "
                         "(largest magnitude of the terms of its equation); 'rhs_by_value': "
                         "per field max_i|a-o| / max_i|o| (floor 1e-2 of the largest field's); "
                         "derivatives: per field and kind max_i|a-o| / max_i|o| (same floor); "
                         "on the oracle sample",
               "sample": int(len(q))}
        for name, prm_, d in (("fp32_mixed", mixed, d32), ("fp64", fp64, d64)):
            dq = d.cpu().numpy()[:, q]
            e_rhs = np.abs(dq - o).max(axis=1) / np.where(sc > 0, sc, 1.0)
            e_val = deriv_err(dq[:, None, :], o[:, None, :])
            gg, hh, _ = phb.mls_derivs(plan, prm_, pos0, lam, U0)
            e_g = deriv_err(gg.cpu().numpy()[:, :, q], go)
            e_h = deriv_err(hh.cpu().numpy()[:, :, q], ho)
            err[name] = float(e_rhs.max())
            err[name + "_rhs_by_value"] = float(e_val.max())
            err[name + "_detail"] = {"rhs": e_rhs.tolist(), "rhs_by_value": e_val.tolist(),
                                     "grad": e_g.tolist(),
                                     "hess": e_h.tolist(),
                                     "derivs_max": float(max(e_g.max(), e_h.max()))}

    fst = torch.empty(n, dtype=torch.int32, device=dev)
    phb.build_neighbors(plan, pos0, lam)
    phb.mhd_rhs(plan, mixed, pos0, lam, U0, fit_status=fst)
    routed = float((fst == 2).float().mean().item())
    tile_stats = plan.stats()

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms_max, "ms_per_step_median": float(np.median(ms)),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 storage, FP32 fit, FP64 routing)",
        "data": "synthetic",
        "config": {"workload": f"{w.name}: {WORKLOAD_TEXT.get(args.workload, w.name)}",
                   "particles": n,
                   "step": "one predictor-corrector step: binning + neighbour lists (skin) + 2 fused "
                           "FP32-mixed fit/RHS evaluations + Heun update; 2 particle-RHS per particle",
                   "launch": "CUDA graph replay of the captured step" if not args.no_graph else "eager",
                   "tile": int(plan.c.tile), "schedule": int(plan.c.schedule),
                   "cell_frac": float(plan.c.cell_frac), "autotuned": tuned is not None,
                   "dt": dt, "skin": skin, "neighbours_per_particle": nbr_inside / n,
                   "particle_order": "library storage order (phb_reorder once before timing; every "
                                     "step still bins, sorts and searches)"
                                     if args.particle_order == "storage" else "workload generator order",
                   "l2": "flushed (256 MiB write) before every timed step; state reset per step",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "roofline_fp64": roofline_fp64,
        "measured_alu_peaks": measured,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "steps_per_s": 1e3 / step_ms_max,
        "eager_ms_per_step": float(np.mean(eager_ms)),
        "fp64": None if value64 is None else
                {"value": value64, "unit": UNIT, "ms_per_step": ms64,
                 "speedup_fp32_mixed_over_fp64": value / value64},
        "rhs_only": {"fp32_mixed_ms": rhs32_ms, "fp64_ms": rhs64_ms,
                     "fp32_mixed_value": n / (rhs32_ms * 1e-3), "fp64_value": n / (rhs64_ms * 1e-3),
                     "neighbour_build_ms": build_ms,
                     "search_ms_in_step": float(np.mean(search_ms)) if search_ms else None,
                     "compaction_ms_in_step": float(np.mean(compact_ms)) if compact_ms else None},
        "adjoint": adjoint,
        "tc_experiment": tc,
        "adaptivity": adapt,
        "err_vs_oracle": err,
        "routed_to_fp64": routed,
        "tiles": tile_stats,
        "autotune": None if tuned is None else {k: tuned[k] for k in ("table", "ms")},
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile != "none":
        run_profile(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
