"""Autotuner for the fused fit's launch shape.

Times the neighbour build plus one fused right-hand side for every candidate
(tile size, tile schedule, cell size) on the caller's particle set and keeps
the fastest; results are cached in a JSON file keyed by the GPU name and a
signature of the particle set and plan.  Candidates that fail to plan (for
example a tile size the library does not support) are skipped.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import torch

from .api import Params, Plan, build_neighbors, mhd_rhs, tensors_of

CANDIDATES = [
    dict(tile=128, schedule=0, cell_frac=1.0),
    dict(tile=128, schedule=1, cell_frac=1.0),
    dict(tile=64, schedule=0, cell_frac=1.0),
    dict(tile=128, schedule=0, cell_frac=0.5),
    dict(tile=128, schedule=1, cell_frac=0.5),
    dict(tile=64, schedule=0, cell_frac=0.5),
]


def cache_path() -> str:
    return os.environ.get("PHB_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "phurbas", "tune.json"))


def signature(w, skin: float, precision: str) -> str:
    h = hashlib.sha1()
    for v in (w.n, tuple(w.box_len), tuple(w.periodic), float(w.lam.min()), float(w.lam.max()),
              round(skin, 12), precision):
        h.update(repr(v).encode())
    # coarse shape of the density: histogram of lambda
    import numpy as np
    hist, _ = np.histogram(w.lam, bins=8)
    h.update(hist.tobytes())
    return h.hexdigest()[:16]


def _time_candidate(w, params: Params, skin: float, cand: dict, reps: int, device) -> float:
    plan = Plan.for_workload(w, skin=skin, device=device, **cand)
    pos, lam, U = tensors_of(w, device)
    out = torch.empty((8, w.n), dtype=torch.float64, device=plan.device)
    build_neighbors(plan, pos, lam)
    mhd_rhs(plan, params, pos, lam, U, out=out)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        build_neighbors(plan, pos, lam, check_capacity=False)
        mhd_rhs(plan, params, pos, lam, U, out=out)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    plan.raise_status("autotune")
    return best


def autotune(w, params: Params | None = None, skin: float = 0.0, reps: int = 3,
             candidates=None, use_cache: bool = True, device="cuda") -> dict:
    """Fastest plan options for workload `w`: {'tile', 'schedule', 'cell_frac', 'ms', 'table'}."""
    params = params or Params(gamma=w.gamma)
    dev = torch.device(device)
    key = f"{torch.cuda.get_device_name(dev)}|{signature(w, skin, params.precision)}"
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]
    table = []
    for cand in candidates or CANDIDATES:
        try:
            ms = _time_candidate(w, params, skin, cand, reps, dev)
        except Exception as e:  # noqa: BLE001 - a candidate the plan rejects
            table.append({**cand, "ms": None, "error": str(e)[:80]})
            continue
        table.append({**cand, "ms": ms})
    ok = [t for t in table if t["ms"] is not None]
    if not ok:
        raise RuntimeError("autotune: no candidate ran")
    best = min(ok, key=lambda t: t["ms"])
    res = {k: best[k] for k in ("tile", "schedule", "cell_frac")}
    res["ms"] = best["ms"]
    res["table"] = table
    res["when"] = time.strftime("%Y-%m-%dT%H:%M:%S")
    if use_cache:
        cache[key] = res
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".tmp{os.getpid()}"
            json.dump(cache, open(tmp, "w"), indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
    return res
