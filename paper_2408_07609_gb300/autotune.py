"""Autotuner of the step kernel's launch shape.

Knobs (none changes the results, only the speed): the strip height (rti_params.tile_y),
the resident CTAs per SM of the step kernel's grid (ctas_per_sm), the schedule (one
persistent launch per chunk, or one launch per step) and, for batches, the chunk length
(steps per graph-captured launch). The tuner times short runs of each candidate on the
GPU with CUDA events, keeps the best third for a longer second round (successive
halving), and caches the choice per hierarchy shape (block sizes and nesting, precision,
options and the library build) in memory and, if asked, in a JSON file.

Beside the choice it fits the per-strip linear cost model t_step = alpha * cells + beta *
strips to the timed candidates, in the manner of the per-block model the paper fits to
its nested-grid kernel (Sec. IV-D, Eq. 5, Fig. 4: a cost per cell plus a fixed cost per
block); alpha is the marginal time per cell update, beta the fixed cost per strip.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import rti

TILE_Y = (32, 48, 64, 96, 128)
CTAS = (0, 4, 3)  # 0: as many CTAs per SM as fit (5 in binary32)
SCHEDULES = (rti.SCHED_PERSISTENT, rti.SCHED_PER_PASS)
CHUNKS = (25, 50, 100, 200)

_memo: dict = {}


def _lib_id() -> str:
    """Identity of the loaded library build (a tuned shape holds for one build only)."""
    path = os.environ.get("RTI_LIBRARY", rti.LIB)
    h = hashlib.sha1()
    with open(path, "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:12]


def shape_key(blocks, precision, **opts) -> str:
    parts = [f"p{int(precision)}"] + [f"{k}={v}" for k, v in sorted(opts.items())]
    for b in blocks:
        parts.append(f"{b['level']}:{b['parent']}:{b['nx']}x{b['ny']}@{b.get('i0', 0)},{b.get('j0', 0)}")
    parts.append(_lib_id())
    return hashlib.sha1("|".join(parts).encode()).hexdigest()[:16]


def strips(blocks, tile_y, tile_x=28) -> int:
    return sum(-(-b["nx"] // tile_x) * -(-b["ny"] // tile_y) for b in blocks)


def _time_handle(h, steps, stream):
    import torch

    h.step(2, stream)
    h.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.step(steps, stream)
    e1.record(stream)
    h.sync()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def fit_cost_model(trials, cells):
    """Least-squares fit of ms_per_step = alpha * cells + beta * strips over the trials of
    one schedule and CTA count (cells is the same for all, so alpha absorbs the constant):
    returns (alpha in ns per cell update, beta in us per strip), or None."""
    rows = [(t["strips"], t["ms_per_step"]) for t in trials]
    if len({r[0] for r in rows}) < 2:
        return None
    A = np.array([[cells, s] for s, _ in rows], float)
    y = np.array([m for _, m in rows], float)
    (a, b), *_ = np.linalg.lstsq(A, y, rcond=None)
    return {"alpha_ns_per_cell": a * 1e6, "beta_us_per_strip": b * 1e3}


def tune_handle(sc, precision=rti.FP32, steps=(10, 40), cache_path=None, tile_y=TILE_Y,
                ctas=CTAS, schedules=SCHEDULES, **opts):
    """Pick strip height, CTAs per SM and schedule for stepping scenario `sc` alone.
    Returns {"tile_y", "ctas_per_sm", "schedule", "ms_per_step", "trials", "model",
    "cached"}."""
    import torch

    key = shape_key(sc.blocks, precision, **opts)
    cache = _load(cache_path)
    if key in cache:
        return dict(cache[key], cached=True)
    stream = torch.cuda.Stream()
    cands = [(ty, c, s) for s in schedules for c in ctas for ty in tile_y]
    trials = []
    for ty, c, s in cands:
        h = rti.Handle.from_scenario(sc, precision=precision, schedule=s, tile=(0, ty),
                                     ctas_per_sm=c, **opts)
        ms = _time_handle(h, steps[0], stream)
        h.close()
        trials.append({"tile_y": ty, "ctas_per_sm": c, "schedule": s, "ms_per_step": ms,
                       "strips": strips(sc.blocks, ty)})
    keep = sorted(trials, key=lambda t: t["ms_per_step"])[:max(1, len(trials) // 3)]
    for t in keep:
        h = rti.Handle.from_scenario(sc, precision=precision, schedule=t["schedule"],
                                     tile=(0, t["tile_y"]), ctas_per_sm=t["ctas_per_sm"], **opts)
        t["ms_per_step_long"] = _time_handle(h, steps[1], stream)
        h.close()
    best = min(keep, key=lambda t: t["ms_per_step_long"])
    base = [t for t in trials if t["schedule"] == best["schedule"]
            and t["ctas_per_sm"] == best["ctas_per_sm"]]
    out = {"tile_y": best["tile_y"], "ctas_per_sm": best["ctas_per_sm"],
           "schedule": best["schedule"], "ms_per_step": best["ms_per_step_long"],
           "trials": trials, "model": fit_cost_model(base, sc.cells), "key": key}
    cache[key] = out
    _save(cache_path, cache)
    return dict(out, cached=False)


def tune_batch(scenarios, precision=rti.FP32, chunk_steps=CHUNKS, tile_y=TILE_Y, ctas=CTAS,
               cache_path=None, rounds=2):
    """Pick strip height, CTAs per SM and chunk length for stepping `scenarios` together in
    one batch (persistent schedule): each candidate times one chunk after a warm-up
    chunk. Returns {"tile_y", "ctas_per_sm", "chunk_steps", "gcups", "trials", "cached"}."""
    import torch

    blocks = [b for sc in scenarios for b in sc.blocks]
    key = shape_key(blocks, precision, batch=len(scenarios))
    cache = _load(cache_path)
    if key in cache:
        return dict(cache[key], cached=True)
    cells = sum(sc.cells for sc in scenarios)
    stream = torch.cuda.Stream()
    trials = []
    for ty in tile_y:
        hs = [rti.Handle.from_scenario(sc, precision=precision, tile=(0, ty)) for sc in scenarios]
        for c in ctas:
            for k in chunk_steps:
                b = rti.Batch(precision, rti.SCHED_PERSISTENT, k, tile_y=ty, ctas_per_sm=c)
                for h in hs:
                    b.add(h, k * (rounds + 1))
                b.step(stream)  # uploads the tables, captures the graph
                b.sync()
                best = float("inf")
                for _ in range(rounds):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    b.step(stream)
                    e1.record(stream)
                    b.sync()
                    best = min(best, e0.elapsed_time(e1))
                b.close()
                trials.append({"tile_y": ty, "ctas_per_sm": c, "chunk_steps": k,
                               "gcups": cells * k / (best / 1e3) / 1e9})
        for h in hs:
            h.close()
    top = max(trials, key=lambda t: t["gcups"])
    out = dict(top, trials=trials, key=key)
    cache[key] = out
    _save(cache_path, cache)
    return dict(out, cached=False)


def _load(path):
    """The cache of `path` (None: this process only)."""
    slot = path or ""
    if slot not in _memo and path and os.path.exists(path):
        with open(path) as f:
            _memo[slot] = json.load(f)
    return _memo.setdefault(slot, {})


def _save(path, cache):
    if path is None:
        return
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f)
    os.replace(tmp, path)
