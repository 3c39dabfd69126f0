#!/usr/bin/env python3
"""Benchmark of the nested shallow-water time step on GB300.

Default run (N = 1): the 46.65 M-cell 5-level hierarchy shaped like the paper's Kochi
model (Table I; synthetic bathymetry and source), binary32, stepped by the CUDA
library through its C ABI. Prints ONE JSON line with GCUPS (cell updates per second /
1e9), the binary64 rate beside it, the projected 6-h wall times, an end-to-end number
through the public API with host buffers, the HBM roofline of the step kernel and the
FP64 CPU oracle timed on the host cores.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With --gpus N > 1 (torchrun, one rank per GPU) every rank steps its own replica of
the hierarchy (independent scenarios, no collective in the data path): weak scaling.
--impl reference times the FP64 oracle on the host cores on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIX_HOURS_STEPS = 108_000  # 6 h at dt = 0.2 s (Sec. V-A)
# Compulsory HBM bytes per cell and step of the one-sweep kernel: it reads eta^n, M^n,
# N^n, h, eta_max (state precision) and Manning n (binary32) and writes eta^{n+1},
# M^{n+1}, N^{n+1}; the rare eta_max / arrival writes are not counted.
BYTES_PER_CELL_STEP = {"f32": 5 * 4 + 4 + 3 * 4,   # 36
                       "f64": 5 * 8 + 4 + 3 * 8}   # 68
# cell-steps of FP64 oracle work per host thread the reference arm spreads over its W + K
# steps (about a minute)
REF_CELL_STEPS = 0.8e9
# DRAM bytes per cell-step that ncu measured for k_step<float> (dram__bytes_read.sum +
# dram__bytes_write.sum of one single-step launch on the 7.95 M-cell 4-level hierarchy,
# divided by its cells); scaled to a launch of the bench by cells x steps. Set to None
# whenever the kernel changes until it is captured again.
NCU_F32_DRAM_BYTES_PER_CELL_STEP = (229.106432e6 + 82.531328e6) / 7.95e6  # 39.20 B


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--schedule", type=int, default=0, help="0 persistent, 1 one launch per step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--tile", type=int, nargs=2, default=(0, 0), help="strip shape (0 0 = default)")
    ap.add_argument("--nest-feedback", choices=("ring", "full"), default="ring",
                    help="fine-to-coarse feedback on the boundary ring or every covered cell")
    ap.add_argument("--nest-flux", choices=("linear", "constant"), default="linear",
                    help="coarse-to-fine edge flux")
    ap.add_argument("--track-velocity", action="store_true",
                    help="keep the maximum water velocity in the timed runs")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-n", type=int, default=30, help="requests in the serving trace")
    ap.add_argument("--serve-scale", type=float, default=1.0 / 60.0,
                    help="time scale of the serving trace (arrivals and durations)")
    ap.add_argument("--serve-pool-gb", type=int, default=32)
    ap.add_argument("--serve-audit-every", type=int, default=10,
                    help="run every N-th request again in FP64 after the trace (0: no audit)")
    ap.add_argument("--serve-sat-n", type=int, default=12,
                    help="requests of the saturation comparison (all arrive at t = 0)")
    ap.add_argument("--serve-sat-scale", type=float, default=1.0 / 120.0,
                    help="duration scale of the saturation comparison")
    ap.add_argument("--serve-real", action="store_true",
                    help="also serve the 10-arrival smoke trace at its real durations (1-6 h)")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--accuracy-c4-steps", type=int, default=2000,
                    help="compare FP32 with FP64 on the 46.65 M-cell workload over N steps "
                         "(0: skip)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-latency", action="store_true",
                    help="skip the small configurations' time per step")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default launch shape (28 x 64 strips, all CTAs that fit, "
                         "persistent) instead of the autotuner's choice")
    ap.add_argument("--tune-cache", default=None, help="JSON file caching the tuned shapes")
    return ap.parse_args()


def dist_setup(n):
    """Rank, world size and a barrier; torchrun sets RANK/WORLD_SIZE for N > 1."""
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells, steps, ms, world):
    """GCUPS of the whole job: every rank steps its own copy of the workload, and the
    job takes as long as its slowest rank."""
    return world * cells * steps / (ms / 1e3) / 1e9


class Clocks:
    """nvidia-smi samples (SM clock, throttle reasons) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def emit(obj):
    print(json.dumps(obj), flush=True)


def workload():
    from paper_2408_07609_gb300 import scenarios

    return scenarios.config4(steps=SIX_HOURS_STEPS)


def handle_options(a):
    """Handle keywords of the run's nesting and output options."""
    return dict(nest_feedback=1 if a.nest_feedback == "full" else 0,
                nest_flux=1 if a.nest_flux == "constant" else 0,
                track_velocity=bool(a.track_velocity))


def time_device(rti, sc, precision, steps, warmup, schedule, world, tile=(0, 0), opts=None,
                ctas_per_sm=0):
    """Kernel-only rate: inputs resident in HBM, CUDA events on the launching stream."""
    import torch

    h = rti.Handle.from_scenario(sc, precision=precision, schedule=schedule, tile=tuple(tile),
                                 ctas_per_sm=ctas_per_sm, **(opts or {}))
    stream = torch.cuda.Stream()
    h.step(warmup, stream)
    h.sync()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.step(steps, stream)
    e1.record(stream)
    h.sync()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    barrier(world)
    h.close()
    return ms


def pinned_like(a, torch):
    """A page-locked host copy of numpy array `a` (made outside any timed region)."""
    import numpy as np

    dt = {np.dtype(np.float64): torch.float64, np.dtype(np.float32): torch.float32}[a.dtype]
    out = torch.empty(a.shape, dtype=dt, pin_memory=True).numpy()
    out[...] = a
    return out


def time_e2e(rti, sc, steps, world, shape=None):
    """The same rate through the public API with host buffers in pinned memory: create
    (bathymetry and Manning n copied in), initial uplift, the steps, and the forecast
    outputs (max depth and arrival time of every block) copied back into the caller's
    arrays, all inside the timed region."""
    import numpy as np
    import torch

    bathy = [pinned_like(np.asarray(x, np.float64), torch) for x in sc.bathy]
    man = [pinned_like(np.asarray(x, np.float32), torch) for x in sc.manning]
    dz = [None if u is None else pinned_like(np.asarray(u, np.float64), torch) for u in sc.uplift]
    outs = [(pinned_like(np.zeros((b["ny"], b["nx"])), torch),
             pinned_like(np.zeros((b["ny"], b["nx"])), torch)) for b in sc.blocks]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    shape = shape or {}
    h = rti.Handle(sc.blocks, bathy, man, sc.dt, sc.g, sc.dry_eps, sc.arrival_thr,
                   precision=rti.FP32, schedule=shape.get("schedule", 0),
                   tile=(0, shape.get("tile_y", 0)), ctas_per_sm=shape.get("ctas_per_sm", 0))
    for k, u in enumerate(dz):
        if u is not None:
            h.set_initial_uplift(k, u)
    h.step(steps)
    for k, (md, at) in enumerate(outs):
        h.max_depth(k, out=md)
        h.arrival_time(k, out=at)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    h2d, d2h = h.transfer_bytes()
    h.close()
    return wall, h2d, d2h


def serving(rti, sc5, a, world):
    """Serving (C5). (1) A Poisson trace (mean inter-arrival 20 s, kinds 3-/4-/5-level
    uniform, 1-6 simulated hours), arrivals and durations scaled by --serve-scale, through
    the continuous-batching FP32 server: p50/p99 time to forecast, scenarios/h, the FP64
    audit. (2) Capacity at saturation: the first --serve-sat-n requests of the trace all
    arriving at t = 0 (durations scaled by --serve-sat-scale), served by the batched FP32
    server and by the plain per-scenario FP64 path (each request created, stepped to its
    end and read back alone, one after another), every request run in both. (3) With
    --serve-real, the 10-arrival smoke trace at its real durations through the server."""
    import torch

    from paper_2408_07609_gb300 import scenarios as S
    from paper_2408_07609_gb300 import serve

    sites = {"3level": S.serving_hierarchy("3level", seed=1000, hours=0.0),
             "4level": S.serving_hierarchy("4level", seed=1001, hours=0.0), "5level": sc5}
    trace = S.poisson_trace(seed=2024, n=a.serve_n, mean_s=20.0)
    barrier(world)
    shape = {"tile_y": 0, "ctas_per_sm": 0}
    if not a.no_autotune:
        from paper_2408_07609_gb300 import autotune

        mix = [S.with_new_source(sites[k], 7 + i) for i, k in enumerate(sorted(sites))]
        t = autotune.tune_batch(mix, precision=rti.FP32, chunk_steps=(50,), tile_y=(32, 64, 96),
                                ctas=(0, 4), cache_path=a.tune_cache)
        shape = {"tile_y": t["tile_y"], "ctas_per_sm": t["ctas_per_sm"]}
    srv = serve.Server(sites, pool_bytes=a.serve_pool_gb << 30, precision=rti.FP32,
                       chunk_steps=50, audit_every=a.serve_audit_every or None, **shape)
    reqs, st = srv.run(trace, time_scale=a.serve_scale, max_wall_s=180.0)
    srv.audit_every = None
    sat = [dict(t, arrival_s=0.0) for t in trace[:a.serve_sat_n]]
    _, s32 = srv.run(sat, time_scale=a.serve_sat_scale, max_wall_s=300.0)
    _, s64 = srv.run_plain(sat, precision=rti.FP64, time_scale=a.serve_sat_scale,
                           max_wall_s=300.0)
    real = None
    if a.serve_real:
        smoke = S.poisson_trace(seed=2025, n=10, mean_s=20.0)
        _, real = srv.run(smoke, time_scale=1.0, max_wall_s=1800.0)
        real = {k: real[k] for k in ("requests", "completed", "wall_s", "p50_s", "p99_s",
                                     "mean_s", "scenarios_per_h", "max_live", "gcups",
                                     "admit_s", "admit_max_s")}
        real["trace"] = "10 Poisson arrivals (mean 20 s), 3/4/5-level uniform, 1-6 h, real durations"
    srv.close()
    del srv
    torch.cuda.empty_cache()
    keys = ("requests", "completed", "wall_s", "scenarios_per_h", "p50_s", "p99_s", "mean_s",
            "max_live", "gcups")
    return {"scenarios_per_h": st["scenarios_per_h"], "p50_s": st["p50_s"], "p99_s": st["p99_s"],
            "mean_s": st["mean_s"], "completed": st["completed"], "requests": st["requests"],
            "max_live": st["max_live"], "gcups": st["gcups"], "precision": "fp32",
            "admit_s": st["admit_s"], "admit_max_s": st["admit_max_s"],
            "launch_shape": shape,
            "fp64_audit": st["audit"],
            "trace": f"{a.serve_n} Poisson arrivals (mean 20 s), 3/4/5-level uniform, "
                     f"1-6 h; arrivals and durations x{a.serve_scale:.4g}; "
                     f"HBM pool {a.serve_pool_gb} GB; chunk 50 steps",
            "saturation": {
                "trace": f"the first {len(sat)} requests of the trace, all arriving at t = 0, "
                         f"durations x{a.serve_sat_scale:.4g}; every request run by both arms",
                "fp32_batched": {k: s32[k] for k in keys},
                "fp64_plain": {k: s64[k] for k in keys},
                "how": "fp32_batched: the continuous-batching server (one persistent launch "
                       "per 50-step chunk over every live request, admission by footprint); "
                       "fp64_plain: one request at a time in arrival order, created, stepped "
                       "to its end and read back alone"},
            "real_durations": real}


def batch_c3(rti, steps=200, warmup=5, tune=True, cache=None):
    """C3: the 64 single grids (sides 128-1024, ~15.9 M cells) stepped together by one
    batch (one persistent, graph-captured launch per chunk), CUDA events around the
    steps, in FP32 (the autotuner's strip height, CTA cap and chunk length, and the
    default shape beside it) and FP64 (default shape)."""
    import torch

    from paper_2408_07609_gb300 import scenarios as S

    grids = S.config3(count=64, steps=steps + warmup)
    cells = sum(g.cells for g in grids)
    out = {"workload": f"64 grids, {cells / 1e6:.2f} M cells"}
    runs = [("fp32_default", rti.FP32, steps, 0, 0), ("fp64", rti.FP64, max(10, steps // 10), 0, 0)]
    if tune:
        from paper_2408_07609_gb300 import autotune

        t = autotune.tune_batch(grids, precision=rti.FP32, chunk_steps=(50, 100, 200),
                                tile_y=(32, 64, 96), ctas=(0, 4), cache_path=cache)
        runs.insert(0, ("fp32", rti.FP32, t["chunk_steps"], t["tile_y"], t["ctas_per_sm"]))
        out["tuned"] = {k: t[k] for k in ("tile_y", "ctas_per_sm", "chunk_steps")}
    for name, prec, n, ty, cap in runs:
        hs = [rti.Handle.from_scenario(g, precision=prec, tile=(0, ty)) for g in grids]
        stream = torch.cuda.Stream()
        b = rti.Batch(prec, rti.SCHED_PERSISTENT, n, tile_y=ty, ctas_per_sm=cap)
        for h in hs:
            b.add(h, n + n)
        b.step(stream)  # warm-up chunk (uploads the tile list, captures the graph)
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(stream)
        e1.record(stream)
        b.sync()
        ms = e0.elapsed_time(e1)
        out[name] = {"value": cells * n / (ms / 1e3) / 1e9, "unit": "GCUPS", "steps": n,
                     "tile_y": ty or 64, "ctas_per_sm": cap}
        b.close()
        for h in hs:
            h.close()
    return out


def accuracy(rti, sc=None, steps=None):
    """FP32 against the FP64 path (which matches the FP64 oracle to 1e-12), by default on
    the 3-level C2 nest over its full hour: max |eta| and max-height error (m), wet/dry
    mismatch (% of cells, final state and ever-wet), arrival-time error (s; max, p99,
    mean)."""
    import numpy as np

    from paper_2408_07609_gb300 import scenarios as S

    sc = S.config2() if sc is None else sc
    steps = sc.steps if steps is None else steps
    hs = {p: rti.Handle.from_scenario(sc, precision=p) for p in (rti.FP32, rti.FP64)}
    for h in hs.values():
        h.step(steps)
    e_eta = e_max = e_open = 0.0
    at_worst = None
    mis_wet = mis_ever = n = 0
    arr_err, arr_mis = [], 0
    for k, b in enumerate(sc.blocks):
        h0 = np.asarray(sc.bathy[k])
        e32, e64 = hs[rti.FP32].get_state(k)[0], hs[rti.FP64].get_state(k)[0]
        m32, m64 = hs[rti.FP32].max_height(k), hs[rti.FP64].max_height(k)
        a32, a64 = hs[rti.FP32].arrival_time(k), hs[rti.FP64].arrival_time(k)
        d = np.abs(e32 - e64)
        if float(d.max()) > e_eta:
            j, i = np.unravel_index(int(d.argmax()), d.shape)
            at_worst = {"block": k, "cell": [int(i), int(j)], "depth64_m": float(h0[j, i] + e64[j, i]),
                        "depth32_m": float(h0[j, i] + e32[j, i])}
        e_eta = max(e_eta, float(d.max()))
        # open water: the cell and its 8 neighbours wet in both runs (no front nearby)
        wet = (h0 + e32 > sc.dry_eps) & (h0 + e64 > sc.dry_eps)
        op = wet.copy()
        op[1:, :] &= wet[:-1, :]
        op[:-1, :] &= wet[1:, :]
        op2 = op.copy()
        op2[:, 1:] &= op[:, :-1]
        op2[:, :-1] &= op[:, 1:]
        if op2.any():
            e_open = max(e_open, float(d[op2].max()))
        both = ~np.isnan(m32) & ~np.isnan(m64)
        if both.any():
            e_max = max(e_max, float(np.abs(m32[both] - m64[both]).max()))
        mis_wet += int(((h0 + e32 > sc.dry_eps) != (h0 + e64 > sc.dry_eps)).sum())
        mis_ever += int((np.isnan(m32) != np.isnan(m64)).sum())
        n += h0.size
        ab = (a32 >= 0) & (a64 >= 0)
        arr_err.append(np.abs(a32[ab] - a64[ab]))
        arr_mis += int(((a32 >= 0) != (a64 >= 0)).sum())
    for h in hs.values():
        h.close()
    ae = np.concatenate(arr_err)
    return {"workload": sc.name, "against": "FP64 GPU path", "steps": steps,
            "max_abs_eta_m": e_eta, "max_abs_eta_open_water_m": e_open, "worst_cell": at_worst,
            "max_abs_max_height_m": e_max,
            "wet_dry_mismatch_pct": 100.0 * mis_wet / n, "ever_wet_mismatch_pct": 100.0 * mis_ever / n,
            "arrival_max_err_s": float(ae.max()) if ae.size else 0.0,
            "arrival_mean_err_s": float(ae.mean()) if ae.size else 0.0,
            "arrival_p99_err_s": float(np.percentile(ae, 99)) if ae.size else 0.0,
            "arrived_cells": int(ae.size),
            "arrival_mismatch_cells": arr_mis}


def latency(rti, steps=200, warmup=5):
    """Time per step of the small configurations, which fit in L2 (so latency, not a
    roofline): the 256 x 256 single grid and the 3-level 765 k-cell nest, each precision,
    one persistent launch of `steps` (the nest: steps / 2) after `warmup`."""
    from paper_2408_07609_gb300 import scenarios as S

    out = {}
    for name, sc, n in (("single_grid_256x256", S.config1(steps=0), steps),
                        ("nest_3level_765k", S.config2(steps=0), steps // 2)):
        for prec, label in ((rti.FP32, "fp32"), (rti.FP64, "fp64")):
            ms = time_device(rti, sc, prec, n, warmup, 0, 1)
            out[f"{name}_{label}_us_per_step"] = 1e3 * ms / n
    return out


def cpu_baseline(sc, steps, parallel):
    """The FP64 oracle, as it stands, on the host: a bounded sample of the workload, in
    its OpenMP build over every host core (parallel) or single-threaded. Returns the
    seconds of the steps and the threads used."""
    from oracle import oracle

    oracle.build()
    o = oracle.from_scenario(sc, parallel=parallel)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    o.close()
    return dt, (oracle.threads() if parallel else 1)


def run_ours(a):
    import torch

    from paper_2408_07609_gb300 import build, rti

    rank, world, local = dist_setup(a.gpus)
    build.build()
    sc = workload()
    cells = sc.cells
    fp32_bytes = rti.footprint(sc.blocks, rti.make_params(sc.dt, precision=rti.FP32))
    shape = {"tile_y": a.tile[1], "ctas_per_sm": 0, "schedule": a.schedule}
    tuned = None
    if not a.no_autotune and not a.tile[0]:
        from paper_2408_07609_gb300 import autotune

        tuned = autotune.tune_handle(sc, precision=rti.FP32, steps=(10, 40),
                                     cache_path=a.tune_cache, tile_y=(32, 48, 64, 96, 128),
                                     ctas=(0, 4), schedules=(rti.SCHED_PERSISTENT,),
                                     **handle_options(a))
        shape = {k: tuned[k] for k in ("tile_y", "ctas_per_sm", "schedule")}
    with Clocks(local) as clk:
        ms32 = time_device(rti, sc, rti.FP32, a.steps, a.warmup, shape["schedule"], world,
                           (0, shape["tile_y"]), handle_options(a), shape["ctas_per_sm"])
    clocks = clk.summary()
    ms32 = max_over_ranks(ms32, world)
    ms64 = time_device(rti, sc, rti.FP64, a.fp64_steps, max(3, a.warmup // 2), a.schedule, world,
                       a.tile, handle_options(a))
    ms64 = max_over_ranks(ms64, world)
    per32, per64 = ms32 / a.steps, ms64 / a.fp64_steps
    gcups32 = whole_job_rate(cells, a.steps, ms32, world)
    gcups64 = whole_job_rate(cells, a.fp64_steps, ms64, world)
    peak, kind = peaks()
    bpc = BYTES_PER_CELL_STEP["f32"] + (4 if a.track_velocity else 0)  # + max-speed plane read
    default_run = (a.nest_feedback, a.nest_flux, a.track_velocity) == ("ring", "linear", False)
    achieved = bpc * cells * a.steps / (ms32 / 1e3) / 1e9  # GB/s of one launch of K steps
    e2e = None
    if not a.no_e2e:
        wall, h2d, d2h = time_e2e(rti, sc, a.steps, world, shape)
        wall = max_over_ranks(wall, world)
        e2e = {"value": world * cells * a.steps / wall / 1e9, "unit": "GCUPS",
               "h2d_bytes_per_step": h2d // a.steps, "d2h_bytes_per_step": d2h // a.steps,
               "includes": "create (bathymetry, Manning n), initial uplift, steps, max depth "
                           "and arrival of every block read back; host arrays in pinned "
                           "memory"}
    srv = None if a.no_serving else serving(rti, sc, a, world)
    acc = None if (a.no_accuracy or rank != 0) else accuracy(rti)
    acc4 = None if (not a.accuracy_c4_steps or rank != 0) else accuracy(rti, sc, a.accuracy_c4_steps)
    c3 = None if a.no_batch else batch_c3(rti, tune=not a.no_autotune, cache=a.tune_cache)
    lat = None if (a.no_latency or rank != 0 or world != 1) else latency(rti)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        dt, cores = cpu_baseline(sc, a.cpu_steps, parallel=True)
        dt1, _ = cpu_baseline(sc, 1, parallel=False)
        cpu = {"value": cells * a.cpu_steps / dt / 1e9, "unit": "GCUPS", "cores": cores,
               "kind": "oracle",
               "sample": f"{a.cpu_steps} FP64 steps of the full 46.65 M-cell hierarchy "
                         f"(C oracle, OpenMP build, {cores} threads)",
               "single_thread": {"value": cells / dt1 / 1e9, "unit": "GCUPS", "cores": 1,
                                 "sample": "1 FP64 step of the full hierarchy, plain build"},
               "nproc": os.cpu_count()}
    if rank == 0:
        emit({
            "metric": "GCUPS of the nested leap-frog step, 46.65 M-cell 5-level hierarchy, "
                      "binary32 (binary64 and 6-h wall times beside it)",
            "value": gcups32, "unit": "GCUPS", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": per32, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": sc.name, "cells": cells, "blocks": len(sc.blocks),
                       "levels": 5, "dt_s": sc.dt, "precision": "fp32",
                       "schedule": "persistent" if shape["schedule"] == 0 else "one launch per step",
                       "strip": [28, shape["tile_y"] or 64],
                       "ctas_per_sm": shape["ctas_per_sm"] or "all that fit",
                       "launch_shape_by": "autotuner" if tuned else "default",
                       "nesting": f"{a.nest_feedback} feedback, {a.nest_flux} edge flux",
                       "max_velocity": bool(a.track_velocity),
                       "l2": f"working set {fp32_bytes / 1e9:.2f} GB (fp32) > 129 MB L2; no flush",
                       "parallelism": f"replicas x{world}"},
            "fp64": {"value": gcups64, "unit": "GCUPS", "ms_per_step": per64,
                     "steps": a.fp64_steps},
            "wall_6h_s": {"fp32": per32 * SIX_HOURS_STEPS / 1e3,
                          "fp64": per64 * SIX_HOURS_STEPS / 1e3,
                          "paper_context": "Kochi 47.2 M cells: 82 s on 32 H100 PCIe, "
                                           "< 2.5 min on 32 Sapphire Rapids CPUs"},
            "e2e": e2e,
            # per timed rti_step: k_set_scen, the step kernel(s), k_advance
            "gpu_launches": 3 if shape["schedule"] == 0 else a.steps + 2,
            "serving": srv,
            "autotune": None if not tuned else {
                "choice": shape, "ms_per_step_short_run": tuned["ms_per_step"],
                "cached": tuned["cached"], "cost_model": tuned["model"],
                "trials": [{k: t[k] for k in ("tile_y", "ctas_per_sm", "schedule", "ms_per_step")}
                           for t in tuned["trials"]]},
            "fp32_accuracy": acc,
            "fp32_accuracy_c4": acc4,
            "batch_c3": c3,
            "latency_small": lat,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": (None if NCU_F32_DRAM_BYTES_PER_CELL_STEP is None
                                     or not default_run else
                                     NCU_F32_DRAM_BYTES_PER_CELL_STEP * cells * a.steps),
                         "traffic_note": "bytes per launch of the timed K steps, scaled from "
                                         "a single-step ncu capture of the 4-level case",
                         "peak_kind": f"{kind} hbm_gbs",
                         "bytes_per_cell_step": bpc,
                         "kernel": ("k_step_flow" if a.nest_feedback == "full" else "k_step")
                                   + f"<float, {(1 if a.track_velocity else 0) | (4 if a.nest_feedback == 'full' else 0)}>"},
            "cpu_baseline": cpu,
            "clocks": clocks,
        })


def reference_sample(sc, per_step_cells):
    """The part of the workload one reference step covers: the longest prefix of its
    blocks (parents come first, so a prefix is itself a nested hierarchy) holding at most
    per_step_cells cells; when even the root holds more, the root's first rows alone
    (its own edges, bathymetry and source), at least 3 of them. Returns the sample,
    its block count and its cells."""
    import copy

    import numpy as np

    root = sc.blocks[0]
    nx, ny = root["nx"], root["ny"]
    sub = copy.copy(sc)
    if nx * ny > per_step_cells:
        rows = max(3, min(ny, int(per_step_cells // nx)))
        sub.blocks = [dict(root, ny=rows)]
        sub.bathy = [np.asarray(sc.bathy[0])[:rows].copy()]
        sub.manning = [np.asarray(sc.manning[0])[:rows].copy()]
        sub.uplift = [None if sc.uplift[0] is None else np.asarray(sc.uplift[0])[:rows].copy()]
        return sub, 1, nx * rows
    n, cells = 1, nx * ny
    while n < len(sc.blocks):
        c = sc.blocks[n]["nx"] * sc.blocks[n]["ny"]
        if cells + c > per_step_cells:
            break
        cells += c
        n += 1
    sub.blocks, sub.bathy, sub.manning = sc.blocks[:n], sc.bathy[:n], sc.manning[:n]
    sub.uplift = sc.uplift[:n]
    return sub, n, cells


def run_reference(a):
    """The FP64 oracle on the host, on the same workload and metric: W untimed warm-up
    steps, then K timed steps, each over a bounded sample of the hierarchy (its first
    blocks, about REF_CELL_STEPS cell-steps in all) so that the run ends within minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle

    sc = workload()
    oracle.build()
    cores = oracle.threads()
    sub, nblk, cells = reference_sample(sc, REF_CELL_STEPS * cores / max(1, a.steps + a.warmup))
    o = oracle.from_scenario(sub, parallel=True)
    o.step(a.warmup)
    t0 = time.perf_counter()
    o.step(a.steps)
    dt = time.perf_counter() - t0
    o.close()
    v = cells * a.steps / dt / 1e9
    part = (f"first {nblk} of {len(sc.blocks)} blocks" if sub.blocks[0]["ny"] == sc.blocks[0]["ny"]
            else f"first {sub.blocks[0]['ny']} rows of the root block")
    sample = (f"{part} ({cells / 1e6:.2f} M of {sc.cells / 1e6:.2f} M cells) per step, "
              f"C oracle, OpenMP build, {cores} threads")
    emit({"impl": "reference",
          "metric": "GCUPS of the nested leap-frog step, 46.65 M-cell 5-level hierarchy, "
                    "binary32 (binary64 and 6-h wall times beside it)",
          "value": v, "unit": "GCUPS", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
          "ms_per_step": dt / max(1, a.steps) * 1e3, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": sc.name, "cells": sc.cells, "sample_cells": cells},
          "cpu_baseline": {"value": v, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                           "sample": sample},
          "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
