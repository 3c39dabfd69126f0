"""Continuous-batching forecast server over the batch API.

Requests (an earthquake source on one of a few pre-built grid hierarchies, the "sites")
arrive over time. A request is admitted as soon as it has arrived and its device
footprint (rti_footprint) fits in a fixed HBM pool; its state then stays resident in the
pool while the batch steps it together with every other live request, chunk by chunk,
in one graph-captured persistent launch. Requests that finish leave the batch between
chunks, their results (maximum height and arrival time of every block) are read back to
the host, and their memory returns to the pool, so new arrivals join while others run.
Time to forecast is measured from a request's arrival to the moment its results are on
the host.

The pool is one caller-owned device allocation (a torch uint8 tensor) carved first-fit
into 256-byte aligned arenas, so admission and retirement allocate no arena of their
own. Admissions happen between chunks: the host part of one (the request's source, the
input scan of rti_create) runs while the chunk just launched is on the GPU, but
rti_create and rti_set_initial_uplift synchronise the device, so the device part of an
admission waits for that chunk and delays the next one. The server records the wall
time spent admitting (admit_s) so that its share of the time to forecast is reported.

`run_plain` serves the same trace the plain way for comparison: one request at a time
in arrival order, each created, stepped to its end and read back alone.

Audit: with audit_every = N, every N-th request (by arrival) is run again in binary64
once the trace is served, off the forecast path, and its forecast outputs (maximum
height and arrival time of every block) are compared with the binary32 forecast.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import rti
from . import scenarios as S

ALIGN = 256


class Pool:
    """First-fit allocator of 256-byte aligned ranges of one device buffer."""

    def __init__(self, nbytes: int, device_buffer=None):
        self.size = int(nbytes) // ALIGN * ALIGN
        self.buf = device_buffer
        self.free = [(0, self.size)]  # sorted (offset, length)
        self.used = {}

    def alloc(self, nbytes: int):
        need = (int(nbytes) + ALIGN - 1) // ALIGN * ALIGN
        for k, (off, ln) in enumerate(self.free):
            if ln >= need:
                if ln == need:
                    self.free.pop(k)
                else:
                    self.free[k] = (off + need, ln - need)
                self.used[off] = need
                return off
        return None

    def release(self, off: int):
        ln = self.used.pop(off)
        self.free.append((off, ln))
        self.free.sort()
        merged = []
        for o, n in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + n)
            else:
                merged.append((o, n))
        self.free = merged

    def view(self, off: int):
        return self.buf[off:off + self.used[off]]

    @property
    def in_use(self) -> int:
        return sum(self.used.values())


@dataclass
class Request:
    rid: int
    kind: str
    seed: int
    hours: float
    arrival_s: float
    nsteps: int = 0
    footprint: int = 0
    cells: int = 0
    admitted_s: float = float("nan")
    admit_wall_s: float = 0.0  # wall time of this request's admission (create + uplift)
    done_s: float = float("nan")
    result: dict = field(default_factory=dict)
    fields: dict = field(default_factory=dict)  # kept for the audit: block -> (max h, arrival)
    audit: dict = field(default_factory=dict)

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def load_sites(kinds=("3level", "4level", "5level"), seed=1000):
    """One fixed hierarchy per kind (the site's grids; requests only change the source)."""
    return {k: S.serving_hierarchy(k, seed=seed + i, hours=0.0) for i, k in enumerate(kinds)}


class Server:
    def __init__(self, sites: dict, pool_bytes: int, precision=rti.FP32, chunk_steps: int = 50,
                 schedule=rti.SCHED_PERSISTENT, keep_fields: bool = False,
                 audit_every: int | None = None, tile_y: int = 0, ctas_per_sm: int = 0):
        import torch

        self.torch = torch
        self.sites = sites
        self.prec = precision
        self.keep = keep_fields
        self.audit_every = audit_every
        self.pool = Pool(pool_bytes, torch.empty(int(pool_bytes), dtype=torch.uint8,
                                                 device="cuda"))
        self.tile_y = int(tile_y)
        self.batch = rti.Batch(precision, schedule, chunk_steps, tile_y=tile_y,
                               ctas_per_sm=ctas_per_sm)
        self.stream = torch.cuda.Stream()
        self.chunk = chunk_steps

    def _admit(self, req: Request, live: dict):
        site = self.sites[req.kind]
        sc = S.with_new_source(site, req.seed)
        off = self.pool.alloc(req.footprint)
        if off is None:
            return False
        h = rti.Handle.from_scenario(sc, precision=self.prec, device_mem=self.pool.view(off),
                                     tile=(0, self.tile_y))
        self.batch.add(h, req.nsteps)
        live[req.rid] = (req, h, off)
        return True

    def _audited(self, req: Request) -> bool:
        return bool(self.audit_every) and req.rid % self.audit_every == 0

    def _retire(self, req: Request, h: rti.Handle, off: int, t0: float):
        out = {}
        for k in range(len(h.blocks)):
            mh, at = h.max_height(k), h.arrival_time(k)
            if self._audited(req):
                req.fields[k] = (mh, at)
            if self.keep:
                out[k] = (mh, at)
            else:
                wet = ~np.isnan(mh)
                out[k] = (float(np.nanmax(mh)) if wet.any() else float("nan"),
                          int((at >= 0).sum()))
        req.result = out
        req.done_s = time.perf_counter() - t0
        self.batch.remove(h)
        h.close()
        self.pool.release(off)

    def _audit(self, req: Request):
        """Run `req` again in binary64 in the pool and compare its forecast outputs."""
        site = self.sites[req.kind]
        sc = S.with_new_source(site, req.seed)
        p = rti.make_params(site.dt, site.g, site.dry_eps, site.arrival_thr, rti.FP64)
        off = self.pool.alloc(rti.footprint(site.blocks, p))
        if off is None:
            raise MemoryError(f"audit of request {req.rid} does not fit the pool")
        h = rti.Handle.from_scenario(sc, precision=rti.FP64, device_mem=self.pool.view(off))
        h.step(req.nsteps)
        d_max, d_arr, mis = 0.0, 0.0, 0
        for k in range(len(h.blocks)):
            mh, at = h.max_height(k), h.arrival_time(k)
            mh32, at32 = req.fields[k]
            both = ~np.isnan(mh) & ~np.isnan(mh32)
            if both.any():
                d_max = max(d_max, float(np.abs(mh[both] - mh32[both]).max()))
            mis += int((np.isnan(mh) != np.isnan(mh32)).sum() + ((at >= 0) != (at32 >= 0)).sum())
            ab = (at >= 0) & (at32 >= 0)
            if ab.any():
                d_arr = max(d_arr, float(np.abs(at[ab] - at32[ab]).max()))
        h.close()
        self.pool.release(off)
        req.fields = {}
        req.audit = dict(max_height_err_m=d_max, arrival_err_s=d_arr, mismatched_cells=mis)

    def run(self, trace, time_scale: float = 1.0, max_wall_s: float | None = None,
            admit_per_chunk: int | None = None):
        """Serve `trace` (dicts with arrival_s, kind, seed, hours); arrival times and
        simulated durations are multiplied by time_scale. At most admit_per_chunk
        requests join between two chunks (None: all that have arrived and fit). The
        binary64 audit of the sampled requests follows the trace.
        Returns (requests, stats)."""
        reqs = self.requests(trace, time_scale)
        for r in reqs:
            if r.footprint > self.pool.size:
                raise ValueError(f"request {r.rid} ({r.kind}) needs {r.footprint} B, "
                                 f"pool is {self.pool.size}")
        pending = list(reqs)
        live = {}
        max_live, chunks = 0, 0
        t0 = time.perf_counter()
        while pending or live:
            now = time.perf_counter() - t0
            if max_wall_s is not None and now > max_wall_s:
                break
            launched = False
            if live:
                with self.torch.cuda.stream(self.stream):
                    self.batch.step(self.stream)
                launched = True
                chunks += 1
            # admissions overlap the chunk in flight (arrival order, while memory fits)
            admitted = 0
            while pending and pending[0].arrival_s <= time.perf_counter() - t0:
                if admit_per_chunk is not None and admitted >= admit_per_chunk:
                    break
                r = pending[0]
                ta0 = time.perf_counter()
                if not self._admit(r, live):
                    break
                r.admitted_s = time.perf_counter() - t0
                r.admit_wall_s = r.admitted_s - (ta0 - t0)
                pending.pop(0)
                admitted += 1
            max_live = max(max_live, len(live))
            if launched:
                self.batch.sync()
                for rid in [k for k, (r, h, o) in live.items() if self.batch.remaining(h) == 0]:
                    r, h, off = live.pop(rid)
                    self._retire(r, h, off, t0)
            elif pending and not live:
                time.sleep(max(0.0, min(0.05, pending[0].arrival_s - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        done = [r for r in reqs if np.isfinite(r.done_s)]
        ta = time.perf_counter()
        audited = [r for r in done if self._audited(r)]
        for r in audited:
            self._audit(r)
        audit = None
        if audited:
            audit = dict(requests=len(audited), wall_s=time.perf_counter() - ta,
                         max_height_err_m=max(r.audit["max_height_err_m"] for r in audited),
                         arrival_err_s=max(r.audit["arrival_err_s"] for r in audited),
                         mismatched_cells=sum(r.audit["mismatched_cells"] for r in audited))
        lat = np.array([r.latency_s for r in done]) if done else np.array([float("nan")])
        cell_steps = float(sum(r.cells * r.nsteps for r in done))
        stats = dict(requests=len(reqs), completed=len(done), wall_s=wall,
                     scenarios_per_h=len(done) / wall * 3600.0 if wall > 0 else float("nan"),
                     p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                     mean_s=float(lat.mean()), max_live=max_live, chunks=chunks,
                     gcups=cell_steps / wall / 1e9 if wall > 0 else float("nan"),
                     admit_s=float(sum(r.admit_wall_s for r in reqs)),
                     admit_max_s=float(max((r.admit_wall_s for r in reqs), default=0.0)),
                     time_scale=time_scale, audit=audit)
        return reqs, stats

    def requests(self, trace, time_scale: float = 1.0, precision=None):
        """Request records of a trace (steps, footprint, cells) without serving it."""
        prec = self.prec if precision is None else precision
        out = []
        for i, t in enumerate(trace):
            site = self.sites[t["kind"]]
            nsteps = max(1, int(round(t["hours"] * 3600.0 * time_scale / site.dt)))
            r = Request(i, t["kind"], int(t["seed"]), float(t["hours"]),
                        float(t["arrival_s"]) * time_scale, nsteps)
            p = rti.make_params(site.dt, site.g, site.dry_eps, site.arrival_thr, prec,
                                tile=(0, self.tile_y))
            r.footprint = rti.footprint(site.blocks, p)
            r.cells = site.cells
            out.append(r)
        return out

    def run_plain(self, trace, precision=rti.FP64, time_scale: float = 1.0,
                  max_wall_s: float | None = None):
        """The plain per-scenario path on the same trace: one request at a time, in arrival
        order, each created in the pool, stepped to its end in one rti_step call and read
        back (maximum height and arrival time of every block) before the next one starts.
        Returns (requests, stats) like run()."""
        reqs = self.requests(trace, time_scale, precision)
        t0 = time.perf_counter()
        for r in reqs:
            now = time.perf_counter() - t0
            if max_wall_s is not None and now > max_wall_s:
                break
            if r.arrival_s > now:
                time.sleep(r.arrival_s - now)
            sc = S.with_new_source(self.sites[r.kind], r.seed)
            off = self.pool.alloc(r.footprint)
            if off is None:
                raise MemoryError(f"request {r.rid} does not fit the pool")
            r.admitted_s = time.perf_counter() - t0
            h = rti.Handle.from_scenario(sc, precision=precision, device_mem=self.pool.view(off),
                                         tile=(0, self.tile_y))
            h.step(r.nsteps, self.stream)
            out = {}
            for k in range(len(h.blocks)):
                mh, at = h.max_height(k), h.arrival_time(k)
                wet = ~np.isnan(mh)
                out[k] = (float(np.nanmax(mh)) if wet.any() else float("nan"),
                          int((at >= 0).sum()))
            r.result = out
            r.done_s = time.perf_counter() - t0
            h.close()
            self.pool.release(off)
        wall = time.perf_counter() - t0
        done = [r for r in reqs if np.isfinite(r.done_s)]
        lat = np.array([r.latency_s for r in done]) if done else np.array([float("nan")])
        cell_steps = float(sum(r.cells * r.nsteps for r in done))
        stats = dict(requests=len(reqs), completed=len(done), wall_s=wall,
                     scenarios_per_h=len(done) / wall * 3600.0 if wall > 0 else float("nan"),
                     p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                     mean_s=float(lat.mean()), max_live=1,
                     gcups=cell_steps / wall / 1e9 if wall > 0 else float("nan"),
                     time_scale=time_scale)
        return reqs, stats

    def close(self):
        for h in list(self.batch.members):
            self.batch.remove(h)
            h.close()
        self.batch.close()
