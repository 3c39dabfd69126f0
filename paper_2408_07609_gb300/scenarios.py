"""Seeded synthetic inputs for the nested-grid tsunami step.

This module builds INPUTS only: block hierarchies, bathymetry h (m, positive
below still water, negative on land), Manning n and initial uplift dz. It holds
none of the time step's arithmetic and is shared by the CUDA path, the oracle
tests and the benchmark.

The paper's Kochi model (Table I: 5 levels at 810/270/90/30/10 m, 1:3 nesting,
dt = 0.2 s) and its bathymetry are not available, so every workload here is a
synthetic stand-in of the same shape: a subduction margin (trench, slope,
shelf), a wiggly coastline, low land with fractal relief, and nested blocks that
follow the coast, finer levels placed in water shallow enough for the CFL rule
of Eq. 4 with a 10 % margin.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

G = 9.81
BC_WALL, BC_RADIATION = 0, 1


@dataclass
class Scenario:
    name: str
    blocks: list            # dicts: level, parent, nx, ny, i0, j0, dx, bc
    bathy: list             # (ny, nx) float64 per block
    manning: list           # (ny, nx) float32 per block
    uplift: list            # (ny, nx) float64 per block, or None (sea at rest)
    dt: float
    steps: int
    g: float = G
    dry_eps: float = 1e-3
    arrival_thr: float = 0.01
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return int(sum(b["nx"] * b["ny"] for b in self.blocks))

    def truncated(self, steps: int) -> "Scenario":
        s = Scenario(**{**self.__dict__})
        s.steps = steps
        return s


# --------------------------------------------------------------------------- helpers
def _fractal(rng, ny, nx, beta=2.0, amp=2.0):
    """Isotropic power-law noise (spectral exponent beta), scaled to max |.| = amp."""
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.rfftfreq(nx)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    k[0, 0] = 1.0
    spec = (rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape)) * k ** (-beta / 2)
    spec[0, 0] = 0.0
    f = np.fft.irfft2(spec, s=(ny, nx))
    m = np.abs(f).max()
    return (f * (amp / m) if m > 0 else f).astype(np.float64)


class _Margin:
    """Cross-shore profile of a subduction margin. x grows landward (east);
    the coastline is at x = xc(y); d = xc(y) - x is the seaward distance."""

    def __init__(self, rng, Ly, xc0, shelf_w, slope_w, shelf_depth, deep, land_max,
                 land_slope, wiggle, trench=None):
        self.xc0, self.shelf_w, self.slope_w = xc0, shelf_w, slope_w
        self.shelf_depth, self.deep, self.land_max, self.land_slope = (
            shelf_depth, deep, land_max, land_slope)
        self.trench = trench  # (distance from coast, depth, width) or None
        nmod = 6
        lam = Ly / np.geomspace(1.5, 40.0, nmod)
        amp = wiggle * (lam / lam[0]) ** 0.8
        amp *= wiggle / amp.sum()
        self.modes = [(a, 2 * math.pi / l, rng.uniform(0, 2 * math.pi)) for a, l in zip(amp, lam)]
        self.wiggle_max = float(sum(a for a, _, _ in self.modes))

    def xc(self, y):
        y = np.asarray(y, dtype=np.float64)
        out = np.full_like(y, self.xc0)
        for a, k, ph in self.modes:
            out += a * np.sin(k * y + ph)
        return out

    def sea_depth(self, d):
        d = np.asarray(d, dtype=np.float64)
        sd, dp, sw, lw = self.shelf_depth, self.deep, self.shelf_w, self.slope_w
        h = np.where(d < sw, sd * d / sw, np.where(d < sw + lw, sd + (dp - sd) * (d - sw) / lw, dp))
        if self.trench is not None:
            td, tdepth, tw = self.trench
            h = h + (tdepth - dp) * np.exp(-(((d - td) / tw) ** 2)) * (d > sw + lw)
        return h

    def depth_limit_distance(self, hlim):
        """Largest seaward distance whose depth stays <= hlim (profile grows seaward)."""
        lo, hi = 0.0, self.shelf_w + self.slope_w
        if self.sea_depth(hi) <= hlim:
            return np.inf
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if self.sea_depth(mid) <= hlim else (lo, mid)
        return lo

    def bathy(self, x, y, relief):
        d = self.xc(y)[:, None] - x[None, :]
        h = self.sea_depth(np.maximum(d, 0.0))
        elev = np.minimum(-d * self.land_slope, self.land_max) + relief
        return np.where(d > 0, h, -elev)


def _ellipse_uplift(x, y, xs, ys, a, b, theta, peak):
    """cos^2-tapered elliptical uplift (semi-axes a, b, strike theta)."""
    X = x[None, :] - xs
    Y = y[:, None] - ys
    u = X * math.cos(theta) + Y * math.sin(theta)
    v = -X * math.sin(theta) + Y * math.cos(theta)
    r = np.sqrt((u / a) ** 2 + (v / b) ** 2)
    return np.where(r < 1.0, peak * np.cos(0.5 * math.pi * np.minimum(r, 1.0)) ** 2, 0.0)


def _gauss_uplift(x, y, xs, ys, sigma, peak):
    return peak * np.exp(-((x[None, :] - xs) ** 2 + (y[:, None] - ys) ** 2) / (2 * sigma**2))


def _place_children(parents, count, nx, ny, margin_cells=3):
    """Distribute `count` children of nx*ny cells over the parent blocks, stacked along y."""
    m = len(parents)
    per = [count // m + (1 if k < count % m else 0) for k in range(m)]
    out = []
    for pk, k in enumerate(per):
        if k == 0:
            continue
        P = parents[pk]
        fh = ny // 3
        free = P["ny"] - 2 * margin_cells - k * fh
        if free < 0 or nx // 3 > P["nx"] - 2 * margin_cells:
            raise ValueError("children do not fit in their parent")
        gap = free // (k + 1)
        for q in range(k):
            j0 = margin_cells + gap * (q + 1) + q * fh
            out.append((pk, j0))
    return out


def coastal_hierarchy(name, seed, root, levels, dt, steps, *, deep=4000.0, trench=None,
                      shelf_w=60e3, slope_w=100e3, shelf_depth=200.0, land_max=30.0,
                      land_slope=0.01, coast_frac=0.75, wiggle=8e3, source=None,
                      relief_amp=2.0, n_sea=0.025, n_land=0.04, land_frac=0.4):
    """Nested coastal hierarchy. root = (nx, ny, dx); levels = [(count, nx, ny), ...];
    source = dict(kind='ellipse', a=..., b=..., peak=...) placed offshore (seeded)."""
    rng = np.random.default_rng(seed)
    rnx, rny, rdx = root
    Lx, Ly = rnx * rdx, rny * rdx
    mg = _Margin(rng, Ly, coast_frac * Lx, shelf_w, slope_w, shelf_depth, deep, land_max,
                 land_slope, wiggle, trench)
    blocks = [dict(level=1, parent=-1, nx=rnx, ny=rny, i0=0, j0=0, dx=rdx,
                   bc=(BC_RADIATION, BC_WALL, BC_RADIATION, BC_RADIATION), x0=0.0, y0=0.0)]
    prev = [0]
    for lev, (count, cnx, cny) in enumerate(levels, start=2):
        pdx = blocks[prev[0]]["dx"]
        cdx = pdx / 3.0
        hlim = 0.9 * (cdx / dt) ** 2 / (2 * G)  # Eq. 4 with a 10 % margin
        dlim = mg.depth_limit_distance(hlim)
        cur = []
        for pk, j0 in _place_children([blocks[p] for p in prev], count, cnx, cny):
            P = blocks[prev[pk]]
            fw, fh = cnx // 3, cny // 3
            ys = P["y0"] + (j0 + np.arange(fh + 1)) * pdx
            xcs = mg.xc(np.linspace(ys[0], ys[-1], 64))
            xw = xcs.mean() - (1.0 - land_frac) * cnx * cdx
            if np.isfinite(dlim):
                xw = max(xw, xcs.max() - dlim + 2 * pdx)
            i0 = int(math.ceil((xw - P["x0"]) / pdx))
            i0 = min(max(i0, 3), P["nx"] - 3 - fw)
            blocks.append(dict(level=lev, parent=prev[pk], nx=cnx, ny=cny, i0=i0, j0=j0, dx=cdx,
                               bc=(BC_WALL,) * 4, x0=P["x0"] + i0 * pdx, y0=P["y0"] + j0 * pdx,
                               hlim=hlim))
            cur.append(len(blocks) - 1)
        prev = cur
    # source offshore, middle third along the coast
    xs = ys = None
    if source is not None:
        ys = Ly * rng.uniform(0.4, 0.6)
        dsrc = shelf_w + slope_w * rng.uniform(0.6, 1.2)
        xs = mg.xc(np.array([ys]))[0] - dsrc
        theta = 0.5 * math.pi + rng.uniform(-0.25, 0.25)
    bathy, manning, uplift = [], [], []
    for k, b in enumerate(blocks):
        x = b["x0"] + (np.arange(b["nx"]) + 0.5) * b["dx"]
        y = b["y0"] + (np.arange(b["ny"]) + 0.5) * b["dx"]
        relief = _fractal(np.random.default_rng([seed, k]), b["ny"], b["nx"], amp=relief_amp)
        h = mg.bathy(x, y, relief)
        if "hlim" in b and h.max() > (b["dx"] / dt) ** 2 / (2 * G):
            raise ValueError(f"block {k} violates the CFL rule (h_max {h.max():.0f} m)")
        bathy.append(h)
        manning.append(np.where(h > 0, n_sea, n_land).astype(np.float32))
        dz = None
        if source is not None:
            if source["kind"] == "ellipse":
                f = _ellipse_uplift(x, y, xs, ys, source["a"], source["b"], theta, source["peak"])
            else:
                f = _gauss_uplift(x, y, xs, ys, source["sigma"], source["peak"])
            if np.any(f != 0):
                dz = f
        uplift.append(dz)
    clean = [{k: v for k, v in b.items() if k in ("level", "parent", "nx", "ny", "i0", "j0", "dx",
                                                   "bc")} for b in blocks]
    return Scenario(name=name, blocks=clean, bathy=bathy, manning=manning, uplift=uplift, dt=dt,
                    steps=steps, meta=dict(seed=seed, source=(xs, ys), margin=mg,
                                           origin=[(b["x0"], b["y0"]) for b in blocks],
                                           source_shape=source, extent=(Lx, Ly),
                                           shelf=(shelf_w, slope_w)))


def with_new_source(site: Scenario, seed: int, peak_range=(2.0, 6.0)) -> Scenario:
    """The same grids, bathymetry and Manning n as `site`, with a new seeded offshore
    source of the site's shape (position along the coast, distance offshore, strike and
    peak drawn from `seed`). Only blocks that the source touches get an uplift array."""
    rng = np.random.default_rng(seed)
    mg, (Lx, Ly) = site.meta["margin"], site.meta["extent"]
    shelf_w, slope_w = site.meta["shelf"]
    shape = dict(site.meta["source_shape"] or dict(kind="ellipse", a=50e3, b=25e3, peak=3.0))
    shape["peak"] = float(rng.uniform(*peak_range))
    ys = Ly * rng.uniform(0.3, 0.7)
    xs = mg.xc(np.array([ys]))[0] - (shelf_w + slope_w * rng.uniform(0.6, 1.2))
    theta = 0.5 * math.pi + rng.uniform(-0.25, 0.25)
    reach = max(shape.get("a", 0.0), 3.0 * shape.get("sigma", 0.0))
    uplift = []
    for b, (x0, y0) in zip(site.blocks, site.meta["origin"]):
        w, h = b["nx"] * b["dx"], b["ny"] * b["dx"]
        if x0 > xs + reach or x0 + w < xs - reach or y0 > ys + reach or y0 + h < ys - reach:
            uplift.append(None)
            continue
        x = x0 + (np.arange(b["nx"]) + 0.5) * b["dx"]
        y = y0 + (np.arange(b["ny"]) + 0.5) * b["dx"]
        if shape["kind"] == "ellipse":
            f = _ellipse_uplift(x, y, xs, ys, shape["a"], shape["b"], theta, shape["peak"])
        else:
            f = _gauss_uplift(x, y, xs, ys, shape["sigma"], shape["peak"])
        uplift.append(f if np.any(f != 0) else None)
    meta = dict(site.meta, seed=seed, source=(xs, ys))
    return Scenario(name=f"{site.name} / source {seed}", blocks=site.blocks, bathy=site.bathy,
                    manning=site.manning, uplift=uplift, dt=site.dt, steps=site.steps,
                    g=site.g, dry_eps=site.dry_eps, arrival_thr=site.arrival_thr, meta=meta)


# --------------------------------------------------------------------------- workloads
def config1(nx=256, ny=256, steps=1800):
    """Single 256x256 grid, dx 1000 m, dt 1 s. Depth 4000 m falling linearly to -20 m
    (land) over the last 40 columns; Gaussian hump 2 m, sigma 20 km, at column 80;
    n = 0.025; radiation west, walls elsewhere."""
    dx = 1000.0
    i = np.arange(nx)
    ramp0 = nx - 40
    prof = np.where(i < ramp0, 4000.0, 4000.0 + (-20.0 - 4000.0) * (i - ramp0 + 1) / 40.0)
    h = np.tile(prof, (ny, 1)).astype(np.float64)
    x = (i + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    dz = _gauss_uplift(x, y, 80.5 * dx, 0.5 * ny * dx, 20e3, 2.0)
    n = np.full((ny, nx), 0.025, np.float32)
    blk = dict(level=1, parent=-1, nx=nx, ny=ny, i0=0, j0=0, dx=dx,
               bc=(BC_RADIATION, BC_WALL, BC_WALL, BC_WALL))
    return Scenario("single-grid 256x256 dx1000 (1800 steps)" if (nx, ny) == (256, 256)
                    else f"single-grid {nx}x{ny} dx1000", [blk], [h], [n], [dz], dt=1.0,
                    steps=steps)


def config2(seed=2, steps=7200):
    """3-level nest 600^2 @ 810 m, 450^2 @ 270 m, 450^2 @ 90 m; dt 0.5 s, 1 h;
    elliptical source 100 x 50 km, 3 m."""
    return coastal_hierarchy(
        "3-level nest 600^2/450^2/450^2 @ 810/270/90 m (1 h)", seed, (600, 600, 810.0),
        [(1, 450, 450), (1, 450, 450)], dt=0.5, steps=steps, deep=4000.0, shelf_w=40e3,
        slope_w=60e3, wiggle=4e3, coast_frac=0.7, source=dict(kind="ellipse", a=50e3, b=25e3,
                                                              peak=3.0), land_frac=0.35)


def config3(seed=3, count=64, steps=2000):
    """64 independent single grids, sides log-uniform in [128, 1024], dx in {90, 270, 810},
    shelf-and-coast bathymetry, Gaussian or elliptical source of 0.5-5 m,
    dt = 0.5 dx / sqrt(2 g h_max) rounded down to 0.01 s."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(round(128 * 8 ** rng.uniform()))
        side = max(128, min(1024, side))
        nx = ny = side
        dx = float(rng.choice([90.0, 270.0, 810.0]))
        L = nx * dx
        deep = float(rng.uniform(1000.0, 4000.0))
        dt = math.floor(100 * 0.5 * dx / math.sqrt(2 * G * deep)) / 100
        kind = "ellipse" if rng.uniform() < 0.5 else "gauss"
        peak = float(rng.uniform(0.5, 5.0))
        size = float(rng.uniform(0.05, 0.10)) * L
        src = (dict(kind="ellipse", a=size, b=0.5 * size, peak=peak) if kind == "ellipse"
               else dict(kind="gauss", sigma=0.5 * size, peak=peak))
        sc = coastal_hierarchy(f"batch grid {k}: {nx}x{ny} dx{dx:.0f}", int(rng.integers(1 << 30)),
                               (nx, ny, dx), [], dt=dt, steps=steps, deep=deep, shelf_w=0.12 * L,
                               slope_w=0.15 * L, land_slope=0.02, wiggle=0.02 * L, source=src)
        out.append(sc)
    return out


def config4(seed=4, steps=108000):
    """5-level nest of about 47 M cells (synthetic analogue of the paper's Kochi model,
    Table I): 2400x2000 @ 810 m; 3 x 900^2 @ 270; 6 x 900^2 @ 90; 12 x 1200^2 @ 30;
    16 x 1200x900 @ 10 m. Trench 7000 m, land to 50 m, 200 x 80 km uplift of 5 m,
    dt 0.2 s, 6 h = 108,000 steps."""
    return coastal_hierarchy(
        "5-level nest 2400x2000 + 3x900^2 + 6x900^2 + 12x1200^2 + 16x1200x900 (46.65 M cells)",
        seed, (2400, 2000, 810.0),
        [(3, 900, 900), (6, 900, 900), (12, 1200, 1200), (16, 1200, 900)], dt=0.2, steps=steps,
        deep=4000.0, trench=(250e3, 7000.0, 30e3), shelf_w=60e3, slope_w=100e3, land_max=50.0,
        wiggle=8e3, coast_frac=0.8, source=dict(kind="ellipse", a=100e3, b=40e3, peak=5.0),
        land_frac=0.35)


def serving_hierarchy(kind, seed, hours=1.0):
    """Scenario shapes of the serving mix: '3level' (~1.2 M cells), '4level' (~7.95 M),
    '5level' (= config4's shape), each with its own seeded source."""
    if kind == "3level":
        dt = 0.5
        sc = coastal_hierarchy("3-level 800x600 + 600^2 + 600^2", seed, (800, 600, 810.0),
                               [(1, 600, 600), (1, 600, 600)], dt=dt, steps=0, shelf_w=40e3,
                               slope_w=60e3, wiggle=4e3, coast_frac=0.7,
                               source=dict(kind="ellipse", a=50e3, b=25e3, peak=3.0))
    elif kind == "4level":
        dt = 0.2
        sc = coastal_hierarchy("4-level 1200x1000 + 3x600^2 + 3x900^2 + 3x1200x900", seed,
                               (1200, 1000, 810.0), [(3, 600, 600), (3, 900, 900),
                                                     (3, 1200, 900)], dt=dt, steps=0,
                               shelf_w=60e3, slope_w=100e3, wiggle=6e3, coast_frac=0.75,
                               source=dict(kind="ellipse", a=80e3, b=30e3, peak=4.0))
    elif kind == "5level":
        sc = config4(seed=seed, steps=0)
        dt = sc.dt
    else:
        raise ValueError(kind)
    sc.steps = int(round(hours * 3600.0 / dt))
    return sc


def poisson_trace(seed, n=120, mean_s=20.0, kinds=("3level", "4level", "5level"),
                  hours=(1, 6)):
    """Poisson arrivals (mean inter-arrival mean_s), uniform over hierarchy kinds,
    simulated duration uniform over the integer hours in [hours[0], hours[1]]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(mean_s, size=n))
    out = []
    for k in range(n):
        out.append(dict(arrival_s=float(t[k]), kind=str(rng.choice(kinds)),
                        hours=int(rng.integers(hours[0], hours[1] + 1)),
                        seed=int(rng.integers(1 << 30))))
    return out
