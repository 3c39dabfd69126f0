"""CUDA path vs the FP64 oracle, element by element, on seeded synthetic inputs.

Binary64 bar: max|gpu - oracle| / max|oracle| <= 1e-12 per field and block (the
kernels perform the oracle's operations in its order, the cube root included, so the
states agree bit for bit; the bar leaves room for the budget sums' order).
Binary32 bar: the accuracy stated for the forecast outputs (max |d eta| in metres,
wet/dry mismatch, arrival error); see test_fp32_accuracy_report.
"""
import os
import sys

import numpy as np
import pytest

from paper_2408_07609_gb300 import scenarios as S

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from parity import TOL64, compare_fp64, relerr  # noqa: E402

pytestmark = pytest.mark.gpu


def run_pair(rti, oracle_mod, sc, steps, precision=0, schedule=0, tile=(0, 0)):
    h = rti.Handle.from_scenario(sc, precision=precision, schedule=schedule, tile=tile)
    o = oracle_mod.from_scenario(sc)
    h.step(steps)
    h.sync()
    o.step(steps)
    return h, o


def test_single_grid_fp64_full_run(rti, oracle_mod):
    """256 x 256, dx 1000 m, 1800 steps: radiation west, coast east (wet/dry), friction."""
    sc = S.config1()
    h, o = run_pair(rti, oracle_mod, sc, sc.steps)
    assert h.steps_done == sc.steps
    compare_fp64(h, o, 1)
    assert (o.arrival_time(0) > 0).sum() > 1000


def test_ragged_single_grid_fp64(rti, oracle_mod):
    """Sizes that are not multiples of the tile, several tiles, both schedules."""
    sc = S.config1(nx=203, ny=157, steps=400)
    for sched in (0, 1):
        h, o = run_pair(rti, oracle_mod, sc, sc.steps, schedule=sched)
        compare_fp64(h, o, 1)


@pytest.mark.parametrize("tile", [(28, 8), (28, 16), (28, 64)])
def test_tile_shapes_bitwise_equal(rti, oracle_mod, tile):
    sc = S.config1(nx=150, ny=90, steps=200)
    h, o = run_pair(rti, oracle_mod, sc, sc.steps, tile=tile)
    compare_fp64(h, o, 1)


def test_three_level_nest_fp64(rti, oracle_mod):
    """600^2 / 450^2 / 450^2 at 810 / 270 / 90 m: the coarse-to-fine pull, the
    fine-to-coarse ring recompute and wet/dry on a fractal coast."""
    sc = S.config2(steps=300)
    h, o = run_pair(rti, oracle_mod, sc, sc.steps)
    compare_fp64(h, o, 3)
    assert o.budget(0)["ring"] != 0.0


def test_lake_at_rest_gpu_bitwise(rti):
    sc = S.config2(steps=0)
    sc.uplift = [None] * len(sc.blocks)
    h = rti.Handle.from_scenario(sc)
    h.step(500)
    for k in range(3):
        e, M, N = h.get_state(k)
        assert np.array_equal(e, np.where(sc.bathy[k] > 0, 0.0, -sc.bathy[k]))
        assert not M.any() and not N.any()


def test_batch_of_grids_fp64_matches_oracle_and_alone(rti, oracle_mod):
    """Grids of different sizes and dt stepped together in one persistent launch:
    each equals the oracle, and equals the same grid stepped alone, bitwise."""
    grids = S.config3(count=64, steps=120)
    pick = sorted(grids, key=lambda s: s.cells)[:6]
    b = rti.Batch(precision=0, chunk_steps=40)
    hs = []
    for sc in pick:
        h = rti.Handle.from_scenario(sc)
        b.add(h, sc.steps)
        hs.append(h)
    while any(b.remaining(h) > 0 for h in hs):
        b.step()
    b.sync()
    for sc, h in zip(pick, hs):
        o = oracle_mod.from_scenario(sc)
        o.step(sc.steps)
        assert h.steps_done == sc.steps
        compare_fp64(h, o, 1)
        alone = rti.Handle.from_scenario(sc)
        alone.step(sc.steps)
        for a, c in zip(h.get_state(0), alone.get_state(0)):
            assert np.array_equal(a, c)
    b.close()


def test_members_with_different_lengths_stop_on_their_own(rti):
    grids = S.config3(count=64, steps=10)
    pick = sorted(grids, key=lambda s: s.cells)[:3]
    b = rti.Batch(precision=1, chunk_steps=7)
    hs = [rti.Handle.from_scenario(sc, precision=1) for sc in pick]
    for h, n in zip(hs, (5, 13, 21)):
        b.add(h, n)
    for _ in range(3):
        b.step()
    b.sync()
    assert [h.steps_done for h in hs] == [5, 13, 21]
    assert [b.remaining(h) for h in hs] == [0, 0, 0]


def test_full_size_five_level_fp64_one_step(rti, oracle_mod):
    """The 46.65 M-cell 5-level hierarchy in the benchmark's launch configuration,
    two steps, every cell of every block against the oracle."""
    sc = S.config4(steps=2)
    h, o = run_pair(rti, oracle_mod, sc, 2)
    compare_fp64(h, o, len(sc.blocks), outputs=False)


def test_nonfinite_level_is_reported(rti):
    sc = S.config1(nx=64, ny=64, steps=1)
    h = rti.Handle.from_scenario(sc)
    e, M, N = h.get_state(0)
    e[10, 10] = np.nan
    h.set_state(0, eta=e)
    h.step(2)
    with pytest.raises(rti.RtiError) as ei:
        h.sync()
    assert ei.value.code == -5


def test_fp32_accuracy_report(rti, oracle_mod):
    """Binary32 path vs the FP64 oracle on the single grid (1800 steps): max |d eta|,
    max |d max-eta|, wet/dry mismatch and arrival error within the stated accuracy."""
    sc = S.config1()
    h, o = run_pair(rti, oracle_mod, sc, sc.steps, precision=1)
    ge, oe = h.get_state(0)[0], o.get_state(0)[0]
    assert np.abs(ge - oe).max() <= 0.01
    gm, om = h.max_height(0), o.max_height(0)
    both = ~np.isnan(gm) & ~np.isnan(om)
    assert np.abs(gm[both] - om[both]).max() <= 0.05
    ever_g, ever_o = ~np.isnan(gm), ~np.isnan(om)
    assert (ever_g ^ ever_o).sum() <= 0.005 * (ever_g | ever_o).sum()
    ga, oa = h.arrival_time(0), o.arrival_time(0)
    m = (ga >= 0) & (oa >= 0)
    assert np.percentile(np.abs(ga[m] - oa[m]), 99) <= 5.0


def _small_nest(levels):
    return S.coastal_hierarchy("small nest", 7, (90, 72, 810.0), levels, dt=0.5, steps=60,
                               shelf_w=10e3, slope_w=15e3, wiggle=1e3, coast_frac=0.6,
                               land_frac=0.4, source=dict(kind="gauss", sigma=6e3, peak=2.0))


def test_mixed_schedules_and_precisions_in_one_process(rti):
    """Handles of both precisions and both schedules created and stepped one after the
    other in one process (a sequence that once faulted on the second handle) all run,
    and the two binary64 schedules agree bitwise."""
    out = {}
    keep = []
    for levels in ([(1, 54, 54)], [(1, 54, 54), (1, 45, 45)]):
        sc = _small_nest(levels)
        for prec, sched in ((0, 0), (0, 1), (1, 0), (1, 1), (0, 0), (0, 1)):
            h = rti.Handle.from_scenario(sc, precision=prec, schedule=sched)
            keep.append(h)
            h.step(5)
            h.sync()
            out[(len(levels), prec, sched)] = [h.get_state(k) for k in range(len(sc.blocks))]
    for nl in (1, 2):
        for a, b in zip(out[(nl, 0, 0)], out[(nl, 0, 1)]):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)


def test_never_wet_cells_report_nan_height_in_both_precisions(rti, oracle_mod):
    """Cells that were never wet report max height NaN and max depth 0, whatever the
    state precision (the binary32 never-wet marker is a rounded -1e30)."""
    sc = S.config1(nx=64, ny=40, steps=20)
    sc.bathy[0][:, -12:] = -5.0  # a strip of dry land the wave cannot reach
    o = oracle_mod.from_scenario(sc)
    o.step(sc.steps)
    never = np.isnan(o.max_height(0))
    assert never.sum() >= 12 * 40
    for prec in (0, 1):
        h = rti.Handle.from_scenario(sc, precision=prec)
        h.step(sc.steps)
        assert np.array_equal(np.isnan(h.max_height(0)), never)
        assert np.all(h.max_depth(0)[never] == 0.0)


def _grid_scenario(name, blocks, dt, steps, seed=0):
    """Flat 50 m sea with a land corner (wet/dry) on every block and a seeded Gaussian
    bump on the root; block coordinates follow the 1:3 nesting."""
    rng = np.random.default_rng(seed)
    bathy, manning, uplift, origin = [], [], [], []
    for k, b in enumerate(blocks):
        if b["parent"] < 0:
            x0 = y0 = 0.0
        else:
            P, (px, py) = blocks[b["parent"]], origin[b["parent"]]
            x0, y0 = px + b["i0"] * P["dx"], py + b["j0"] * P["dx"]
        origin.append((x0, y0))
        x = x0 + (np.arange(b["nx"]) + 0.5) * b["dx"]
        y = y0 + (np.arange(b["ny"]) + 0.5) * b["dx"]
        X, Y = np.meshgrid(x, y)
        h = np.full((b["ny"], b["nx"]), 50.0) + rng.uniform(-1, 1, (b["ny"], b["nx"]))
        land = (X > x0 + 0.8 * b["nx"] * b["dx"]) & (Y > y0 + 0.8 * b["ny"] * b["dx"])
        h[land] = -2.0
        bathy.append(h)
        manning.append(np.where(h > 0, 0.025, 0.04).astype(np.float32))
        uplift.append(None)
    R = blocks[0]
    Lx, Ly = R["nx"] * R["dx"], R["ny"] * R["dx"]
    xr = (np.arange(R["nx"]) + 0.5) * R["dx"]
    yr = (np.arange(R["ny"]) + 0.5) * R["dx"]
    Xr, Yr = np.meshgrid(xr, yr)
    sig = max(R["dx"], 0.15 * min(Lx, Ly))
    uplift[0] = 1.5 * np.exp(-((Xr - 0.4 * Lx) ** 2 + (Yr - 0.45 * Ly) ** 2) / (2 * sig**2))
    return S.Scenario(name=name, blocks=blocks, bathy=bathy, manning=manning, uplift=uplift,
                      dt=dt, steps=steps)


def _root(nx, ny, dx=100.0, bc=(1, 1, 1, 1)):
    return dict(level=1, parent=-1, nx=nx, ny=ny, i0=0, j0=0, dx=dx, bc=bc)


@pytest.mark.parametrize("shape", [(3, 3), (5, 300), (300, 5), (28, 64), (29, 65), (57, 3)])
def test_degenerate_single_grids_fp64(rti, oracle_mod, shape):
    """Grids of the minimum size, thinner than a strip, exactly one strip, and one cell
    past it: every strip is an edge strip and halo lanes fall outside the block."""
    nx, ny = shape
    sc = _grid_scenario(f"grid {nx}x{ny}", [_root(nx, ny)], dt=1.0, steps=150, seed=nx * ny)
    for sched in (0, 1):
        h, o = run_pair(rti, oracle_mod, sc, sc.steps, schedule=sched)
        compare_fp64(h, o, 1)
        h.close()
        o.close()


def test_smallest_children_fp64(rti, oracle_mod):
    """A child of 3 x 3 cells (one parent cell, whose ring is itself), a 6 x 9 child and a
    grandchild of 3 x 3 inside it, each at the 3-cell margin of its parent."""
    blocks = [_root(40, 36, dx=300.0),
              dict(level=2, parent=0, nx=3, ny=3, i0=3, j0=3, dx=100.0, bc=(0, 0, 0, 0)),
              dict(level=2, parent=0, nx=15, ny=18, i0=30, j0=27, dx=100.0, bc=(0, 0, 0, 0)),
              dict(level=3, parent=2, nx=3, ny=3, i0=3, j0=3, dx=100.0 / 3, bc=(0, 0, 0, 0))]
    sc = _grid_scenario("smallest children", blocks, dt=0.5, steps=200, seed=7)
    h, o = run_pair(rti, oracle_mod, sc, sc.steps)
    compare_fp64(h, o, len(blocks))
    assert max(abs(o.budget(k)["ring"]) for k in range(2)) > 0


def test_max_velocity_fp64_single_grid_and_nest(rti, oracle_mod):
    """R11: the running maximum of the cell-centre speed, on a single grid with a coast
    and on the three-level nest (child edges pulled from the parent), against the
    oracle; a handle created without tracking refuses the read."""
    for sc in (S.config1(steps=300), S.config2(steps=200)):
        h = rti.Handle.from_scenario(sc, precision=rti.FP64, track_velocity=True)
        o = oracle_mod.from_scenario(sc)
        h.step(sc.steps)
        h.sync()
        o.step(sc.steps)
        for k in range(len(sc.blocks)):
            g, r = h.max_velocity(k), o.max_velocity(k)
            assert relerr(g, r) <= TOL64, (sc.name, k, relerr(g, r))
            assert r.max() > 0 or k > 0
        compare_fp64(h, o, len(sc.blocks))
        h.close()
        o.close()
    h = rti.Handle.from_scenario(S.config1(nx=40, ny=40, steps=0), precision=rti.FP64)
    with pytest.raises(rti.RtiError) as e:
        h.max_velocity(0)
    assert e.value.code == -8


def test_domain_volume_budget_closes(rti, oracle_mod):
    """rti_volume: the root level's budget of the whole domain. It equals the oracle's
    root budget and closes: V(t) = V(0) - boundary outflow + clip + feedback."""
    sc = _small_nest([(1, 54, 54), (1, 45, 45)])
    h = rti.Handle.from_scenario(sc, precision=rti.FP64)
    v0 = h.volume()
    assert v0["outflow"] == 0 and v0["clip"] == 0 and v0["feedback"] == 0
    o = oracle_mod.from_scenario(sc)
    h.step(200)
    o.step(200)
    v = h.volume()
    ob = o.budget(0)
    assert abs(v["volume"] - ob["volume"]) <= 1e-12 * abs(ob["volume"])
    for key, okey in (("outflow", "outflow"), ("clip", "clip"), ("feedback", "ring")):
        assert abs(v[key] - ob[okey]) <= 1e-9 * max(1.0, abs(ob[okey])), key
    assert v["outflow"] != 0 and v["feedback"] != 0
    assert abs(v["volume"] - (v0["volume"] - v["outflow"] + v["clip"] + v["feedback"])) \
        <= 1e-12 * v0["volume"]
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_outflow_limit_puddle_matches_oracle(rti, oracle_mod, precision):
    """The front's outflow limit on a draining 0.1 m puddle over flat land (the oracle
    pin's case): binary64 to 1e-12, binary32 to 1e-6 m, after the limited step and the
    one that empties the puddle."""
    nx = ny = 5
    blk = dict(level=1, parent=-1, nx=nx, ny=ny, i0=0, j0=0, dx=1.0, bc=(0, 0, 0, 0))
    hh = np.full((ny, nx), -1.0)
    nn = np.zeros((ny, nx), np.float32)
    eta = np.full((ny, nx), 1.0)
    eta[2, 2] = 1.1
    h = rti.Handle([blk], [hh], [nn], dt=1.0, precision=precision)
    h.set_state(0, eta=eta)
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=1.0)
    o.set_state(0, eta=eta)
    for _ in range(2):
        h.step(1)
        o.step(1)
        for a, b in zip(h.get_state(0), o.get_state(0)):
            if precision == 0:
                assert relerr(a, b) <= TOL64
            else:
                assert np.abs(a - b).max() <= 1e-6
    h.close()


def test_full_size_five_level_fp32_two_steps(rti, oracle_mod):
    """The benchmark's own configuration (binary32, persistent launch, 28 x 64 strips)
    on the 46.65 M-cell hierarchy, two steps, every cell of every block against the
    oracle: levels within 1e-4 m and fluxes within 1e-4 of the block's largest flux
    (binary32 rounding of a 5 m, 7 km-deep wave)."""
    sc = S.config4(steps=2)
    h, o = run_pair(rti, oracle_mod, sc, 2, precision=rti.FP32)
    for k in range(len(sc.blocks)):
        ge, gM, gN = h.get_state(k)
        oe, oM, oN = o.get_state(k)
        assert np.abs(ge - oe).max() <= 1e-4, k
        for a, b in ((gM, oM), (gN, oN)):
            assert np.abs(a - b).max() <= 1e-4 * max(np.abs(b).max(), 1e-3), k
    h.close()
