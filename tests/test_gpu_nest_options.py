"""Nesting options on the CUDA path: full two-way fine-to-coarse feedback (every covered
parent cell takes the child mean) and piecewise-constant coarse-to-fine edge flux.

Binary64 against the oracle run with the same options (<= 1e-12, as every binary64
parity test), with strips of 28 x 64 and 28 x 8 cells (the smaller ones lie wholly
inside a child footprint, so the feedback covers strips that meet no ring), under both
schedules; binary32 within the forecast bounds; the lake at rest bitwise; and handles
with different options stepped together in one batch, each equal to itself alone.
"""
import os
import sys

import numpy as np
import pytest

from paper_2408_07609_gb300 import scenarios as S

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from parity import compare_fp64, relerr  # noqa: E402

pytestmark = pytest.mark.gpu
OPTIONS = [(1, 0), (0, 1), (1, 1)]  # (nest_feedback, nest_flux); (0, 0) is the default


def wide_nest(steps=300):
    """3 levels, 200 x 120 @ 810 m root, a 216 x 135 child (72 x 45 parent cells) and a
    135 x 90 grandchild; eight 28 x 8 root strips and two level-2 strips lie inside a
    footprint with their halo. Gaussian source, land, drying."""
    return S.coastal_hierarchy(
        "3-level nest, wide child", 9, (200, 120, 810.0), [(1, 216, 135), (1, 135, 90)],
        dt=0.5, steps=steps, shelf_w=15e3, slope_w=20e3, wiggle=2e3, coast_frac=0.6,
        land_frac=0.4, source=dict(kind="gauss", sigma=8e3, peak=2.0))


@pytest.mark.parametrize("tile", [(0, 0), (28, 8)])
@pytest.mark.parametrize("fb,fl", OPTIONS)
def test_nest_options_fp64(rti, oracle_mod, fb, fl, tile):
    sc = wide_nest()
    h = rti.Handle.from_scenario(sc, precision=rti.FP64, tile=tile, nest_feedback=fb,
                                 nest_flux=fl)
    o = oracle_mod.from_scenario(sc, nest_feedback=fb, nest_flux=fl)
    h.step(sc.steps)
    h.sync()
    o.step(sc.steps)
    compare_fp64(h, o, 3)
    # the option is in effect: the default reading ends elsewhere
    d = oracle_mod.from_scenario(sc)
    d.step(sc.steps)
    assert max(relerr(h.get_state(k)[0], d.get_state(k)[0]) for k in range(2)) > 1e-7
    h.close()


def test_full_feedback_per_step_schedule_fp64(rti, oracle_mod):
    sc = wide_nest(steps=200)
    h = rti.Handle.from_scenario(sc, precision=rti.FP64, schedule=rti.SCHED_PER_PASS,
                                 tile=(28, 8), nest_feedback=rti.NEST_FULL,
                                 nest_flux=rti.FLUX_CONSTANT)
    o = oracle_mod.from_scenario(sc, nest_feedback=1, nest_flux=1)
    h.step(sc.steps)
    h.sync()
    o.step(sc.steps)
    compare_fp64(h, o, 3)
    h.close()


def test_nest_options_fp32_within_forecast_bounds(rti, oracle_mod):
    sc = wide_nest(steps=600)
    h = rti.Handle.from_scenario(sc, precision=rti.FP32, nest_feedback=rti.NEST_FULL,
                                 nest_flux=rti.FLUX_CONSTANT)
    o = oracle_mod.from_scenario(sc, nest_feedback=1, nest_flux=1)
    h.step(sc.steps)
    h.sync()
    o.step(sc.steps)
    for k in range(3):
        assert np.abs(h.get_state(k)[0] - o.get_state(k)[0]).max() <= 0.05
        g, r = h.max_height(k), o.max_height(k)
        both = ~np.isnan(g) & ~np.isnan(r)
        assert np.abs(g[both] - r[both]).max() <= 0.05
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_lake_at_rest_with_options_bitwise(rti, precision):
    sc = S.config2(steps=0)
    sc.uplift = [None] * len(sc.blocks)
    h = rti.Handle.from_scenario(sc, precision=precision, tile=(28, 8),
                                 nest_feedback=rti.NEST_FULL, nest_flux=rti.FLUX_CONSTANT)
    rest = [h.get_state(k)[0] for k in range(3)]
    if precision == 0:
        for k in range(3):
            assert np.array_equal(rest[k], np.where(sc.bathy[k] > 0, 0.0, -sc.bathy[k]))
    h.step(300)
    for k in range(3):
        e, M, N = h.get_state(k)
        assert np.array_equal(e, rest[k])
        assert not M.any() and not N.any()
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_mixes_nesting_options(rti, precision):
    """Handles with different options in one launch: each ends where it ends alone (the
    options are per block, not per launch). Bitwise, except a binary32 handle without full
    feedback: in a batch with full feedback it runs that compiled variant of the step
    kernel, whose binary32 contractions (fused multiply-adds) may round differently in
    the last bit; it stays within 1 mm of itself alone."""
    sc = wide_nest(steps=120)
    opts = [(0, 0), (1, 1), (1, 0)]
    b = rti.Batch(precision=precision, chunk_steps=50)
    hs = []
    for fb, fl in opts:
        h = rti.Handle.from_scenario(sc, precision=precision, nest_feedback=fb, nest_flux=fl)
        b.add(h, sc.steps)
        hs.append(h)
    while any(b.remaining(h) > 0 for h in hs):
        b.step()
    b.sync()
    for (fb, fl), h in zip(opts, hs):
        alone = rti.Handle.from_scenario(sc, precision=precision, nest_feedback=fb,
                                         nest_flux=fl)
        alone.step(sc.steps)
        for k in range(3):
            for a, c in zip(h.get_state(k), alone.get_state(k)):
                if precision == 0 or fb == 1:
                    assert np.array_equal(a, c), (fb, fl, k)
            if precision == 1 and fb == 0:
                d = np.abs(h.get_state(k)[0] - alone.get_state(k)[0]).max()
                assert d <= 1e-3, (fl, k, d)
        alone.close()
    b.close()
