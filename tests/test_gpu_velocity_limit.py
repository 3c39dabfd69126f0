"""The optional velocity limit (R12) on the CUDA path against the oracle: the draining
puddle where it binds on every front face (both precisions), and the 3-level nest with a
limit that binds at its fronts (binary64 to the parity bar, binary32 within the forecast
bounds)."""
import os
import sys

import numpy as np
import pytest

from paper_2408_07609_gb300 import scenarios as S

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from parity import TOL64, check_fp32, compare_fp64, fp32_metrics, relerr  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_velocity_limit_puddle_matches_oracle(rti, oracle_mod, precision):
    nx = ny = 5
    blk = dict(level=1, parent=-1, nx=nx, ny=ny, i0=0, j0=0, dx=1.0, bc=(0, 0, 0, 0))
    hh = np.full((ny, nx), -1.0)
    nn = np.zeros((ny, nx), np.float32)
    eta = np.full((ny, nx), 1.0)
    eta[2, 2] = 1.1
    h = rti.Handle([blk], [hh], [nn], dt=1.0, precision=precision, velocity_limit=0.1)
    h.set_state(0, eta=eta)
    o = oracle_mod.Oracle([blk], [hh], [nn], dt=1.0, vel_limit=0.1)
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


def test_velocity_limit_three_level_nest(rti, oracle_mod):
    """A 3-level nest whose source sits next to its coast (the oracle pin's hierarchy), with
    a limit of 0.5 m/s that binds where the wave runs up: binary64 against the oracle with
    the same limit, binary32 within the forecast bounds, and the limited run differs from
    the unlimited one. In a batch beside an unlimited member, each equals itself alone."""
    sc = S.coastal_hierarchy("vl", 5, (60, 54, 810.0), [(1, 36, 36), (1, 27, 27)], dt=0.5,
                             steps=1500, shelf_w=8e3, slope_w=10e3, wiggle=1e3, coast_frac=0.6,
                             land_frac=0.4, source=dict(kind="gauss", sigma=4e3, peak=2.0))
    o = oracle_mod.from_scenario(sc, vel_limit=0.5)
    h = rti.Handle.from_scenario(sc, precision=rti.FP64, velocity_limit=0.5)
    h.step(sc.steps)
    o.step(sc.steps)
    compare_fp64(h, o, len(sc.blocks))
    ref = rti.Handle.from_scenario(sc, precision=rti.FP64)
    ref.step(sc.steps)
    assert any(not np.array_equal(h.get_state(k)[1], ref.get_state(k)[1]) for k in range(3))
    h32 = rti.Handle.from_scenario(sc, precision=rti.FP32, velocity_limit=0.5)
    h32.step(sc.steps)
    check_fp32(fp32_metrics(h32, o, sc), sc.dt)
    # one batch: the limited member and an unlimited one, each as alone
    b = rti.Batch(precision=rti.FP64, chunk_steps=500)
    m1 = rti.Handle.from_scenario(sc, precision=rti.FP64, velocity_limit=0.5)
    m2 = rti.Handle.from_scenario(sc, precision=rti.FP64)
    b.add(m1, sc.steps)
    b.add(m2, sc.steps)
    for _ in range(3):
        b.step()
    b.sync()
    for k in range(len(sc.blocks)):
        for x, y in zip(m1.get_state(k), h.get_state(k)):
            assert np.array_equal(x, y)
        for x, y in zip(m2.get_state(k), ref.get_state(k)):
            assert np.array_equal(x, y)
    b.close()
    for x in (h, ref, h32, o, m1, m2):
        x.close()
