"""Failure detection without a GPU fault.

The bounded device-wide barrier: when its wait runs out, the persistent launch ends
with RTI_ERR_TIMEOUT reported by the next call that waits, the context stays usable, and
the handle, given a new state, steps correctly again. The host watchdog: a wait with a
deadline returns RTI_ERR_TIMEOUT while the work is still running and leaves it alone. A
request removed from a running batch mid-run leaves the others bitwise unchanged.

The wait is made to run out by shortening it (RTI_BARRIER_SPIN_CYCLES, read when a
handle is created) far below the time one strip takes: the CTAs without a strip reach
the first barrier at once and give up after about a microsecond. The same limit bounds
the wait of full feedback's ring strips for their children's strip flags. No kernel
faults, traps or hangs; every CTA leaves by the bounded wait.
"""
import os
import sys

import pytest

from paper_2408_07609_gb300 import scenarios as S

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from parity import compare_fp64  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_barrier_wait_runs_out_and_the_handle_recovers(rti, oracle_mod, monkeypatch, precision):
    sc = S.config1(nx=120, ny=100, steps=12)
    monkeypatch.setenv("RTI_BARRIER_SPIN_CYCLES", "2000")
    h = rti.Handle.from_scenario(sc, precision=precision, schedule=rti.SCHED_PERSISTENT)
    monkeypatch.delenv("RTI_BARRIER_SPIN_CYCLES")
    h.step(sc.steps)  # one cooperative launch of 12 steps: 11 barriers
    with pytest.raises(rti.RtiError) as ei:
        h.sync()
    assert ei.value.code == -6
    h.sync()  # reported once: the condition is cleared
    # a new state, then chunks of one step (no barrier inside a launch)
    h.set_initial_uplift(0, sc.uplift[0])
    for _ in range(sc.steps):
        h.step(1)
    h.sync()
    assert h.steps_done == sc.steps
    o = oracle_mod.from_scenario(sc)
    o.step(sc.steps)
    if precision == 0:
        compare_fp64(h, o, 1)
    else:
        import numpy as np

        assert np.abs(h.get_state(0)[0] - o.get_state(0)[0]).max() <= 1e-4
    h.close()
    # a handle created with the normal wait steps the same chunk through its barriers
    h2 = rti.Handle.from_scenario(sc, precision=precision, schedule=rti.SCHED_PERSISTENT)
    h2.step(sc.steps)
    h2.sync()
    if precision == 0:
        compare_fp64(h2, o, 1)
    h2.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_strip_flag_wait_runs_out(rti, oracle_mod, monkeypatch, precision):
    """Full feedback, one launch per step (no device-wide barrier): a parent's ring strip
    waits for the flags of the child strips under its region. With the wait shortened
    far below a strip's duration it gives up, the launch ends, and the next wait reports
    RTI_ERR_TIMEOUT once; the context stays usable (a handle with the normal wait then
    matches the oracle)."""
    sc = S.coastal_hierarchy(
        "3-level nest, wide child", 9, (200, 120, 810.0), [(1, 216, 135), (1, 135, 90)],
        dt=0.5, steps=3, shelf_w=15e3, slope_w=20e3, wiggle=2e3, coast_frac=0.6,
        land_frac=0.4, source=dict(kind="gauss", sigma=8e3, peak=2.0))
    monkeypatch.setenv("RTI_BARRIER_SPIN_CYCLES", "2000")
    h = rti.Handle.from_scenario(sc, precision=precision, schedule=rti.SCHED_PER_PASS,
                                 nest_feedback=rti.NEST_FULL)
    monkeypatch.delenv("RTI_BARRIER_SPIN_CYCLES")
    h.step(sc.steps)
    with pytest.raises(rti.RtiError) as ei:
        h.sync()
    assert ei.value.code == -6
    h.sync()  # reported once: the condition is cleared
    h.close()
    h2 = rti.Handle.from_scenario(sc, precision=precision, schedule=rti.SCHED_PER_PASS,
                                  nest_feedback=rti.NEST_FULL)
    h2.step(sc.steps)
    h2.sync()
    o = oracle_mod.from_scenario(sc, nest_feedback=1)
    o.step(sc.steps)
    if precision == 0:
        compare_fp64(h2, o, 3)
    h2.close()


def test_host_watchdog_times_out_and_the_work_completes(rti):
    """rti_sync_timeout with a deadline far shorter than the enqueued work returns TIMEOUT
    without disturbing it; a later wait finds the steps done and the state equal to an
    undisturbed run, bitwise."""
    import numpy as np

    sc = S.config2(steps=0)
    h = rti.Handle.from_scenario(sc, precision=rti.FP64)
    h.step(400)  # about 0.4 s of binary64 work
    with pytest.raises(rti.RtiError) as ei:
        h.sync(timeout=0.0)
    assert ei.value.code == -6
    h.sync(timeout=120.0)
    assert h.steps_done == 400
    ref = rti.Handle.from_scenario(sc, precision=rti.FP64)
    ref.step(400)
    ref.sync()
    for k in range(len(sc.blocks)):
        for a, b in zip(h.get_state(k), ref.get_state(k)):
            assert np.array_equal(a, b)
    h.close()
    ref.close()


def test_request_removed_mid_run_leaves_the_others_unchanged(rti):
    """Three grids in one batch; one is removed after the first chunk (as a cancelled
    forecast would be). The other two finish bitwise equal to themselves stepped alone."""
    import numpy as np

    grids = sorted(S.config3(count=64, steps=120), key=lambda g: g.cells)[:3]
    b = rti.Batch(precision=rti.FP32, chunk_steps=40)
    hs = [rti.Handle.from_scenario(sc, precision=rti.FP32) for sc in grids]
    for h, sc in zip(hs, grids):
        b.add(h, sc.steps)
    b.step()
    b.sync(timeout=60.0)
    b.remove(hs[1])
    while any(b.remaining(h) > 0 for h in (hs[0], hs[2])):
        b.step()
    b.sync()
    for k in (0, 2):
        alone = rti.Handle.from_scenario(grids[k], precision=rti.FP32)
        alone.step(grids[k].steps)
        for a, c in zip(hs[k].get_state(0), alone.get_state(0)):
            assert np.array_equal(a, c)
        alone.close()
    assert hs[1].steps_done == 40
    b.close()
    for h in hs:
        h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_is_bitwise(rti, precision):
    """Checkpoint after 150 steps, resume in a fresh handle, step 150 more: every state
    value, output and budget term equals the uninterrupted 300-step run, bitwise."""
    import numpy as np

    sc = S.config2(steps=0)
    a = rti.Handle.from_scenario(sc, precision=precision, track_velocity=True)
    a.step(150)
    ck = a.checkpoint()
    a.step(150)
    b = rti.Handle.from_scenario(sc, precision=precision, track_velocity=True)
    b.restore(ck)
    assert b.steps_done == 150
    b.step(150)
    assert b.steps_done == a.steps_done == 300
    for k in range(len(sc.blocks)):
        for x, y in zip(a.get_state(k), b.get_state(k)):
            assert np.array_equal(x, y)
        for f in ("max_height", "arrival_time", "max_velocity"):
            assert np.array_equal(getattr(a, f)(k), getattr(b, f)(k), equal_nan=True), f
        assert a.budget(k) == b.budget(k)
    c = rti.Handle.from_scenario(sc, precision=1 - precision, track_velocity=True)
    with pytest.raises(rti.RtiError):
        c.restore(ck)  # another precision: refused
    for h in (a, b, c):
        h.close()
