"""The bounded device-wide barrier: when its wait runs out, the persistent launch ends
with RTI_ERR_TIMEOUT reported by the next call that waits, the context stays usable, and
the handle, given a new state, steps correctly again.

The wait is made to run out by shortening it (RTI_BARRIER_SPIN_CYCLES, read when a
handle is created) far below the time one strip takes: the CTAs without a strip reach
the first barrier at once and give up after about a microsecond. No kernel faults,
traps or hangs; every CTA leaves by the bounded wait.
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
