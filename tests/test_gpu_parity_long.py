"""GPU parity at the run lengths of the workloads (Sec. V-A, Table I shape): the 3-level
nest over its full hour, every grid of the 64-grid batch over 2000 steps, and the
46.65 M-cell 5-level hierarchy over 500 steps, each in binary64 against the oracle
(1e-12, element by element, with the outputs and budgets) and in binary32 against the
forecast bounds. The oracle runs in its OpenMP build (bitwise equal to the plain build,
tests/test_oracle_openmp.py) or, for the batch, one plain oracle per grid on a thread
each (ctypes releases the interpreter lock during the C call).
"""
import concurrent.futures as cf
import os
import sys

import numpy as np
import pytest

from paper_2408_07609_gb300 import scenarios as S

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from parity import check_fp32, compare_fp64, fp32_metrics  # noqa: E402

pytestmark = pytest.mark.gpu


def test_three_level_nest_full_hour(rti, oracle_mod):
    """C2: 600^2 / 450^2 / 450^2 at 810 / 270 / 90 m, dt 0.5 s, 7200 steps (1 h), in
    binary64. Every operation of the step on both sides is an IEEE-rounded +, -, *, /,
    sqrt or the same stated cube-root iteration, in the same order, so the states agree
    bit for bit after the full hour (the budgets, summed in another order, to 1e-12).
    The binary32 path over the same hour is in test_fp32_accuracy."""
    sc = S.config2()
    o = oracle_mod.from_scenario(sc, parallel=True)
    h64 = rti.Handle.from_scenario(sc, precision=rti.FP64)
    h64.step(sc.steps)
    o.step(sc.steps)
    compare_fp64(h64, o, len(sc.blocks))
    for k in range(len(sc.blocks)):
        for a, b in zip(h64.get_state(k), o.get_state(k)):
            assert np.array_equal(a, b), k
    assert o.budget(0)["ring"] != 0.0 and o.budget(2)["clip"] >= 0.0
    arrived = sum(int((o.arrival_time(k) >= 0).sum()) for k in range(3))
    assert arrived > 100000
    h64.close()
    o.close()


def _oracle_run(oracle_mod, sc):
    o = oracle_mod.from_scenario(sc)
    o.step(sc.steps)
    return o


def test_batch_all_64_grids_2000_steps(rti, oracle_mod):
    """C3: all 64 grids (sides 128-1024, 15.9 M cells) stepped together by one batch in
    each precision for their 2000 steps; every grid against its own oracle run."""
    grids = S.config3()
    assert len(grids) == 64 and all(g.steps == 2000 for g in grids)
    with cf.ThreadPoolExecutor(max_workers=oracle_mod.threads()) as ex:
        futs = [ex.submit(_oracle_run, oracle_mod, sc) for sc in grids]
        handles = {}
        for prec in (rti.FP64, rti.FP32):
            b = rti.Batch(precision=prec, chunk_steps=500)
            hs = [rti.Handle.from_scenario(sc, precision=prec) for sc in grids]
            for h, sc in zip(hs, grids):
                b.add(h, sc.steps)
            while any(b.remaining(h) > 0 for h in hs):
                b.step()
            b.sync()
            handles[prec] = (b, hs)
        oracles = [f.result() for f in futs]
    for sc, o, h64, h32 in zip(grids, oracles, handles[rti.FP64][1], handles[rti.FP32][1]):
        assert h64.steps_done == h32.steps_done == sc.steps
        compare_fp64(h64, o, 1)
        check_fp32(fp32_metrics(h32, o, sc), sc.dt)
        o.close()
    for b, hs in handles.values():
        b.close()
        for h in hs:
            h.close()


def test_five_level_500_steps(rti, oracle_mod):
    """C4: the 46.65 M-cell hierarchy in the benchmark's launch configuration, 500 steps
    (100 s), every cell of every block, both precisions."""
    sc = S.config4(steps=500)
    o = oracle_mod.from_scenario(sc, parallel=True)
    h64 = rti.Handle.from_scenario(sc, precision=rti.FP64)
    h64.step(sc.steps)
    o.step(sc.steps)
    compare_fp64(h64, o, len(sc.blocks))
    h64.close()
    h32 = rti.Handle.from_scenario(sc, precision=rti.FP32)
    h32.step(sc.steps)
    check_fp32(fp32_metrics(h32, o, sc), sc.dt)
    h32.close()
    o.close()
