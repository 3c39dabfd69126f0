"""Serving: continuous batching over the batch API (C5 pattern).

CPU: the pool allocator behind footprint admission. GPU: a request's results are the
same served alone and served in a mix that overlaps it (bitwise: the per-cell
arithmetic of a scenario does not depend on what else is in the batch), and a pool that
holds one scenario at a time serialises admission without losing a request.
"""
import numpy as np
import pytest

from paper_2408_07609_gb300 import scenarios as S


def test_pool_first_fit_and_coalescing():
    from paper_2408_07609_gb300.serve import Pool

    p = Pool(10 * 256)
    a = p.alloc(300)   # 512 bytes
    b = p.alloc(256)
    c = p.alloc(1000)  # 1024 bytes
    assert (a, b, c) == (0, 512, 768)
    assert p.alloc(1024) is None  # 2560 - 1792 = 768 left
    p.release(b)
    assert p.alloc(200) == 512  # first fit reuses the hole
    p.release(512)
    p.release(a)
    assert p.free[0] == (0, 768)  # a and b coalesced
    p.release(c)
    assert p.free == [(0, 2560)] and p.in_use == 0


def _trace(kinds, arrivals, seeds, hours):
    return [dict(arrival_s=t, kind=k, seed=s, hours=h)
            for t, k, s, h in zip(arrivals, kinds, seeds, hours)]


@pytest.mark.gpu
def test_result_is_the_same_alone_and_in_the_mix(rti):
    from paper_2408_07609_gb300.serve import Server

    sites = {"small": S.coastal_hierarchy(
        "serving test 300x240 + 180^2 + 180^2", 77, (300, 240, 810.0),
        [(1, 180, 180), (1, 180, 180)], dt=0.5, steps=0, shelf_w=20e3, slope_w=30e3,
        wiggle=2e3, coast_frac=0.7, source=dict(kind="ellipse", a=30e3, b=15e3, peak=3.0))}
    # durations of 240, 300 and 180 steps; one admission per 40-step chunk, so the second
    # and third requests join while the first is in flight
    trace = _trace(["small"] * 3, [0.0, 0.0, 0.0], [5, 6, 7],
                   [240 * 0.5 / 3600, 300 * 0.5 / 3600, 180 * 0.5 / 3600])
    srv = Server(sites, pool_bytes=1 << 30, precision=rti.FP32, chunk_steps=40, keep_fields=True)
    reqs, stats = srv.run(trace, admit_per_chunk=1)
    srv.close()
    assert stats["completed"] == 3 and stats["max_live"] == 3
    assert reqs[0].admitted_s < reqs[1].admitted_s < reqs[2].admitted_s
    for r in reqs:
        sc = S.with_new_source(sites["small"], r.seed)
        h = rti.Handle.from_scenario(sc, precision=rti.FP32)
        h.step(r.nsteps)
        h.sync()
        for k in range(len(sc.blocks)):
            mh, at = r.result[k]
            assert np.array_equal(np.isnan(mh), np.isnan(h.max_height(k)))
            assert np.array_equal(mh[~np.isnan(mh)], h.max_height(k)[~np.isnan(mh)]), (r.rid, k)
            assert np.array_equal(at, h.arrival_time(k)), (r.rid, k)
        assert np.nanmax(r.result[0][0]) > 0.1  # the source made a wave
        h.close()


@pytest.mark.gpu
def test_admission_by_footprint_serialises_when_the_pool_holds_one(rti):
    from paper_2408_07609_gb300.serve import Server

    sites = {"c1": S.coastal_hierarchy("serving test 200x160", 3, (200, 160, 1000.0), [],
                                       dt=1.0, steps=0, shelf_w=30e3, slope_w=40e3,
                                       source=dict(kind="gauss", sigma=10e3, peak=2.0))}
    p = rti.make_params(1.0, precision=rti.FP32)
    fp = rti.footprint(sites["c1"].blocks, p)
    trace = _trace(["c1"] * 4, [0.0, 0.0, 0.0, 0.0], [1, 2, 3, 4], [100 / 3600] * 4)
    srv = Server(sites, pool_bytes=fp + fp // 2, precision=rti.FP32, chunk_steps=25)
    reqs, stats = srv.run(trace)
    srv.close()
    assert stats["completed"] == 4 and stats["max_live"] == 1
    done = sorted(reqs, key=lambda r: r.done_s)
    assert [r.rid for r in done] == [0, 1, 2, 3]  # admitted in arrival order
    assert all(r.admitted_s >= prev.done_s for prev, r in zip(done, done[1:]))


@pytest.mark.gpu
def test_fp64_audit_sample_checks_the_fp32_forecasts(rti, oracle_mod):
    """audit_every=2 reruns requests 0 and 2 in binary64 after the trace. The audit's
    binary64 run is itself the oracle's result (to 1e-12), and the binary32 forecasts it
    checks stay within the forecast bounds (max height 5 cm)."""
    from paper_2408_07609_gb300.serve import Server

    sites = {"c1": S.coastal_hierarchy("serving audit 120x96", 4, (120, 96, 1000.0), [],
                                       dt=1.0, steps=0, shelf_w=20e3, slope_w=30e3,
                                       source=dict(kind="gauss", sigma=8e3, peak=2.0))}
    trace = _trace(["c1"] * 3, [0.0, 0.0, 0.0], [11, 12, 13], [150 / 3600] * 3)
    srv = Server(sites, pool_bytes=1 << 28, precision=rti.FP32, chunk_steps=50, audit_every=2)
    reqs, stats = srv.run(trace)
    srv.close()
    a = stats["audit"]
    assert a["requests"] == 2 and [bool(r.audit) for r in reqs] == [True, False, True]
    assert 0 < a["max_height_err_m"] <= 0.05
    # the audit compares against the binary64 path: recompute request 2's error here
    r = reqs[2]
    sc = S.with_new_source(sites["c1"], r.seed)
    o = oracle_mod.from_scenario(sc)
    o.step(r.nsteps)
    h = rti.Handle.from_scenario(sc, precision=rti.FP32)
    h.step(r.nsteps)
    g, ref = h.max_height(0), o.max_height(0)
    both = ~np.isnan(g) & ~np.isnan(ref)
    assert abs(np.abs(g[both] - ref[both]).max() - r.audit["max_height_err_m"]) <= 1e-9
    h.close()
