"""The OpenMP build of the oracle gives the same bits as the single-threaded build (no
GPU). The long GPU parity runs use the OpenMP build, so this is what lets them stand in
for the plain oracle."""
import numpy as np
import pytest


def _nest(S):
    return S.coastal_hierarchy("omp", 5, (60, 54, 810.0), [(1, 36, 36), (1, 27, 27)], dt=0.5,
                               steps=0, shelf_w=8e3, slope_w=10e3, wiggle=1e3, coast_frac=0.6,
                               land_frac=0.4, source=dict(kind="gauss", sigma=4e3, peak=3.0))


@pytest.mark.parametrize("fb", [0, 1])
def test_openmp_build_is_bitwise_equal(oracle_mod, fb, monkeypatch):
    from paper_2408_07609_gb300 import scenarios as S

    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    sc = _nest(S)
    runs = [oracle_mod.from_scenario(sc, parallel=par, nest_feedback=fb) for par in (False, True)]
    for o in runs:
        o.step(400)
    a, b = runs
    clipped = 0.0
    for k in range(len(sc.blocks)):
        for x, y in zip(a.get_state(k), b.get_state(k)):
            assert np.array_equal(x, y)
        for f in ("max_height", "max_depth", "arrival_time", "max_velocity"):
            assert np.array_equal(getattr(a, f)(k), getattr(b, f)(k), equal_nan=True), f
        assert a.budget(k) == b.budget(k)
        clipped += a.budget(k)["clip"]
    assert a.budget(0)["outflow"] != 0 and a.budget(0)["ring"] != 0
