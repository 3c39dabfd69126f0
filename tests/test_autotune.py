"""The autotuner's host logic (CPU) and one tuning run on the GPU."""
import json

import numpy as np
import pytest

from paper_2408_07609_gb300 import scenarios as S


def test_strip_count_and_cost_model_fit():
    from paper_2408_07609_gb300 import autotune as A

    blocks = [dict(level=1, parent=-1, nx=100, ny=130), dict(level=2, parent=0, nx=30, ny=27)]
    # 100 columns -> 4 strips of 28 across; 130 rows -> 3 of 64; the child 2 x 1
    assert A.strips(blocks, 64) == 4 * 3 + 2 * 1
    assert A.strips(blocks, 32) == 4 * 5 + 2 * 1
    cells = 100 * 130 + 30 * 27
    alpha, beta = 2e-9, 3e-6  # ms per cell update, ms per strip
    trials = [{"strips": A.strips(blocks, ty), "ms_per_step": alpha * cells + beta * A.strips(blocks, ty)}
              for ty in (32, 64, 128)]
    m = A.fit_cost_model(trials, cells)
    assert np.isclose(m["alpha_ns_per_cell"], alpha * 1e6, rtol=1e-9)
    assert np.isclose(m["beta_us_per_strip"], beta * 1e3, rtol=1e-9)
    assert A.fit_cost_model(trials[:1], cells) is None


def test_cache_round_trip(tmp_path, monkeypatch):
    from paper_2408_07609_gb300 import autotune as A

    path = str(tmp_path / "tune.json")
    c = A._load(path)
    c["k"] = {"tile_y": 96}
    A._save(path, c)
    A._memo.clear()
    assert A._load(path)["k"]["tile_y"] == 96
    assert json.load(open(path)) == {"k": {"tile_y": 96}}


@pytest.mark.gpu
def test_tuned_shape_is_a_candidate_and_results_do_not_depend_on_it(rti, tmp_path):
    from paper_2408_07609_gb300 import autotune as A

    sc = S.config1(nx=150, ny=120, steps=30)
    path = str(tmp_path / "tune.json")
    r = A.tune_handle(sc, precision=rti.FP64, steps=(3, 6), cache_path=path, tile_y=(32, 64),
                      ctas=(0, 2), schedules=(rti.SCHED_PERSISTENT,))
    assert not r["cached"] and r["tile_y"] in (32, 64) and r["ctas_per_sm"] in (0, 2)
    assert len(r["trials"]) == 4
    assert A.tune_handle(sc, precision=rti.FP64, cache_path=path)["cached"]
    ref = rti.Handle.from_scenario(sc, precision=rti.FP64)
    ref.step(sc.steps)
    h = rti.Handle.from_scenario(sc, precision=rti.FP64, tile=(0, r["tile_y"]),
                                 ctas_per_sm=r["ctas_per_sm"], schedule=r["schedule"])
    h.step(sc.steps)
    for a, b in zip(ref.get_state(0), h.get_state(0)):
        assert np.array_equal(a, b)
    b = A.tune_batch(sorted(S.config3(count=64, steps=10), key=lambda g: g.cells)[:3],
                     precision=rti.FP32, chunk_steps=(5, 10), tile_y=(32, 64), ctas=(0,),
                     rounds=1)
    assert b["tile_y"] in (32, 64) and b["chunk_steps"] in (5, 10) and b["gcups"] > 0
