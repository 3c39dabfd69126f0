"""The synthetic workloads have the shapes of the paper's (host-only checks)."""
import json
import os

import numpy as np

from paper_2408_07609_gb300 import scenarios as S

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_kochi_grid.json")


def test_table1_golden_is_consistent():
    t = json.load(open(GOLD))
    assert sum(l["cells"] for l in t["levels"]) == t["total_cells"]
    assert sum(l["blocks"] for l in t["levels"]) == t["total_blocks"]
    dxs = [l["dx_m"] for l in t["levels"]]
    assert all(a == 3 * b for a, b in zip(dxs, dxs[1:]))


def test_config4_has_the_kochi_shape():
    """Same level count, dx ladder and dt as Table I; total cells within 2 %."""
    t = json.load(open(GOLD))
    sc = S.config4(steps=1)
    assert sc.dt == t["dt_s"]
    levels = sorted({b["level"] for b in sc.blocks})
    assert levels == [l["level"] for l in t["levels"]]
    for l in t["levels"]:
        dx = {b["dx"] for b in sc.blocks if b["level"] == l["level"]}
        assert len(dx) == 1 and abs(dx.pop() - l["dx_m"]) < 1e-9
    assert abs(sc.cells - t["total_cells"]) <= 0.02 * t["total_cells"]
    assert sc.cells == 46_650_000
    # every child lies in shallow enough water for Eq. 4 (the generator checks too)
    for b, h in zip(sc.blocks, sc.bathy):
        assert b["dx"] / sc.dt >= np.sqrt(2 * sc.g * max(h.max(), 0.0))


def test_config_shapes():
    assert S.config1().cells == 65536
    assert S.config2(steps=1).cells == 765_000
    c3 = S.config3(steps=1)
    sides = [s.blocks[0]["nx"] for s in c3]
    assert len(c3) == 64 and min(sides) >= 128 and max(sides) <= 1024
    assert len(set(s.dt for s in c3)) > 1  # each grid has its own CFL-derived dt
    t = S.poisson_trace(1, n=10)
    assert len(t) == 10 and all(a["arrival_s"] < b["arrival_s"] for a, b in zip(t, t[1:]))
