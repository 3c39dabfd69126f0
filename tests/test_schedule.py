"""Host-side scheduling of a group's work list (rti_schedule.h), without a GPU: the
full-feedback order puts every child strip before the ring strips that wait for it in
the same step, and the dataflow dependencies of a chunk cover each strip's 3 x 3
neighbourhood and its nest partners both ways, with every wait on a strip handed out
earlier (so bounded waits on running warps cannot close a cycle). The checks run in
tests/schedule_check.cpp, built here with the host compiler against the library's own
header, on the benchmark's 5-level hierarchy, a 3-level nest and a batch of two."""
import os
import shutil
import subprocess

import pytest

from paper_2408_07609_gb300 import scenarios as S

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("sched") / "schedule_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2408_07609_gb300", "csrc"),
                    os.path.join(HERE, "schedule_check.cpp"), "-o", exe], check=True)
    return exe


def wide_nest():
    return S.coastal_hierarchy(
        "3-level nest, wide child", 9, (200, 120, 810.0), [(1, 216, 135), (1, 135, 90)],
        dt=0.5, steps=1, shelf_w=15e3, slope_w=20e3, wiggle=2e3, coast_frac=0.6,
        land_frac=0.4, source=dict(kind="gauss", sigma=8e3, peak=2.0))


def run(exe, blocks, full, tile=(28, 64), workers=3040, steps=3):
    lines = [f"{tile[0]} {tile[1]} {workers} {int(full)} {steps} {len(blocks)}"]
    lines += [f"{b['nx']} {b['ny']} {b['parent']} {b['i0']} {b['j0']}" for b in blocks]
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
    return [int(v) for v in r.stdout.split()[1:]]


def batch(*hierarchies):
    """The block list of a batch: each member's blocks after the previous ones."""
    out = []
    for blocks in hierarchies:
        base = len(out)
        out += [dict(b, parent=b["parent"] + base if b["parent"] >= 0 else -1) for b in blocks]
    return out


@pytest.mark.parametrize("full", [True, False])
def test_five_level_hierarchy(checker, full):
    blocks = S.config4(steps=0).blocks
    n, ndeps = run(checker, blocks, full)
    assert n == 27331 and ndeps >= 9 * n - 2 * 3000  # at least the neighbourhoods


@pytest.mark.parametrize("tile", [(28, 64), (28, 8), (28, 128)])
@pytest.mark.parametrize("workers", [3040, 16])
def test_nest_strip_shapes_and_grids(checker, tile, workers):
    run(checker, wide_nest().blocks, True, tile=tile, workers=workers, steps=4)


def test_batch_of_two_hierarchies(checker):
    run(checker, batch(S.config2(steps=0).blocks, wide_nest().blocks), True, steps=3)
