"""The C-ABI library loads and exports every entry point include/rti.h declares, and
its host-side validation works without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "rti.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rti_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(rti):
    L = C.CDLL(rti.LIB)
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    # the binding wraps every one of them
    bound = set(re.findall(r'"(rti_\w+)"', open(rti.__file__).read()))
    assert set(names) <= bound


def blk(**kw):
    d = dict(level=1, parent=-1, nx=30, ny=30, i0=0, j0=0, dx=100.0, bc=(0, 0, 0, 0))
    d.update(kw)
    return d


def test_footprint_and_validation_on_host(rti):
    p = rti.make_params(dt=0.5)
    fp = rti.footprint([blk()], p)
    assert fp > 30 * 30 * 8 * 8
    assert rti.footprint([blk()], rti.make_params(dt=0.5, precision=rti.FP32)) < fp
    bad = [blk(), blk(level=2, parent=0, nx=30, ny=30, i0=2, j0=3, dx=100 / 3)]
    with pytest.raises(rti.RtiError) as e:
        rti.footprint(bad, p)
    assert e.value.code == -3
    with pytest.raises(rti.RtiError) as e:
        rti.footprint([blk(nx=2)], p)
    assert e.value.code == -1
    with pytest.raises(rti.RtiError) as e:
        rti.footprint([blk()], rti.make_params(dt=0.5, tile=(48, 16)))
    assert e.value.code == -1
    # nesting options: both values of each are accepted, nothing else
    for fb in (rti.NEST_RING, rti.NEST_FULL):
        for fl in (rti.FLUX_LINEAR, rti.FLUX_CONSTANT):
            assert rti.footprint([blk()], rti.make_params(dt=0.5, nest_feedback=fb,
                                                          nest_flux=fl)) == fp
    for kw in (dict(nest_feedback=2), dict(nest_flux=-1)):
        with pytest.raises(rti.RtiError) as e:
            rti.footprint([blk()], rti.make_params(dt=0.5, **kw))
        assert e.value.code == -1


def test_create_rejects_cfl_before_any_device_call(rti):
    """Eq. 4 per block: dx/dt >= sqrt(2 g h_max). Checked on the host first."""
    h = np.full((30, 30), 1000.0)
    n = np.zeros((30, 30), np.float32)
    with pytest.raises(rti.RtiError) as e:
        rti.Handle([blk()], [h], [n], dt=1.0)
    assert e.value.code == -2
    with pytest.raises(rti.RtiError) as e:
        rti.Handle([blk()], [np.full((30, 30), np.nan)], [n], dt=0.1)
    assert e.value.code == -1


def test_threaded_input_scan_finds_the_first_offending_block(rti):
    """Inputs above 4 x 2^20 cells are scanned by several host threads in chunks. The
    answer is still the serial one: a non-finite value in any chunk is INVALID_ARG, a
    block whose deepest cell breaks Eq. 4 is CFL, and the first offending block in
    order decides between the two. All of it before any device call."""
    nx, ny = 2100, 2100  # 4.41 M cells, five chunks
    big = [blk(nx=nx, ny=ny, dx=100.0)]
    n = np.zeros((ny, nx), np.float32)
    h = np.full((ny, nx), 10.0)
    h[-1, -1] = 1000.0  # the deepest cell sits in the last chunk: dx/dt = 100 < 140
    with pytest.raises(rti.RtiError) as e:
        rti.Handle(big, [h], [n], dt=1.0)
    assert e.value.code == -2
    h[-1, -1] = 10.0
    n[ny - 3, 5] = np.inf  # a non-finite Manning n in the last chunk
    with pytest.raises(rti.RtiError) as e:
        rti.Handle(big, [h], [n], dt=1.0)
    assert e.value.code == -1
    # two blocks: the first breaks Eq. 4, the second holds a NaN -> CFL (first decides)
    two = [blk(nx=300, ny=300, dx=810.0), blk(level=2, parent=0, nx=270, ny=270, i0=100,
                                                j0=100, dx=270.0)]
    hb = [np.full((300, 300), 8000.0), np.full((270, 270), np.nan)]
    nb = [np.zeros((300, 300), np.float32), np.zeros((270, 270), np.float32)]
    with pytest.raises(rti.RtiError) as e:
        rti.Handle(two, hb, nb, dt=3.0)
    assert e.value.code == -2


def test_error_strings(rti):
    L = rti.lib()
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert L.rti_error_string(code)


def test_planes_beyond_32_bit_offsets_are_rejected(rti):
    """The kernels index a plane with 32-bit element offsets: a block whose padded plane
    has 2^31 elements or more is refused on the host."""
    big = blk(nx=1 << 20, ny=4096)
    with pytest.raises(rti.RtiError) as e:
        rti.footprint([big], rti.make_params(dt=0.5))
    assert e.value.code == -1
    ok = blk(nx=(1 << 20) - 9, ny=2040)  # pitch 2^20, 2045 rows: 2^31 - 3 x 2^20 elements
    assert rti.footprint([ok], rti.make_params(dt=0.5, precision=rti.FP32)) > 0


def test_velocity_tracking_adds_a_plane_and_is_refused_without_state(rti):
    """track_velocity adds one state-precision plane per block to the footprint; the
    allocation-free entry has no plane for it and refuses it before any device work."""
    base = rti.footprint([blk(nx=300, ny=200)], rti.make_params(dt=0.5, precision=rti.FP32))
    more = rti.footprint([blk(nx=300, ny=200)],
                         rti.make_params(dt=0.5, precision=rti.FP32, track_velocity=True))
    pitch = (300 + 9 + 31) // 32 * 32
    assert more - base >= pitch * 205 * 4
    st = rti.NoAllocState()
    with pytest.raises(rti.RtiError) as e:
        rti.step_noalloc(blk(nx=64, ny=64), rti.make_params(1.0, track_velocity=True), st, 0, 1)
    assert e.value.code == -1 and "track_velocity" in str(e.value)


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No fallback: with the library absent, the first call raises (in a fresh process,
    so the library this session loaded stays loaded)."""
    import subprocess
    import sys

    code = ("from paper_2408_07609_gb300 import rti\n"
            "try:\n    rti.lib()\nexcept RuntimeError as e:\n    print('raised', 'missing' in str(e))\n")
    env = dict(os.environ, RTI_LIBRARY=str(tmp_path / "absent.so"), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr


def test_header_is_plain_c():
    """include/rti.h compiles as C99 on its own: plain pointers and sizes, no C++ or
    torch types in the boundary."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    r = subprocess.run([gcc, "-fsyntax-only", "-x", "c", "-std=c99", "-Wall", "-Werror",
                        os.path.join(ROOT, "include", "rti.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
