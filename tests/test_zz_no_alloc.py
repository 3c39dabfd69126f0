"""rti_step_noalloc, the allocation-free entry point, against rti_create + rti_step.

Some callers cannot call cudaMalloc (a service that hands all device memory to its own
pool, or code that must not risk a failing or device-synchronising allocation). For
them the library steps one caller-owned grid with its scratch in a static device
array. Both paths run the same kernels on the same strips, so their results agree
bitwise. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2408_07609_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


class CallerState:
    """The state arrays, allocated by the caller (torch) in the library's layout, with
    the library's own row pitch or any other one the call allows (>= nx + 9, a multiple
    of 4)."""

    def __init__(self, torch, rti, nx, ny, dtype, pitch=None):
        self.nx, self.ny = nx, ny
        self.pitch = rti.noalloc_pitch(nx) if pitch is None else pitch
        self.rows = ny + 5
        mk = lambda dt: torch.zeros(self.rows * self.pitch, dtype=dt, device="cuda")
        self.eta = [mk(dtype), mk(dtype)]
        self.M = [mk(dtype), mk(dtype)]
        self.N = [mk(dtype), mk(dtype)]
        self.h, self.emax = mk(dtype), mk(dtype)
        self.man = mk(torch.float32)
        self.arr = mk(torch.int32)
        st = rti.NoAllocState()
        for q in range(2):
            st.eta[q], st.M[q], st.N[q] = (self.eta[q].data_ptr(), self.M[q].data_ptr(),
                                           self.N[q].data_ptr())
        st.h, st.manning = self.h.data_ptr(), self.man.data_ptr()
        st.max_eta, st.arrival_step, st.pitch = self.emax.data_ptr(), self.arr.data_ptr(), self.pitch
        self.st = st

    def view(self, t, ncols, nrows):
        return t.view(self.rows, self.pitch)[2:2 + nrows, 4:4 + ncols]

    def put(self, t, a, ncols, nrows):
        import torch

        self.view(t, ncols, nrows).copy_(torch.as_tensor(a).to(t.dtype))

    def get(self, t, ncols, nrows):
        return self.view(t, ncols, nrows).double().cpu().numpy()


def tight_pitch(nx):
    """The smallest pitch the call allows: nx + 9 rounded up to a multiple of 4."""
    return (nx + 9 + 3) // 4 * 4


@pytest.mark.parametrize("precision,schedule,nx,tight", [
    (0, 0, 150, False), (0, 1, 150, False), (1, 0, 150, False),
    # 155 + 9 = 164: a pitch below the library's own 192, so the last strip's staged
    # rows end at the row's end (zero-filled chunks) and its halo reads the margin
    (0, 0, 155, True), (1, 0, 155, True)])
def test_noalloc_matches_rti_step_on_two_calls(rti, precision, schedule, nx, tight):
    import torch

    ny = 90
    sc = S.config1(nx=nx, ny=ny, steps=60)
    ref = rti.Handle.from_scenario(sc, precision=precision, schedule=schedule)
    dtype = torch.float64 if precision == 0 else torch.float32
    cs = CallerState(torch, rti, nx, ny, dtype, pitch=tight_pitch(nx) if tight else None)
    if tight:
        assert cs.pitch == 164 and cs.pitch != rti.noalloc_pitch(nx)
    eta0, _, _ = ref.get_state(0)
    emax0 = ref.max_height(0)
    arr0 = ref.arrival_time(0)
    cs.put(cs.eta[0], eta0, nx, ny)
    cs.put(cs.h, sc.bathy[0], nx, ny)
    cs.put(cs.man, sc.manning[0], nx, ny)
    cs.put(cs.emax, np.where(np.isnan(emax0), -1e30, emax0), nx, ny)
    cs.put(cs.arr, np.where(arr0 < 0, -1, np.rint(arr0 / sc.dt)).astype(np.int32), nx, ny)
    params = rti.make_params(sc.dt, precision=precision, schedule=schedule)
    done = 0
    for n in (23, 37):  # two calls in a row
        rti.step_noalloc(ref.blocks[0], params, cs.st, done, n)
        ref.step(n)
        ref.sync()
        done += n
        p = done & 1
        ge, gM, gN = ref.get_state(0)
        assert np.array_equal(cs.get(cs.eta[p], nx, ny), ge)
        assert np.array_equal(cs.get(cs.M[p], nx + 1, ny), gM)
        assert np.array_equal(cs.get(cs.N[p], nx, ny + 1), gN)
        gm = ref.max_height(0)
        em = cs.get(cs.emax, nx, ny)
        wet = ~np.isnan(gm)
        assert np.array_equal(wet, em > -1e29)
        assert np.array_equal(em[wet], gm[wet])
        ga = ref.arrival_time(0)
        ca = cs.get(cs.arr, nx, ny)
        assert np.array_equal(np.where(ca < 0, -1.0, ca * sc.dt), ga)
    ref.close()


def test_noalloc_rejects_grids_beyond_its_scratch(rti):
    """8192^2 cells are 37,504 strips of 28 x 64, far above the 4096-strip scratch: the
    call returns before any device work. The arrays are host memory, which the second
    host check (device memory only) would refuse as well, so no launch can follow."""
    big = dict(level=1, parent=-1, nx=8192, ny=8192, i0=0, j0=0, dx=1000.0, bc=(0, 0, 0, 0))
    host = np.zeros(1 << 10, dtype=np.float64)
    st = rti.NoAllocState()
    for q in range(2):
        st.eta[q] = st.M[q] = st.N[q] = host.ctypes.data
    st.h = st.manning = st.max_eta = st.arrival_step = host.ctypes.data
    st.pitch = rti.noalloc_pitch(8192)
    with pytest.raises(rti.RtiError) as ei:
        rti.step_noalloc(big, rti.make_params(1.0, tile=(28, 64)), st, 0, 1)
    assert ei.value.code == -1 and "tiles exceeds" in str(ei.value)


def test_noalloc_rejects_host_addresses(rti):
    """A grid that fits the scratch but whose arrays are not device memory is refused
    on the host, before any launch."""
    small = dict(level=1, parent=-1, nx=64, ny=64, i0=0, j0=0, dx=1000.0, bc=(0, 0, 0, 0))
    host = np.zeros(1 << 16, dtype=np.float64)
    st = rti.NoAllocState()
    for q in range(2):
        st.eta[q] = st.M[q] = st.N[q] = host.ctypes.data
    st.h = st.manning = st.max_eta = st.arrival_step = host.ctypes.data
    st.pitch = rti.noalloc_pitch(64)
    with pytest.raises(rti.RtiError) as ei:
        rti.step_noalloc(small, rti.make_params(1.0), st, 0, 1)
    assert ei.value.code == -1 and "not device memory" in str(ei.value)
