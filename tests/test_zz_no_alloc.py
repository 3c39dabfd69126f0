"""rti_step_noalloc, the allocation-free entry point, against rti_create + rti_step.

Some callers cannot call cudaMalloc (a service that hands all device memory to its own
pool, or code that must not risk a failing or device-synchronising allocation). For
them the library steps one caller-owned grid with its scratch in a static device
array. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2408_07609_gb300 import scenarios as S

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a - b).max()


class CallerState:
    """The state arrays, allocated by the caller (torch) in the library's layout."""

    def __init__(self, torch, rti, nx, ny, dtype):
        self.nx, self.ny, self.pitch = nx, ny, rti.noalloc_pitch(nx)
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


@pytest.mark.parametrize("precision,schedule", [(0, 0), (0, 1), (1, 0)])
def test_noalloc_matches_rti_step_on_two_calls(rti, precision, schedule):
    import torch

    sc = S.config1(nx=150, ny=90, steps=60)
    nx, ny = 150, 90
    ref = rti.Handle.from_scenario(sc, precision=precision, schedule=schedule)
    dtype = torch.float64 if precision == 0 else torch.float32
    cs = CallerState(torch, rti, nx, ny, dtype)
    eta0, _, _ = ref.get_state(0)
    emax0 = ref.max_height(0)
    arr0 = ref.arrival_time(0)
    cs.put(cs.eta[0], eta0, nx, ny)
    cs.put(cs.h, sc.bathy[0], nx, ny)
    cs.put(cs.man, sc.manning[0], nx, ny)
    cs.put(cs.emax, np.where(np.isnan(emax0), -1e30, emax0), nx, ny)
    cs.put(cs.arr, np.where(arr0 < 0, -1, np.rint(arr0 / sc.dt)).astype(np.int32), nx, ny)
    params = rti.make_params(sc.dt, precision=precision, schedule=schedule)
    tol = TOL64 if precision == 0 else 1e-6
    done = 0
    for n in (23, 37):  # two calls in a row
        rti.step_noalloc(ref.blocks[0], params, cs.st, done, n)
        ref.step(n)
        ref.sync()
        done += n
        p = done & 1
        ge, gM, gN = ref.get_state(0)
        assert relerr(cs.get(cs.eta[p], nx, ny), ge) <= tol
        assert relerr(cs.get(cs.M[p], nx + 1, ny), gM) <= tol
        assert relerr(cs.get(cs.N[p], nx, ny + 1), gN) <= tol
        gm = ref.max_height(0)
        em = cs.get(cs.emax, nx, ny)
        wet = ~np.isnan(gm)
        assert np.array_equal(wet, em > -1e29)
        assert relerr(em[wet], gm[wet]) <= tol
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
