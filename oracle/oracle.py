"""ctypes loader for the FP64 CPU oracle (oracle/rti_oracle.c).

TEST INFRASTRUCTURE ONLY. Imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the product package never imports
it. It builds the C source with gcc (no FMA contraction) into ``oracle/_build`` twice:
single-threaded, and with OpenMP over the rows of each loop (``parallel=True``); the two
builds give identical bits (the one in-step sum over cells is formed row by row in
order in both).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librti_oracle.so")
LIB_OMP = os.path.join(BUILD, "librti_oracle_omp.so")
SRC = os.path.join(HERE, "rti_oracle.c")

BC_WALL, BC_RADIATION = 0, 1
ERRORS = {0: "ok", -1: "invalid argument", -2: "CFL violated", -3: "bad nesting", -4: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle, single-threaded and with OpenMP. -ffp-contract=off: gcc fuses
    a*b+c on Arm by default. Returns the single-threaded library's path."""
    os.makedirs(BUILD, exist_ok=True)
    src_t = max(os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "rti_oracle.h")))
    for out, extra in ((LIB, []), (LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < src_t:
            tmp = out + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                 *extra, "-shared", "-o", tmp, SRC, "-lm"]
            )
            os.replace(tmp, out)
    return LIB


def threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else every core this process may
    run on)."""
    v = os.environ.get("OMP_NUM_THREADS")
    if v and v.isdigit():
        return int(v)
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


class _Block(C.Structure):
    _fields_ = [("level", C.c_int), ("parent", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("i0", C.c_int), ("j0", C.c_int), ("dx", C.c_double), ("bc", C.c_int * 4)]


NEST_RING, NEST_FULL = 0, 1
FLUX_LINEAR, FLUX_CONSTANT = 0, 1


class _Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("g", C.c_double), ("dry_eps", C.c_double),
                ("arrival_thr", C.c_double), ("nest_feedback", C.c_int), ("nest_flux", C.c_int),
                ("vel_limit", C.c_double)]


_libs = {}


def lib(path=None):
    """The oracle library (default: built from rti_oracle.c); `path` loads another build
    of the same source, which the mutation tests use."""
    key = path or LIB
    if key not in _libs:
        L = C.CDLL(path or build())
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Block), C.c_int, C.POINTER(dp),
                                 C.POINTER(C.POINTER(C.c_float)), C.POINTER(_Params),
                                 C.POINTER(C.c_int)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_initial_uplift.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_steps_done.argtypes = [C.c_void_p]
        L.orc_steps_done.restype = C.c_long
        for name in ("orc_get_state", "orc_set_state"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        for name in ("orc_get_max_height", "orc_get_max_depth", "orc_get_max_velocity",
                     "orc_get_arrival_time",
                     "orc_get_budget"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_cube_root.argtypes = [C.c_double]
        L.orc_cube_root.restype = C.c_double
        for name in ("orc_phase_mass", "orc_phase_momentum", "orc_phase_edges",
                     "orc_phase_swap", "orc_means_count", "orc_edge_count"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int]
        for name in ("orc_pack_means", "orc_unpack_means", "orc_get_edge_fluxes",
                     "orc_set_edge_fluxes"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_end_step.argtypes = [C.c_void_p]
        _libs[key] = L
    return _libs[key]


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


class Oracle:
    """One nested-grid hierarchy stepped by the FP64 oracle.

    ``blocks`` is a list of dicts with keys level, parent, nx, ny, i0, j0, dx, bc
    (the same fields as the C-ABI block descriptor). ``bathy``/``manning`` are
    lists of (ny, nx) arrays. ``parallel=True`` runs the OpenMP build (same bits).
    """

    def __init__(self, blocks, bathy, manning, dt, g=9.81, dry_eps=1e-3, arrival_thr=0.01,
                 lib_path=None, nest_feedback=NEST_RING, nest_flux=FLUX_LINEAR,
                 parallel=False, vel_limit=0.0):
        if parallel and lib_path is None:
            build()
            lib_path = LIB_OMP
        self._L = L = lib(lib_path)
        nb = len(blocks)
        arr = (_Block * nb)()
        for k, b in enumerate(blocks):
            arr[k].level = int(b["level"])
            arr[k].parent = int(b["parent"])
            arr[k].nx, arr[k].ny = int(b["nx"]), int(b["ny"])
            arr[k].i0, arr[k].j0 = int(b.get("i0", 0)), int(b.get("j0", 0))
            arr[k].dx = float(b["dx"])
            for s in range(4):
                arr[k].bc[s] = int(b.get("bc", (0, 0, 0, 0))[s])
        self._h = [np.ascontiguousarray(x, dtype=np.float64) for x in bathy]
        self._n = [np.ascontiguousarray(x, dtype=np.float32) for x in manning]
        hp = (C.POINTER(C.c_double) * nb)(*[_dptr(x) for x in self._h])
        npp = (C.POINTER(C.c_float) * nb)(
            *[x.ctypes.data_as(C.POINTER(C.c_float)) for x in self._n])
        prm = _Params(dt, g, dry_eps, arrival_thr, int(nest_feedback), int(nest_flux),
                      float(vel_limit))
        err = C.c_int(0)
        self.blocks = [dict(b) for b in blocks]
        self.dt = dt
        self._s = L.orc_create(arr, nb, hp, npp, C.byref(prm), C.byref(err))
        if not self._s:
            raise OracleError(err.value)

    def close(self):
        if getattr(self, "_s", None):
            self._L.orc_destroy(self._s)
            self._s = None

    __del__ = close

    def _chk(self, rc):
        if rc != 0:
            raise OracleError(rc)

    def shape(self, k):
        return self.blocks[k]["ny"], self.blocks[k]["nx"]

    def set_initial_uplift(self, k, dz):
        ny, nx = self.shape(k)
        dz = np.ascontiguousarray(dz, dtype=np.float64).reshape(ny, nx)
        self._chk(self._L.orc_set_initial_uplift(self._s, k, _dptr(dz)))

    def step(self, n=1):
        self._chk(self._L.orc_step(self._s, int(n)))

    @property
    def steps_done(self):
        return self._L.orc_steps_done(self._s)

    def get_state(self, k):
        ny, nx = self.shape(k)
        eta = np.empty((ny, nx))
        M = np.empty((ny, nx + 1))
        N = np.empty((ny + 1, nx))
        self._chk(self._L.orc_get_state(self._s, k, _dptr(eta), _dptr(M), _dptr(N)))
        return eta, M, N

    def set_state(self, k, eta=None, M=None, N=None):
        ny, nx = self.shape(k)
        c = lambda a, s: None if a is None else np.ascontiguousarray(a, np.float64).reshape(s)
        eta, M, N = c(eta, (ny, nx)), c(M, (ny, nx + 1)), c(N, (ny + 1, nx))
        self._chk(self._L.orc_set_state(self._s, k, _dptr(eta), _dptr(M), _dptr(N)))

    def _field(self, fn, k):
        ny, nx = self.shape(k)
        out = np.empty((ny, nx))
        self._chk(getattr(self._L, fn)(self._s, k, _dptr(out)))
        return out

    def max_height(self, k):
        return self._field("orc_get_max_height", k)

    def max_velocity(self, k):
        return self._field("orc_get_max_velocity", k)

    def max_depth(self, k):
        return self._field("orc_get_max_depth", k)

    def arrival_time(self, k):
        return self._field("orc_get_arrival_time", k)

    def budget(self, k):
        out = np.empty(4)
        self._chk(self._L.orc_get_budget(self._s, k, _dptr(out)))
        return dict(volume=out[0], outflow=out[1], clip=out[2], ring=out[3])

    # -- one step in phases, for a hierarchy split over ranks (rti_oracle.h) --
    def phase_mass(self, k):
        self._chk(self._L.orc_phase_mass(self._s, k))

    def pack_means(self, k):
        n = self._L.orc_means_count(self._s, k)
        if n < 0:
            raise OracleError(n)
        out = np.empty(n)
        self._chk(self._L.orc_pack_means(self._s, k, _dptr(out)))
        return out

    def unpack_means(self, k, v):
        v = np.ascontiguousarray(v, np.float64)
        if v.size != self._L.orc_means_count(self._s, k):
            raise ValueError("means of the wrong size")
        self._chk(self._L.orc_unpack_means(self._s, k, _dptr(v)))

    def phase_momentum(self, k):
        self._chk(self._L.orc_phase_momentum(self._s, k))

    def edge_fluxes(self, k):
        n = self._L.orc_edge_count(self._s, k)
        if n < 0:
            raise OracleError(n)
        out = np.empty(n)
        self._chk(self._L.orc_get_edge_fluxes(self._s, k, _dptr(out)))
        return out

    def set_edge_fluxes(self, k, v):
        v = np.ascontiguousarray(v, np.float64)
        if v.size != self._L.orc_edge_count(self._s, k):
            raise ValueError("edge fluxes of the wrong size")
        self._chk(self._L.orc_set_edge_fluxes(self._s, k, _dptr(v)))

    def phase_edges(self, k):
        self._chk(self._L.orc_phase_edges(self._s, k))

    def phase_swap(self, k):
        self._chk(self._L.orc_phase_swap(self._s, k))

    def end_step(self):
        self._chk(self._L.orc_end_step(self._s))


def cube_root(x):
    """The oracle's cube root (the friction term's D^(7/3)) of one number."""
    return lib().orc_cube_root(float(x))


def from_scenario(sc, **kw):
    """Oracle built from a scenario object of paper_2408_07609_gb300.scenarios."""
    o = Oracle(sc.blocks, sc.bathy, sc.manning, sc.dt, g=sc.g, dry_eps=sc.dry_eps,
               arrival_thr=sc.arrival_thr, **kw)
    for k, dz in enumerate(sc.uplift):
        if dz is not None:
            o.set_initial_uplift(k, dz)
    return o
