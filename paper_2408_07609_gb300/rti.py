"""Python binding of the C ABI in include/rti.h (argument marshalling only).

Every step of the time integration runs in the CUDA library librti.so; this module
only converts numpy arrays and streams to the pointers the C functions take. It
fails loudly when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

FP64, FP32 = 0, 1
SCHED_PERSISTENT, SCHED_PER_PASS = 0, 1
BC_WALL, BC_RADIATION = 0, 1
NEST_RING, NEST_FULL = 0, 1        # fine-to-coarse feedback: boundary ring, every covered cell
FLUX_LINEAR, FLUX_CONSTANT = 0, 1  # coarse-to-fine edge flux: linear along the edge, constant

OK = 0
ERR = {-1: "INVALID_ARG", -2: "CFL", -3: "NESTING", -4: "OOM", -5: "NONFINITE", -6: "TIMEOUT",
       -7: "CUDA", -8: "STATE"}


class RtiError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"rti error {code} ({ERR.get(code, '?')}): {msg}")
        self.code = code


class Block(C.Structure):
    _fields_ = [("level", C.c_int), ("parent", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("i0", C.c_int), ("j0", C.c_int), ("dx", C.c_double), ("bc", C.c_int * 4)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("g", C.c_double), ("dry_eps", C.c_double),
                ("arrival_thr", C.c_double), ("precision", C.c_int), ("schedule", C.c_int),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("track_velocity", C.c_int),
                ("nest_feedback", C.c_int), ("nest_flux", C.c_int), ("ctas_per_sm", C.c_int),
                ("velocity_limit", C.c_double)]


class BatchConfig(C.Structure):
    _fields_ = [("precision", C.c_int), ("schedule", C.c_int), ("chunk_steps", C.c_int),
                ("tile_y", C.c_int), ("ctas_per_sm", C.c_int)]


class NoAllocState(C.Structure):
    """Device pointers of a caller-owned single-grid state (rti_noalloc_state)."""
    _fields_ = [("eta", C.c_void_p * 2), ("M", C.c_void_p * 2), ("N", C.c_void_p * 2),
                ("h", C.c_void_p), ("manning", C.c_void_p), ("max_eta", C.c_void_p),
                ("arrival_step", C.c_void_p), ("pitch", C.c_int)]


_lib = None
_dp = C.POINTER(C.c_double)
_vp = C.c_void_p


def lib():
    """The loaded librti.so; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is None:
        path = os.environ.get("RTI_LIBRARY", LIB)  # e.g. the range-checked build
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: the CUDA library must be built first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(path)
        sig = {
            "rti_footprint": (C.c_int, [C.POINTER(Block), C.c_int, C.POINTER(Params),
                                        C.POINTER(C.c_size_t)]),
            "rti_create": (C.c_int, [C.POINTER(Block), C.c_int, C.POINTER(_dp),
                                     C.POINTER(C.POINTER(C.c_float)), C.POINTER(Params), _vp,
                                     C.c_size_t, C.POINTER(_vp)]),
            "rti_set_initial_uplift": (C.c_int, [_vp, C.c_int, _dp]),
            "rti_step": (C.c_int, [_vp, C.c_int, _vp]),
            "rti_sync": (C.c_int, [_vp]),
            "rti_sync_timeout": (C.c_int, [_vp, C.c_double]),
            "rti_batch_sync_timeout": (C.c_int, [_vp, C.c_double]),
            "rti_get_max_depth": (C.c_int, [_vp, C.c_int, _dp]),
            "rti_get_max_height": (C.c_int, [_vp, C.c_int, _dp]),
            "rti_get_arrival_time": (C.c_int, [_vp, C.c_int, _dp]),
            "rti_get_max_velocity": (C.c_int, [_vp, C.c_int, _dp]),
            "rti_get_state": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp]),
            "rti_set_state": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp]),
            "rti_get_budget": (C.c_int, [_vp, C.c_int, _dp]),
            "rti_checkpoint_bytes": (C.c_size_t, [_vp]),
            "rti_checkpoint_save": (C.c_int, [_vp, _vp, C.c_size_t]),
            "rti_checkpoint_load": (C.c_int, [_vp, _vp, C.c_size_t]),
            "rti_volume": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
            "rti_get_transfer_bytes": (C.c_int, [_vp, C.POINTER(C.c_longlong),
                                                 C.POINTER(C.c_longlong)]),
            "rti_steps_done": (C.c_longlong, [_vp]),
            "rti_num_blocks": (C.c_int, [_vp]),
            "rti_num_cells": (C.c_longlong, [_vp]),
            "rti_destroy": (None, [_vp]),
            "rti_last_error": (C.c_char_p, [_vp]),
            "rti_error_string": (C.c_char_p, [C.c_int]),
            "rti_batch_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(_vp)]),
            "rti_batch_create_ex": (C.c_int, [C.POINTER(BatchConfig), C.POINTER(_vp)]),
            "rti_batch_add": (C.c_int, [_vp, _vp, C.c_longlong]),
            "rti_batch_remove": (C.c_int, [_vp, _vp]),
            "rti_batch_step": (C.c_int, [_vp, _vp]),
            "rti_batch_remaining": (C.c_longlong, [_vp, _vp]),
            "rti_batch_sync": (C.c_int, [_vp]),
            "rti_batch_destroy": (None, [_vp]),
            "rti_step_noalloc": (C.c_int, [C.POINTER(Block), C.POINTER(Params),
                                           C.POINTER(NoAllocState), C.c_longlong, C.c_int, _vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):  # torch.cuda.Stream
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _blocks_array(blocks):
    arr = (Block * len(blocks))()
    for k, b in enumerate(blocks):
        arr[k].level, arr[k].parent = int(b["level"]), int(b["parent"])
        arr[k].nx, arr[k].ny = int(b["nx"]), int(b["ny"])
        arr[k].i0, arr[k].j0 = int(b.get("i0", 0)), int(b.get("j0", 0))
        arr[k].dx = float(b["dx"])
        for s in range(4):
            arr[k].bc[s] = int(b.get("bc", (0, 0, 0, 0))[s])
    return arr


def make_params(dt, g=9.81, dry_eps=1e-3, arrival_thr=0.01, precision=FP64,
                schedule=SCHED_PERSISTENT, tile=(0, 0), track_velocity=False,
                nest_feedback=None, nest_flux=None, ctas_per_sm=0, velocity_limit=0.0):
    return Params(float(dt), float(g), float(dry_eps), float(arrival_thr), int(precision),
                  int(schedule), int(tile[0]), int(tile[1]), int(bool(track_velocity)),
                  NEST_RING if nest_feedback is None else int(nest_feedback),
                  FLUX_LINEAR if nest_flux is None else int(nest_flux), int(ctas_per_sm),
                  float(velocity_limit))


def footprint(blocks, params: Params) -> int:
    out = C.c_size_t(0)
    arr = _blocks_array(blocks)
    rc = lib().rti_footprint(arr, len(blocks), C.byref(params), C.byref(out))
    if rc:
        raise RtiError(rc, "footprint")
    return out.value


class Handle:
    """One nested-grid hierarchy resident on the GPU (rti_create)."""

    def __init__(self, blocks, bathy, manning, dt, g=9.81, dry_eps=1e-3, arrival_thr=0.01,
                 precision=FP64, schedule=SCHED_PERSISTENT, tile=(0, 0), device_mem=None,
                 track_velocity=False, nest_feedback=None, nest_flux=None, ctas_per_sm=0,
                 velocity_limit=0.0):
        L = lib()
        self.blocks = [dict(b) for b in blocks]
        self.params = make_params(dt, g, dry_eps, arrival_thr, precision, schedule, tile,
                                  track_velocity, nest_feedback, nest_flux, ctas_per_sm,
                                  velocity_limit)
        self.dt = float(dt)
        nb = len(blocks)
        arr = _blocks_array(blocks)
        hs = [np.ascontiguousarray(x, np.float64) for x in bathy]
        ns = [np.ascontiguousarray(x, np.float32) for x in manning]
        hp = (_dp * nb)(*[x.ctypes.data_as(_dp) for x in hs])
        np_ = (C.POINTER(C.c_float) * nb)(*[x.ctypes.data_as(C.POINTER(C.c_float)) for x in ns])
        mem, nbytes = None, 0
        if device_mem is not None:  # e.g. a torch uint8 CUDA tensor owned by the caller
            self._mem = device_mem
            mem, nbytes = C.c_void_p(device_mem.data_ptr()), device_mem.numel() * device_mem.element_size()
        out = _vp()
        rc = L.rti_create(arr, nb, hp, np_, C.byref(self.params), mem, nbytes, C.byref(out))
        if rc:
            raise RtiError(rc, "rti_create: " + (L.rti_last_error(None) or b"").decode())
        self._h = out

    @classmethod
    def from_scenario(cls, sc, precision=FP64, schedule=SCHED_PERSISTENT, tile=(0, 0),
                      device_mem=None, track_velocity=False, nest_feedback=None,
                      nest_flux=None, ctas_per_sm=0, velocity_limit=0.0):
        h = cls(sc.blocks, sc.bathy, sc.manning, sc.dt, sc.g, sc.dry_eps, sc.arrival_thr,
                precision, schedule, tile, device_mem, track_velocity, nest_feedback, nest_flux,
                ctas_per_sm, velocity_limit)
        for k, dz in enumerate(sc.uplift):
            if dz is not None:
                h.set_initial_uplift(k, dz)
        return h

    # -- calls
    def _chk(self, rc, what):
        if rc:
            raise RtiError(rc, f"{what}: {lib().rti_last_error(self._h).decode()}")

    def shape(self, k):
        return self.blocks[k]["ny"], self.blocks[k]["nx"]

    def set_initial_uplift(self, k, dz):
        ny, nx = self.shape(k)
        a = None if dz is None else np.ascontiguousarray(dz, np.float64).reshape(ny, nx)
        self._chk(lib().rti_set_initial_uplift(self._h, k, None if a is None else a.ctypes.data_as(_dp)),
                  "set_initial_uplift")

    def step(self, n=1, stream=None):
        self._chk(lib().rti_step(self._h, int(n), _stream_ptr(stream)), "step")

    def sync(self, timeout=None):
        """Wait for the enqueued work (at most `timeout` seconds: RtiError TIMEOUT after)."""
        if timeout is None:
            self._chk(lib().rti_sync(self._h), "sync")
        else:
            self._chk(lib().rti_sync_timeout(self._h, float(timeout)), "sync_timeout")

    def get_state(self, k):
        ny, nx = self.shape(k)
        eta, M, N = np.empty((ny, nx)), np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
        self._chk(lib().rti_get_state(self._h, k, eta.ctypes.data_as(_dp), M.ctypes.data_as(_dp),
                                      N.ctypes.data_as(_dp)), "get_state")
        return eta, M, N

    def set_state(self, k, eta=None, M=None, N=None):
        ny, nx = self.shape(k)
        cv = lambda a, s: None if a is None else np.ascontiguousarray(a, np.float64).reshape(s)
        eta, M, N = cv(eta, (ny, nx)), cv(M, (ny, nx + 1)), cv(N, (ny + 1, nx))
        p = lambda a: None if a is None else a.ctypes.data_as(_dp)
        self._chk(lib().rti_set_state(self._h, k, p(eta), p(M), p(N)), "set_state")

    def _field(self, fn, k, out=None):
        """out: a C-contiguous (ny, nx) float64 array to fill (e.g. pinned host memory);
        None allocates one."""
        ny, nx = self.shape(k)
        if out is None:
            out = np.empty((ny, nx))
        elif out.shape != (ny, nx) or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError(f"out must be a C-contiguous ({ny}, {nx}) float64 array")
        self._chk(getattr(lib(), fn)(self._h, k, out.ctypes.data_as(_dp)), fn)
        return out

    def max_depth(self, k, out=None):
        return self._field("rti_get_max_depth", k, out)

    def max_height(self, k, out=None):
        return self._field("rti_get_max_height", k, out)

    def arrival_time(self, k, out=None):
        return self._field("rti_get_arrival_time", k, out)

    def max_velocity(self, k, out=None):
        return self._field("rti_get_max_velocity", k, out)

    def budget(self, k):
        out = np.empty(4)
        self._chk(lib().rti_get_budget(self._h, k, out.ctypes.data_as(_dp)), "budget")
        return dict(volume=out[0], outflow=out[1], clip=out[2], ring=out[3])

    def checkpoint(self) -> bytes:
        """The whole handle's state as bytes (rti_checkpoint_save)."""
        n = lib().rti_checkpoint_bytes(self._h)
        buf = C.create_string_buffer(n)
        self._chk(lib().rti_checkpoint_save(self._h, buf, n), "checkpoint_save")
        return buf.raw

    def restore(self, data: bytes):
        """Resume from a checkpoint of a handle with the same blocks and params."""
        buf = C.create_string_buffer(data, len(data))
        self._chk(lib().rti_checkpoint_load(self._h, buf, len(data)), "checkpoint_load")

    def volume(self):
        """Whole-domain budget over the root blocks (rti_volume)."""
        v = [C.c_double(0.0) for _ in range(4)]
        self._chk(lib().rti_volume(self._h, *[C.byref(x) for x in v]), "volume")
        return dict(volume=v[0].value, outflow=v[1].value, clip=v[2].value, feedback=v[3].value)

    def transfer_bytes(self):
        a, b = C.c_longlong(0), C.c_longlong(0)
        self._chk(lib().rti_get_transfer_bytes(self._h, C.byref(a), C.byref(b)), "transfer_bytes")
        return a.value, b.value

    @property
    def steps_done(self):
        return lib().rti_steps_done(self._h)

    @property
    def cells(self):
        return lib().rti_num_cells(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().rti_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many hierarchies stepped together by one persistent, graph-captured launch."""

    def __init__(self, precision=FP32, schedule=SCHED_PERSISTENT, chunk_steps=50, tile_y=0,
                 ctas_per_sm=0):
        out = _vp()
        cfg = BatchConfig(int(precision), int(schedule), int(chunk_steps), int(tile_y),
                          int(ctas_per_sm))
        rc = lib().rti_batch_create_ex(C.byref(cfg), C.byref(out))
        if rc:
            raise RtiError(rc, "rti_batch_create_ex")
        self._b = out
        self.chunk = int(chunk_steps)
        self.members = []

    def add(self, h: Handle, nsteps: int):
        rc = lib().rti_batch_add(self._b, h._h, int(nsteps))
        if rc:
            raise RtiError(rc, "rti_batch_add")
        self.members.append(h)

    def remove(self, h: Handle):
        rc = lib().rti_batch_remove(self._b, h._h)
        if rc:
            raise RtiError(rc, "rti_batch_remove")
        self.members.remove(h)

    def step(self, stream=None):
        rc = lib().rti_batch_step(self._b, _stream_ptr(stream))
        if rc:
            raise RtiError(rc, "rti_batch_step")

    def remaining(self, h: Handle) -> int:
        return lib().rti_batch_remaining(self._b, h._h)

    def sync(self, timeout=None):
        rc = (lib().rti_batch_sync(self._b) if timeout is None
              else lib().rti_batch_sync_timeout(self._b, float(timeout)))
        if rc:
            raise RtiError(rc, "rti_batch_sync")

    def close(self):
        if getattr(self, "_b", None):
            lib().rti_batch_destroy(self._b)
            self._b = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def noalloc_pitch(nx):
    """Row pitch (elements) of the library's layout for a grid nx cells wide."""
    return (nx + 9 + 31) // 32 * 32


def step_noalloc(block, params: Params, state: NoAllocState, steps_done, nsteps, stream=None):
    """rti_step_noalloc: step one caller-owned root grid without any device allocation."""
    arr = _blocks_array([block])
    rc = lib().rti_step_noalloc(arr, C.byref(params), C.byref(state), int(steps_done),
                                int(nsteps), _stream_ptr(stream))
    if rc:
        raise RtiError(rc, "rti_step_noalloc: " + (lib().rti_last_error(None) or b"").decode())
