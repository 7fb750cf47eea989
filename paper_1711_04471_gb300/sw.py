"""2-D shallow-water model (Sec. 6.2 of arXiv:1711.04471) on the GPU.

Thin wrapper of the sw_* entry points of libgbsw.so; the state lives in
device memory owned by the library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N


class SW:
    def __init__(self, params: dict, H: np.ndarray, eta0: np.ndarray, stream=None):
        L = N.lib()
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        p = N.SWParams(self.nx, self.ny, params["dx"], params["dy"], params["dt"],
                       params.get("g", 9.81), params.get("eps", 0.05), params.get("hmin", 0.05))
        H = np.ascontiguousarray(H, dtype=np.float64)
        eta0 = np.ascontiguousarray(eta0, dtype=np.float64)
        if H.shape != (self.ny, self.nx) or eta0.shape != (self.ny, self.nx):
            raise ValueError("H and eta0 must be (ny, nx)")
        h = C.c_void_p()
        N.check(L.sw_create(C.byref(p), N.ptr(H, C.c_double), N.ptr(eta0, C.c_double),
                            N.stream_handle(stream), C.byref(h)), "sw_create")
        self._h = h

    def step(self, nsteps: int) -> "SW":
        N.check(N.lib().sw_step(self._h, int(nsteps)), "sw_step")
        return self

    def set_blocking(self, T: int) -> None:
        N.check(N.lib().sw_set_blocking(self._h, int(T)), "sw_set_blocking")

    def set_tiling(self, T: int, rows: int) -> None:
        """Steps per launch T and the row-segment height of the streaming
        kernel (0: automatic), or rows < 0 for the tile kernel: -1 with
        32-row tiles, -h with h-row tiles (T = 1..3)."""
        N.check(N.lib().sw_set_tiling(self._h, int(T), int(rows)), "sw_set_tiling")

    def autotune(self, trial_steps: int = 60):
        """Pick the fused depth and the row-segment height (or tile height,
        rows < 0) by timing them on this grid (the state is restored);
        returns (T, rows) in the encoding of set_tiling."""
        T, rows = C.c_int(), C.c_int()
        N.check(N.lib().sw_autotune(self._h, int(trial_steps), C.byref(T), C.byref(rows)), "sw_autotune")
        return T.value, rows.value

    def volume(self):
        v, w = C.c_double(), C.c_double()
        N.check(N.lib().sw_volume(self._h, C.byref(v), C.byref(w)), "sw_volume")
        return v.value, w.value

    def get_state(self, eta=None, u=None, v=None, wet=None, want=("eta", "u", "v", "wet")):
        nx, ny = self.nx, self.ny
        if eta is None and "eta" in want:
            eta = np.empty((ny, nx), np.float32)
        if u is None and "u" in want:
            u = np.empty((ny, nx + 1), np.float32)
        if v is None and "v" in want:
            v = np.empty((ny + 1, nx), np.float32)
        if wet is None and "wet" in want:
            wet = np.empty((ny, nx), np.uint8)
        N.check(N.lib().sw_get_state(self._h, N.ptr(eta, C.c_float), N.ptr(u, C.c_float),
                                     N.ptr(v, C.c_float), N.ptr(wet, C.c_uint8)), "sw_get_state")
        return dict(eta=eta, u=u, v=v, wet=wet)

    def set_state(self, eta=None, u=None, v=None):
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
        eta, u, v = f(eta), f(u), f(v)
        N.check(N.lib().sw_set_state(self._h, N.ptr(eta, C.c_float), N.ptr(u, C.c_float),
                                     N.ptr(v, C.c_float)), "sw_set_state")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().sw_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SW64:
    """The 2DSW step in FP64 end to end (sw64_* entry points): the same
    method and parameters as SW, three kernels per step, every operation
    rounded as written."""

    def __init__(self, params: dict, H: np.ndarray, eta0: np.ndarray, stream=None):
        L = N.lib()
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        p = N.SWParams(self.nx, self.ny, params["dx"], params["dy"], params["dt"],
                       params.get("g", 9.81), params.get("eps", 0.05), params.get("hmin", 0.05))
        H = np.ascontiguousarray(H, dtype=np.float64)
        eta0 = np.ascontiguousarray(eta0, dtype=np.float64)
        if H.shape != (self.ny, self.nx) or eta0.shape != (self.ny, self.nx):
            raise ValueError("H and eta0 must be (ny, nx)")
        h = C.c_void_p()
        N.check(L.sw64_create(C.byref(p), N.ptr(H, C.c_double), N.ptr(eta0, C.c_double),
                              N.stream_handle(stream), C.byref(h)), "sw64_create")
        self._h = h

    def step(self, nsteps: int) -> "SW64":
        N.check(N.lib().sw64_step(self._h, int(nsteps)), "sw64_step")
        return self

    def volume(self):
        v, w = C.c_double(), C.c_double()
        N.check(N.lib().sw64_volume(self._h, C.byref(v), C.byref(w)), "sw64_volume")
        return v.value, w.value

    def get_state(self):
        nx, ny = self.nx, self.ny
        eta = np.empty((ny, nx))
        u = np.empty((ny, nx + 1))
        v = np.empty((ny + 1, nx))
        wet = np.empty((ny, nx), np.uint8)
        N.check(N.lib().sw64_get_state(self._h, N.ptr(eta, C.c_double), N.ptr(u, C.c_double),
                                       N.ptr(v, C.c_double), N.ptr(wet, C.c_uint8)), "sw64_get_state")
        return dict(eta=eta, u=u, v=v, wet=wet)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().sw64_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SWBatch:
    """Ensemble of independent 2DSW instances stepped by one persistent
    kernel (sw_batch_* entry points)."""

    def __init__(self, members, stream=None):
        L = N.lib()
        self.n = len(members)
        self.shapes = [(m.ny, m.nx) for m in members]
        params = (N.SWParams * self.n)()
        self._H = [np.ascontiguousarray(m.H, dtype=np.float64) for m in members]
        self._E = [np.ascontiguousarray(m.eta0, dtype=np.float64) for m in members]
        for k, m in enumerate(members):
            params[k] = N.SWParams(m.nx, m.ny, m.dx, m.dy, m.dt, m.g, m.eps, m.hmin)
        dpp = C.POINTER(C.c_double)
        Hp = (dpp * self.n)(*[a.ctypes.data_as(dpp) for a in self._H])
        Ep = (dpp * self.n)(*[a.ctypes.data_as(dpp) for a in self._E])
        h = C.c_void_p()
        N.check(L.sw_batch_create(self.n, C.cast(params, C.c_void_p), Hp, Ep, N.stream_handle(stream), C.byref(h)),
                "sw_batch_create")
        self._h = h
        self._H = self._E = None

    def step(self, nsteps: int):
        N.check(N.lib().sw_batch_step(self._h, int(nsteps)), "sw_batch_step")

    def step_separate(self, nsteps: int):
        N.check(N.lib().sw_batch_step_separate(self._h, int(nsteps)), "sw_batch_step_separate")

    def volumes(self):
        v = np.empty(self.n)
        w = np.empty(self.n)
        N.check(N.lib().sw_batch_volumes(self._h, N.ptr(v, C.c_double), N.ptr(w, C.c_double)), "sw_batch_volumes")
        return v, w

    def get_state(self, m: int):
        ny, nx = self.shapes[m]
        eta = np.empty((ny, nx), np.float32)
        u = np.empty((ny, nx + 1), np.float32)
        v = np.empty((ny + 1, nx), np.float32)
        N.check(N.lib().sw_batch_get_state(self._h, int(m), eta.ctypes.data_as(C.c_void_p),
                                           u.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p)),
                "sw_batch_get_state")
        return dict(eta=eta, u=u, v=v)

    def set_tiling(self, steps_per_level: int, rows_per_item: int):
        N.check(N.lib().sw_batch_set_tiling(self._h, int(steps_per_level), int(rows_per_item)), "sw_batch_set_tiling")

    def get_tiling(self):
        t, r = C.c_int(), C.c_int()
        N.check(N.lib().sw_batch_get_tiling(self._h, C.byref(t), C.byref(r)), "sw_batch_get_tiling")
        return t.value, r.value

    def autotune(self, trial_steps: int = 12, cache_path: str | None = None):
        t, r = C.c_int(), C.c_int()
        cp = None if cache_path is None else cache_path.encode()
        N.check(N.lib().sw_batch_autotune(self._h, int(trial_steps), cp, C.byref(t), C.byref(r)), "sw_batch_autotune")
        return t.value, r.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().sw_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
