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
