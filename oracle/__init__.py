"""FP64 CPU oracle for the 2DSW and UFLES time steps (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is independent of the CUDA
library: it shares no source, header, table or helper with it.  The C code
lives in ``oracle/*.c``; this module only marshals numpy arrays to it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_libs = {}
_use_openmp = False


def lib(openmp: bool | None = None):
    """The serial oracle library, or its OpenMP build (same sources, outer
    loops of the maps on all host cores, bitwise equal results).  With
    openmp=None, the build chosen by use_openmp()."""
    key = _use_openmp if openmp is None else bool(openmp)
    if key not in _libs:
        L = C.CDLL(_build.build(openmp=key))
        _declare(L)
        _libs[key] = L
    return _libs[key]


def use_openmp(flag: bool) -> None:
    """Route every oracle call that does not name a build to the OpenMP
    build (True) or the serial one (False, the default)."""
    global _use_openmp
    _use_openmp = bool(flag)


def threads(n: int = 0, openmp: bool = True) -> int:
    """Threads of the OpenMP build's parallel maps (n > 0 sets it); 1 for
    the serial build."""
    return int(lib(openmp).oracle_threads(int(n)))


class SWParams(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dt", C.c_double), ("g", C.c_double), ("eps", C.c_double), ("hmin", C.c_double)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def _declare(L):
    L.oracle_sw_run.argtypes = [C.POINTER(SWParams), _dp, _dp, _dp, _dp, C.c_int, C.POINTER(C.c_double)]
    L.oracle_sw_run.restype = C.c_int
    L.oracle_sw_volume.argtypes = [C.POINTER(SWParams), _dp, _dp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.oracle_sw_volume.restype = None
    L.oracle_threads.argtypes = [C.c_int]
    L.oracle_threads.restype = C.c_int
    if hasattr(L, "oracle_les_declare_marker"):
        from . import les as _les
        _les.declare(L)
    if hasattr(L, "oracle_unet_declare_marker"):
        from . import unet as _unet
        _unet.declare(L)


def _pad(a: np.ndarray) -> np.ndarray:
    ny, nx = a.shape
    out = np.zeros((ny + 2, nx + 2))
    out[1:-1, 1:-1] = a
    return out


class SWState:
    """2DSW state in the oracle's padded layout.

    eta: (ny, nx) interior cells; u: (ny, nx+1) east faces i = 0..nx;
    v: (ny+1, nx) north faces j = 0..ny (wall faces included, always 0).
    """

    def __init__(self, params: dict, H: np.ndarray, eta0: np.ndarray):
        self.p = SWParams(**{k: params[k] for k in ("nx", "ny", "dx", "dy", "dt", "g", "eps", "hmin")})
        ny, nx = H.shape
        assert (nx, ny) == (self.p.nx, self.p.ny)
        self.H = _pad(np.asarray(H, dtype=np.float64))
        self.eta = _pad(np.asarray(eta0, dtype=np.float64))
        self.u = np.zeros((ny + 2, nx + 2))
        self.v = np.zeros((ny + 2, nx + 2))
        self.margin = float("inf")

    def set_velocity(self, u: np.ndarray, v: np.ndarray):
        ny, nx = self.p.ny, self.p.nx
        self.u[:] = 0.0
        self.v[:] = 0.0
        self.u[1:ny + 1, 0:nx + 1] = u
        self.v[0:ny + 1, 1:nx + 1] = v

    def run(self, nsteps: int) -> "SWState":
        m = C.c_double(0.0)
        rc = lib().oracle_sw_run(C.byref(self.p), self.H, self.eta, self.u, self.v, int(nsteps), C.byref(m))
        if rc != 0:
            raise MemoryError("oracle_sw_run: allocation failed")
        self.margin = min(self.margin, m.value)
        return self

    def volume(self):
        vol, wv = C.c_double(), C.c_double()
        lib().oracle_sw_volume(C.byref(self.p), self.H, self.eta, C.byref(vol), C.byref(wv))
        return vol.value, wv.value

    # Views in the public (interior / face) layout.
    @property
    def eta_i(self):
        return self.eta[1:-1, 1:-1].copy()

    @property
    def u_f(self):
        return self.u[1:-1, 0:self.p.nx + 1].copy()

    @property
    def v_f(self):
        return self.v[0:self.p.ny + 1, 1:-1].copy()

    @property
    def wet_i(self):
        h = self.H[1:-1, 1:-1] + self.eta[1:-1, 1:-1]
        return (h > self.p.hmin).astype(np.uint8)
