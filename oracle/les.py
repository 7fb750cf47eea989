"""numpy wrapper of the FP64 UFLES oracle (oracle/les_oracle.c).

Test infrastructure only.  Arrays use the oracle's padded layout
(nz+2, ny+2, nx+2), x fastest; ``solid`` is (nz, ny, nx) uint8.
"""
from __future__ import annotations

import ctypes as C

import numpy as np


class LESParams(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dt", C.c_double),
                ("u_ref", C.c_double), ("z_ref", C.c_double), ("z0", C.c_double), ("cs", C.c_double),
                ("nu", C.c_double), ("alpha", C.c_double), ("beta", C.c_double), ("omega", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int)]


class LESStateC(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("u", "v", "w", "p", "fuo", "fvo", "fwo", "gu", "gv", "gw", "fu", "fv", "fw", "nut", "b")] + \
               [("step", C.c_int)]


DEFAULTS = dict(dx=4.0, dt=0.025, u_ref=5.0, z_ref=10.0, z0=0.1, cs=0.1, nu=1.5e-5, alpha=-100.0, beta=-10.0,
                omega=1.8, tol=1e-6, max_iter=100000)

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_P = C.POINTER(LESParams)


def declare(L):
    def sig(name, res, args):
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    sig("oracle_les_velnw", None, [_P, _dp, _dp, _dp, _dp])
    sig("oracle_les_bondv1", None, [_P, _dp, _dp, _dp])
    sig("oracle_les_velfg", None, [_P, _dp, _dp, _dp, _dp, _dp, _dp])
    sig("oracle_les_feedbf", None, [_P, _u8p, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp])
    sig("oracle_les_nut", None, [_P, _dp, _dp, _dp, _dp])
    sig("oracle_les_visc", None, [_P, _dp, _dp, _dp, _dp, _dp, _dp, _dp])
    sig("oracle_les_adam", None, [_P, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp])
    sig("oracle_les_rhs", None, [_P, _dp, _dp, _dp, _dp])
    sig("oracle_les_apply_A", None, [_P, _dp, _dp])
    sig("oracle_les_residual", C.c_double, [_P, _dp, _dp])
    sig("oracle_les_sor", C.c_int, [_P, _dp, _dp, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_double)])
    sig("oracle_les_init", None, [_P, _u8p, C.POINTER(LESStateC)])
    sig("oracle_les_step", C.c_int, [_P, _u8p, C.POINTER(LESStateC), C.POINTER(C.c_int), C.POINTER(C.c_double)])


def _L():
    from . import lib
    return lib()


def make_params(nx, ny, nz, **kw) -> LESParams:
    d = dict(DEFAULTS)
    d.update(kw)
    return LESParams(nx, ny, nz, d["dx"], d["dt"], d["u_ref"], d["z_ref"], d["z0"], d["cs"], d["nu"], d["alpha"],
                     d["beta"], d["omega"], d["tol"], int(d["max_iter"]))


def padded(P: LESParams) -> np.ndarray:
    return np.zeros((P.nz + 2, P.ny + 2, P.nx + 2))


def interior(a: np.ndarray) -> np.ndarray:
    return a[1:-1, 1:-1, 1:-1]


class LESState:
    """Full UFLES oracle state.  u, v, w hold the predicted velocity u*
    between steps (velnw projects it at the start of the next step)."""

    NAMES = ("u", "v", "w", "p", "fuo", "fvo", "fwo", "gu", "gv", "gw", "fu", "fv", "fw", "nut", "b")

    def __init__(self, P: LESParams, solid: np.ndarray):
        self.P = P
        self.solid = np.ascontiguousarray(solid, dtype=np.uint8)
        assert self.solid.shape == (P.nz, P.ny, P.nx)
        for n in self.NAMES:
            setattr(self, n, padded(P))
        self._c = LESStateC(*[getattr(self, n).ctypes.data for n in self.NAMES], 0)
        _L().oracle_les_init(C.byref(P), self.solid, C.byref(self._c))
        self.history = []

    @property
    def step_count(self):
        return self._c.step

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            it, rr = C.c_int(), C.c_double()
            rc = _L().oracle_les_step(C.byref(self.P), self.solid, C.byref(self._c), C.byref(it), C.byref(rr))
            self.history.append((it.value, rr.value, rc))
        return self


def velnw(P, p, u, v, w):
    _L().oracle_les_velnw(C.byref(P), p, u, v, w)


def bondv1(P, u, v, w):
    _L().oracle_les_bondv1(C.byref(P), u, v, w)


def velfg(P, u, v, w):
    fu, fv, fw = padded(P), padded(P), padded(P)
    _L().oracle_les_velfg(C.byref(P), u, v, w, fu, fv, fw)
    return fu, fv, fw


def nut(P, u, v, w):
    out = padded(P)
    _L().oracle_les_nut(C.byref(P), u, v, w, out)
    return out


def visc(P, u, v, w, nu_t, fu, fv, fw):
    _L().oracle_les_visc(C.byref(P), u, v, w, nu_t, fu, fv, fw)


def feedbf(P, solid, u, v, w, gu, gv, gw, fu, fv, fw):
    _L().oracle_les_feedbf(C.byref(P), np.ascontiguousarray(solid, dtype=np.uint8), u, v, w, gu, gv, gw, fu, fv, fw)


def adam(P, first, u, v, w, fu, fv, fw, fuo, fvo, fwo):
    _L().oracle_les_adam(C.byref(P), int(first), u, v, w, fu, fv, fw, fuo, fvo, fwo)


def rhs(P, u, v, w):
    b = padded(P)
    _L().oracle_les_rhs(C.byref(P), u, v, w, b)
    return b


def apply_A(P, p):
    out = padded(P)
    _L().oracle_les_apply_A(C.byref(P), p, out)
    return out


def residual(P, b, p) -> float:
    return _L().oracle_les_residual(C.byref(P), b, p)


def sor(P, b, p, omega=None, tol=None, max_iter=None):
    it, rr = C.c_int(), C.c_double()
    rc = _L().oracle_les_sor(C.byref(P), b, p, P.omega if omega is None else omega, P.tol if tol is None else tol,
                             P.max_iter if max_iter is None else max_iter, C.byref(it), C.byref(rr))
    return rc, it.value, rr.value
