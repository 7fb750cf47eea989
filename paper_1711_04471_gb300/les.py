"""Urban LES time step (Sec. 6.3 of arXiv:1711.04471) and the stand-alone
pressure solve, on the GPU.  Thin wrapper of the les_* / poisson_solve
entry points of libgbsw.so."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N
from ._native_ext import LESParams, LESState, LESStats

FIELDS = dict(u=0, v=1, w=2, p=3, fuo=4, fvo=5, fwo=6, gu=7, gv=8, gw=9, nut=10, b=11)

def _host_empty(shape, dtype) -> np.ndarray:
    """An uninitialised host array in page-locked memory, which the copy
    engine reads and writes directly (a pageable array goes through the
    library's staging buffer), from torch's caching host allocator: the
    array keeps its block alive, and a freed block serves the next array."""
    import torch
    t = torch.empty(shape, dtype=torch.float64 if dtype == np.float64 else torch.float32, pin_memory=True)
    return t.numpy()


DEFAULTS = dict(dx=4.0, dt=0.025, u_ref=5.0, z_ref=10.0, z0=0.1, cs=0.1, nu=1.5e-5, alpha=-100.0, beta=-10.0,
                omega=1.8, tol=1e-6, max_iter=100000, check_every=10)


class LES:
    def __init__(self, nx: int, ny: int, nz: int, solid: np.ndarray | None = None, stream=None, **kw):
        d = dict(DEFAULTS)
        d.update(kw)
        self.shape = (nz, ny, nx)
        self.params = LESParams(nx, ny, nz, d["dx"], d["dt"], d["u_ref"], d["z_ref"], d["z0"], d["cs"], d["nu"],
                                d["alpha"], d["beta"], d["omega"], d["tol"], int(d["max_iter"]),
                                int(d["check_every"]))
        self._solid = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8)
        if self._solid is not None and self._solid.shape != self.shape:
            raise ValueError("solid must be (nz, ny, nx)")
        h = C.c_void_p()
        sp = None if self._solid is None else self._solid.ctypes.data_as(C.c_void_p)
        N.check(N.lib().les_create(C.byref(self.params), sp, N.stream_handle(stream), C.byref(h)), "les_create")
        self._h = h

    def step(self, nsteps: int = 1, stats: bool = True):
        arr = (LESStats * max(1, nsteps))() if stats else None
        st = N.lib().les_step(self._h, int(nsteps), arr)
        N.check(st, "les_step")
        if not stats:
            return st
        return [dict(iters=a.iters, status=a.status, rel_res=a.rel_res, ms_predictor=a.ms_predictor,
                     ms_solve=a.ms_solve, ms_guess=a.ms_guess) for a in arr[:nsteps]]

    def get(self, name: str) -> np.ndarray:
        nz, ny, nx = self.shape
        out = _host_empty((nz + 2, ny + 2, nx + 2), np.float64 if name == "p" else np.float32)
        N.check(N.lib().les_get_field(self._h, FIELDS[name], out.ctypes.data_as(C.c_void_p)), "les_get_field")
        return out

    def set(self, name: str, arr: np.ndarray):
        nz, ny, nx = self.shape
        a = np.ascontiguousarray(arr, dtype=np.float64 if name == "p" else np.float32)
        if a.shape != (nz + 2, ny + 2, nx + 2):
            raise ValueError("fields are exchanged in the padded (nz+2, ny+2, nx+2) layout")
        N.check(N.lib().les_set_field(self._h, FIELDS[name], a.ctypes.data_as(C.c_void_p)), "les_set_field")

    STATE = ("u", "v", "w", "p", "fu_old", "fv_old", "fw_old", "gu", "gv", "gw")

    def get_state(self) -> dict:
        """Checkpoint: every field the next step depends on (padded layout)
        and the step count."""
        nz, ny, nx = self.shape
        out = {n: _host_empty((nz + 2, ny + 2, nx + 2), np.float64 if n == "p" else np.float32)
               for n in self.STATE}
        st = LESState(*[out[n].ctypes.data for n in self.STATE], 0)
        N.check(N.lib().les_get_state(self._h, C.byref(st)), "les_get_state")
        out["step"] = st.step
        return out

    def set_state(self, state: dict):
        """Restart from a checkpoint of get_state (fields missing from the
        dict keep their current values)."""
        nz, ny, nx = self.shape
        keep = {}
        for n in self.STATE:
            if n in state:
                a = np.ascontiguousarray(state[n], dtype=np.float64 if n == "p" else np.float32)
                if a.shape != (nz + 2, ny + 2, nx + 2):
                    raise ValueError("fields are exchanged in the padded (nz+2, ny+2, nx+2) layout")
                keep[n] = a
        st = LESState(*[keep[n].ctypes.data if n in keep else None for n in self.STATE],
                      int(state.get("step", self.step_count)))
        N.check(N.lib().les_set_state(self._h, C.byref(st)), "les_set_state")

    @property
    def step_count(self) -> int:
        s = C.c_int()
        N.check(N.lib().les_get_step(self._h, C.byref(s)), "les_get_step")
        return s.value

    @step_count.setter
    def step_count(self, v: int):
        N.check(N.lib().les_set_step(self._h, int(v)), "les_set_step")

    def set_solver(self, omega=None, tol=None, max_iter=None, check_every=None):
        p = self.params
        p.omega = p.omega if omega is None else omega
        p.tol = p.tol if tol is None else tol
        p.max_iter = p.max_iter if max_iter is None else int(max_iter)
        p.check_every = p.check_every if check_every is None else int(check_every)
        N.check(N.lib().les_set_solver(self._h, p.omega, p.tol, p.max_iter, p.check_every), "les_set_solver")

    def set_check_prediction(self, on: bool):
        """Predicted convergence checks (on by default): see
        les_set_check_prediction in include/gbsw.h."""
        N.check(N.lib().les_set_check_prediction(self._h, int(bool(on))), "les_set_check_prediction")

    def set_warm_start(self, net, factor: int = 0):
        """Use a UNet (paper_1711_04471_gb300.unet.UNet) as the pressure warm
        start, run on the grid coarsened by `factor` (0: the default, 16 on
        a 256 x 256 x 128 grid), or None for the previous pressure.  The
        network must outlive its use here."""
        N.check(N.lib().les_set_warm_start_factor(self._h, int(factor)), "les_set_warm_start_factor")
        self._net = net
        N.check(N.lib().les_set_warm_start(self._h, None if net is None else net._h), "les_set_warm_start")

    def set_fixed_iterations(self, niter: int):
        """Paper mode: exactly niter SOR iterations per step (0 = tolerance-driven)."""
        N.check(N.lib().les_set_fixed_iterations(self._h, int(niter)), "les_set_fixed_iterations")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().les_destroy(self._h)
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


def poisson_solve(p, b, dx: float, omega=1.8, tol=1e-6, max_iter=100000, check_every=10, stream=None):
    """Solve A p = b in place on CUDA float32 tensors of shape (nz, ny, nx).
    Returns (status, iterations, relative residual)."""
    nz, ny, nx = p.shape
    assert b.shape == p.shape
    it, rr = C.c_int(), C.c_double()
    st = N.lib().poisson_solve(nx, ny, nz, dx, N.tensor_ptr(p, "float32"), N.tensor_ptr(b, "float32"), omega, tol,
                               int(max_iter), int(check_every), N.stream_handle(stream), C.byref(it), C.byref(rr))
    N.check(st, "poisson_solve")
    return st, it.value, rr.value


def warm_start_features(p, b, dx: float, f: int, stream=None):
    """Network input of the warm start from CUDA tensors p (float64) and b
    (float32) of shape (nz, ny, nx).  Returns (x, s): x a CUDA float32
    tensor (nz/f, ny/f, nx/f, 2), s the scale of the network's output."""
    import torch
    nz, ny, nx = p.shape
    assert b.shape == p.shape
    x = torch.empty((nz // f, ny // f, nx // f, 2), dtype=torch.float32, device=p.device)
    s = C.c_double()
    N.check(N.lib().warm_start_features(nx, ny, nz, dx, int(f), N.tensor_ptr(p, "float64"), N.tensor_ptr(b, "float32"),
                                        N.tensor_ptr(x, "float32"), C.byref(s), N.stream_handle(stream)),
            "warm_start_features")
    return x, s.value


def warm_start_apply(out, scale: float, p, f: int, stream=None):
    """p += scale * prolong(out) in place; out CUDA float32 (nz/f, ny/f, nx/f),
    p CUDA float64 (nz, ny, nx)."""
    nz, ny, nx = p.shape
    assert tuple(out.shape) == (nz // f, ny // f, nx // f)
    N.check(N.lib().warm_start_apply(nx, ny, nz, int(f), N.tensor_ptr(out, "float32"), float(scale),
                                     N.tensor_ptr(p, "float64"), N.stream_handle(stream)), "warm_start_apply")
