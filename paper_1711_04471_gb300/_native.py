"""ctypes binding of libgbsw.so (argument marshalling only).

Every numerical step runs inside the CUDA library; this module converts
numpy arrays and torch streams/tensors to the plain pointers and sizes of
the C ABI declared in include/gbsw.h.  There is no fallback: if the library
is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbsw.so")

GBSW_OK = 0
GBSW_NOT_CONVERGED = 1

_lib = None


class GBSWError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = _lib
        name = L.gbsw_status_string(status).decode() if L else str(status)
        detail = L.gbsw_last_error().decode() if L else ""
        super().__init__(f"{where}: {name} ({status}) {detail}".strip())
        self.status = status


class SWParams(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dt", C.c_double), ("g", C.c_double), ("eps", C.c_double), ("hmin", C.c_double)]


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)


def _sig(L, name, res, args):
    f = getattr(L, name)
    f.restype = res
    f.argtypes = args


def _declare(L):
    _sig(L, "gbsw_status_string", C.c_char_p, [C.c_int])
    _sig(L, "gbsw_last_error", C.c_char_p, [])
    _sig(L, "gbsw_version", C.c_int, [])
    _sig(L, "sw_create", C.c_int, [C.POINTER(SWParams), _dp, _dp, _vp, C.POINTER(_vp)])
    _sig(L, "sw_step", C.c_int, [_vp, C.c_int])
    _sig(L, "sw_volume", C.c_int, [_vp, _dp, _dp])
    _sig(L, "sw_get_state", C.c_int, [_vp, _fp, _fp, _fp, C.POINTER(C.c_uint8)])
    _sig(L, "sw_set_state", C.c_int, [_vp, _fp, _fp, _fp])
    _sig(L, "sw_set_blocking", C.c_int, [_vp, C.c_int])
    _sig(L, "sw_set_tiling", C.c_int, [_vp, C.c_int, C.c_int])
    _sig(L, "sw_autotune", C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)])
    _sig(L, "sw_destroy", None, [_vp])
    _sig(L, "sw64_create", C.c_int, [C.POINTER(SWParams), _dp, _dp, _vp, C.POINTER(_vp)])
    _sig(L, "sw64_step", C.c_int, [_vp, C.c_int])
    _sig(L, "sw64_volume", C.c_int, [_vp, _dp, _dp])
    _sig(L, "sw64_get_state", C.c_int, [_vp, _dp, _dp, _dp, C.POINTER(C.c_uint8)])
    _sig(L, "sw64_destroy", None, [_vp])
    from . import _native_ext
    _native_ext.declare(L, _sig)


def lib():
    """Load libgbsw.so once (libgbsw_debug.so, the bounds-checked build, when
    the environment sets GBSW_DEBUG_BOUNDS=1); raise if it has not been
    built."""
    global _lib
    if _lib is None:
        path = LIB_PATH
        if os.environ.get("GBSW_DEBUG_BOUNDS") == "1":
            path = os.path.join(os.path.dirname(LIB_PATH), "libgbsw_debug.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1711_04471_gb300.build.build()")
        L = C.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def check(status: int, where: str) -> int:
    if status < 0:
        raise GBSWError(status, where)
    return status


def ptr(a: np.ndarray | None, ctype):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(ctype))


def stream_handle(stream) -> int | None:
    """cudaStream_t of a torch.cuda.Stream, an int handle, or None."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def tensor_ptr(t, dtype_name: str):
    """Device pointer of a contiguous torch tensor of the given dtype."""
    import torch
    want = {"float32": torch.float32, "float64": torch.float64, "bfloat16": torch.bfloat16,
            "uint8": torch.uint8, "int32": torch.int32}[dtype_name]
    if t.dtype != want or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"expected a contiguous CUDA {dtype_name} tensor")
    return C.c_void_p(t.data_ptr())
