"""Declarations of the later-added C-ABI entry points (see include/gbsw.h)."""
import ctypes as C


def declare(L, sig):
    vp, fp, dp = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_double)
    sig(L, "sw_volume_noalloc", C.c_int,
        [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, vp, vp, vp, vp])
