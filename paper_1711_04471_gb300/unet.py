"""Warm-start U-Net for the pressure solve (thin wrapper of the unet_*
entry points of libgbsw.so).  Parameters are exchanged as one flat FP32
vector in the order documented in include/gbsw.h."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N

LAYERS = [("l1a", 2, 16), ("l1b", 16, 16), ("l2a", 16, 32), ("l2b", 32, 32), ("l3a", 32, 64), ("l3b", 64, 32),
          ("l2c", 64, 16), ("l1c", 32, 16)]


def unflatten(flat: np.ndarray) -> dict:
    """Flat parameter vector -> {name.w: (27, cout, cin), name.b: (cout,), head.w: (1, 16), head.b: (1,)}."""
    P, o = {}, 0
    for name, ci, co in LAYERS:
        n = 27 * co * ci
        P[name + ".w"] = flat[o:o + n].reshape(27, co, ci)
        o += n
        P[name + ".b"] = flat[o:o + co]
        o += co
    P["head.w"] = flat[o:o + 16].reshape(1, 16)
    P["head.b"] = flat[o + 16:o + 17]
    assert o + 17 == flat.size
    return P


def flatten(P: dict) -> np.ndarray:
    parts = []
    for name, _, _ in LAYERS:
        parts += [np.ravel(P[name + ".w"]), np.ravel(P[name + ".b"])]
    parts += [np.ravel(P["head.w"]), np.ravel(P["head.b"])]
    return np.concatenate(parts).astype(np.float32)


class UNet:
    def __init__(self, seed: int = 0, stream=None):
        h = C.c_void_p()
        N.check(N.lib().unet_create(int(seed), N.stream_handle(stream), C.byref(h)), "unet_create")
        self._h = h
        self.n_params = N.lib().unet_num_params()

    def get_params(self) -> np.ndarray:
        a = np.empty(self.n_params, np.float32)
        N.check(N.lib().unet_get_params(self._h, a.ctypes.data_as(C.c_void_p), self.n_params), "unet_get_params")
        return a

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        N.check(N.lib().unet_set_params(self._h, a.ctypes.data_as(C.c_void_p), self.n_params), "unet_set_params")

    def forward(self, x):
        """x: CUDA float32 (n, D, H, W, 2) -> CUDA float32 (n, D, H, W)."""
        import torch
        n, D, H, W, _ = x.shape
        y = torch.empty((n, D, H, W), dtype=torch.float32, device=x.device)
        N.check(N.lib().unet_forward(self._h, n, D, H, W, N.tensor_ptr(x, "float32"), N.tensor_ptr(y, "float32")),
                "unet_forward")
        return y

    def gradients(self, x, target):
        n, D, H, W, _ = x.shape
        g = np.empty(self.n_params, np.float32)
        loss = C.c_double()
        N.check(N.lib().unet_gradients(self._h, n, D, H, W, N.tensor_ptr(x, "float32"), N.tensor_ptr(target, "float32"),
                                       g.ctypes.data_as(C.c_void_p), C.byref(loss)), "unet_gradients")
        return loss.value, g

    def train_step(self, x, target, lr: float) -> float:
        n, D, H, W, _ = x.shape
        loss = C.c_double()
        N.check(N.lib().unet_train_step(self._h, n, D, H, W, N.tensor_ptr(x, "float32"),
                                        N.tensor_ptr(target, "float32"), float(lr), C.byref(loss)), "unet_train_step")
        return loss.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().unet_destroy(self._h)
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
