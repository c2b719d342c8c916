"""Python binding of the autofocus network's C ABI (include/hv_af.h): argument
marshalling only, every step runs in libhv.so."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import hv

NPARAMS = 62337
SIDE = 128


class hv_af_desc(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("device", C.c_int), ("max_batch", C.c_uint32),
                ("reserved", C.c_uint32), ("stream", C.c_void_p)]


class hv_af_adam(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


_done = False


def _lib():
    global _done
    L = hv.lib()
    if not _done:
        P = C.POINTER
        sig = {
            "hv_af_open": ([P(hv_af_desc), P(C.c_void_p)], C.c_int),
            "hv_af_set_params": ([C.c_void_p, P(C.c_float), C.c_size_t], C.c_int),
            "hv_af_get_params": ([C.c_void_p, P(C.c_float), C.c_size_t], C.c_int),
            "hv_af_forward": ([C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p], C.c_int),
            "hv_af_loss_grad": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p],
                                C.c_int),
            "hv_af_train_step": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, P(hv_af_adam), C.c_void_p],
                                 C.c_int),
            "hv_af_synchronize": ([C.c_void_p], C.c_int),
            "hv_af_last_error": ([C.c_void_p], C.c_char_p),
            "hv_af_close": ([C.c_void_p], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _done = True
    return L


def _dev(t, what):
    ptr, kind, nbytes = hv._ptr_kind(t)
    if kind != hv.HV_MEM_DEVICE:
        raise ValueError(f"{what} must be device memory")
    return C.c_void_p(ptr), nbytes


class Autofocus:
    """One network on one device; tensors passed in are CUDA tensors."""

    def __init__(self, max_batch, device=0, stream=None):
        d = hv_af_desc(C.sizeof(hv_af_desc), device, max_batch, 0, C.c_void_p(stream or 0))
        self.h = C.c_void_p()
        s = _lib().hv_af_open(C.byref(d), C.byref(self.h))
        if s != hv.HV_OK:
            raise hv.HvError(s, "hv_af_open failed")
        self.max_batch = max_batch

    def _check(self, s):
        if s != hv.HV_OK:
            raise hv.HvError(s, _lib().hv_af_last_error(self.h).decode(errors="replace"))

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(_lib().hv_af_set_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size))

    def get_params(self) -> np.ndarray:
        a = np.zeros(NPARAMS, dtype=np.float32)
        self._check(_lib().hv_af_get_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), a.size))
        return a

    def forward(self, x, z_out):
        xp, _ = _dev(x, "x")
        zp, _ = _dev(z_out, "z_out")
        self._check(_lib().hv_af_forward(self.h, xp, x.shape[0], zp))

    def loss_grad(self, x, z_target, loss, grad=None):
        xp, _ = _dev(x, "x")
        tp, _ = _dev(z_target, "z_target")
        lp, _ = _dev(loss, "loss")
        gp = _dev(grad, "grad")[0] if grad is not None else None
        self._check(_lib().hv_af_loss_grad(self.h, xp, tp, x.shape[0], lp, gp))

    def train_step(self, x, z_target, loss=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        xp, _ = _dev(x, "x")
        tp, _ = _dev(z_target, "z_target")
        lp = _dev(loss, "loss")[0] if loss is not None else None
        opt = hv_af_adam(lr, beta1, beta2, eps)
        self._check(_lib().hv_af_train_step(self.h, xp, tp, x.shape[0], C.byref(opt), lp))

    def synchronize(self):
        """Wait for the network's work; raises if a device wait gave up."""
        self._check(_lib().hv_af_synchronize(self.h))

    def close(self):
        if self.h is not None and self.h.value:
            _lib().hv_af_close(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
