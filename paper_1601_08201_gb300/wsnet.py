"""ctypes binding of the warm-start network (C ABI in include/wsnet.h).

Argument marshalling only: the network's forward, backward and optimiser
steps run in the CUDA kernels of libsgtv.so. Tensors are passed as device
addresses (e.g. torch_tensor.data_ptr()); parameter and gradient copies are
NumPy float32 arrays.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import sgtv

_P = ctypes.c_void_p
_lib = None


def load():
    global _lib
    if _lib is None:
        lib = sgtv.load()
        sig = {
            "wsnet_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_uint64, _P]),
            "wsnet_num_outputs": (ctypes.c_int32, [_P]),
            "wsnet_unpack_dual": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_float, _P, _P]),
            "wsnet_destroy": (ctypes.c_int, [_P]),
            "wsnet_num_params": (ctypes.c_int64, [_P]),
            "wsnet_get_params": (ctypes.c_int, [_P, _P]),
            "wsnet_set_params": (ctypes.c_int, [_P, _P]),
            "wsnet_get_grads": (ctypes.c_int, [_P, _P]),
            "wsnet_forward": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
            "wsnet_loss_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P]),
            "wsnet_adam_step": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
            "wsnet_pack_input": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                                ctypes.c_float, _P, _P]),
            "wsnet_unpack_output": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_float, _P, _P]),
            "wsnet_last_error": (ctypes.c_char_p, [_P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return ["wsnet_create", "wsnet_destroy", "wsnet_num_params", "wsnet_get_params", "wsnet_set_params",
            "wsnet_get_grads", "wsnet_forward", "wsnet_loss_grad", "wsnet_adam_step", "wsnet_pack_input",
            "wsnet_unpack_output", "wsnet_last_error", "wsnet_num_outputs", "wsnet_unpack_dual"]


class WarmNet:
    """The encoder-decoder of include/wsnet.h on the current device."""

    def __init__(self, H, W, Q, max_batch, seed=0, stream=None, n_dual=0):
        lib = load()
        self.h = ctypes.c_void_p()
        rc = lib.wsnet_create(ctypes.byref(self.h), H, W, Q, n_dual, max_batch, seed, stream)
        if rc:
            raise sgtv.SgtvError(rc, "wsnet_create failed")
        self.H, self.W, self.Q, self.max_batch, self.n_dual = H, W, Q, max_batch, n_dual

    @property
    def num_outputs(self):
        return int(load().wsnet_num_outputs(self.h))

    def _check(self, rc):
        if rc:
            raise sgtv.SgtvError(rc, load().wsnet_last_error(self.h).decode())

    @property
    def num_params(self):
        return int(load().wsnet_num_params(self.h))

    def get_params(self):
        a = np.empty(self.num_params, np.float32)
        self._check(load().wsnet_get_params(self.h, a.ctypes.data))
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, np.float32)
        assert a.size == self.num_params
        self._check(load().wsnet_set_params(self.h, a.ctypes.data))

    def get_grads(self):
        a = np.empty(self.num_params, np.float32)
        self._check(load().wsnet_get_grads(self.h, a.ctypes.data))
        return a

    def forward(self, x_ptr, n, out_ptr):
        self._check(load().wsnet_forward(self.h, x_ptr, n, out_ptr))

    def loss_grad(self, x_ptr, t_ptr, n):
        loss = ctypes.c_double()
        self._check(load().wsnet_loss_grad(self.h, x_ptr, t_ptr, n, ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(load().wsnet_adam_step(self.h, lr, beta1, beta2, eps))

    def close(self):
        if self.h:
            load().wsnet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_input(bp_ptr, Nx, Nz, Nq, scale, level, x_ptr, stream=None):
    rc = load().wsnet_pack_input(bp_ptr, Nx, Nz, Nq, scale, level, x_ptr, stream)
    if rc:
        raise sgtv.SgtvError(rc, "wsnet_pack_input")


def unpack_output(out_ptr, Nx, Nz, Nq, scale, f_ptr, stream=None):
    rc = load().wsnet_unpack_output(out_ptr, Nx, Nz, Nq, scale, f_ptr, stream)
    if rc:
        raise sgtv.SgtvError(rc, "wsnet_unpack_output")


def unpack_dual(out_ptr, Nx, Nz, Nq, n_dual, tau, c_ptr, stream=None):
    rc = load().wsnet_unpack_dual(out_ptr, Nx, Nz, Nq, n_dual, tau, c_ptr, stream)
    if rc:
        raise sgtv.SgtvError(rc, "wsnet_unpack_dual")
