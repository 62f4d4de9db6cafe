"""ctypes binding of the warm-start network (include/hcran_mlp.h): argument
marshalling only; every step runs in the library's tensor-core kernels."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import hcran

IN, HIDDEN, OUT, FEATURES = 16, 256, 16, 4


def _check(fn: str, rc: int):
    if rc != 0:
        raise RuntimeError("%s failed with code %d" % (fn, rc))


class MLP:
    """The network on the current CUDA device (FP32 master weights, BF16 copies)."""

    def __init__(self, seed: int = 0, max_rows: int = 1 << 16):
        self.lib = hcran.load()
        self.h = C.c_void_p()
        _check("hcran_mlp_create", self.lib.hcran_mlp_create(C.byref(self.h), seed, max_rows))
        n = C.c_int64()
        _check("hcran_mlp_param_count", self.lib.hcran_mlp_param_count(self.h, C.byref(n)))
        self.n_params = n.value
        self.max_rows = max_rows

    def close(self):
        if self.h:
            self.lib.hcran_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        a = np.zeros(self.n_params, np.float32)
        _check("hcran_mlp_get_params", self.lib.hcran_mlp_get_params(self.h, a.ctypes.data_as(hcran._fp)))
        return a

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == self.n_params
        _check("hcran_mlp_set_params", self.lib.hcran_mlp_set_params(self.h, a.ctypes.data_as(hcran._fp)))

    def grads(self) -> np.ndarray:
        a = np.zeros(self.n_params, np.float32)
        _check("hcran_mlp_get_grads", self.lib.hcran_mlp_get_grads(self.h, a.ctypes.data_as(hcran._fp)))
        return a

    def forward(self, x, out, stream=None):
        """x: [T][16] bfloat16 CUDA tensor, out: [T][16] float32 CUDA tensor."""
        _check("hcran_mlp_forward", self.lib.hcran_mlp_forward(
            self.h, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(out.data_ptr()), _st(stream)))

    def loss_grad(self, out, target, mask, loss, nout: int = 3, stream=None):
        _check("hcran_mlp_loss_grad", self.lib.hcran_mlp_loss_grad(
            self.h, C.c_void_p(out.data_ptr()), C.c_void_p(target.data_ptr()), C.c_void_p(mask.data_ptr()),
            out.shape[0], nout, C.c_void_p(loss.data_ptr()), _st(stream)))

    def backward(self, x, stream=None):
        _check("hcran_mlp_backward", self.lib.hcran_mlp_backward(
            self.h, C.c_void_p(x.data_ptr()), x.shape[0], _st(stream)))

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
        _check("hcran_mlp_adam", self.lib.hcran_mlp_adam(self.h, lr, beta1, beta2, eps, _st(stream)))

    def tc_failed(self) -> bool:
        f = C.c_int32()
        _check("hcran_mlp_tc_status", self.lib.hcran_mlp_tc_status(C.byref(f)))
        return bool(f.value)


def _st(stream):
    return C.c_void_p(stream.cuda_stream) if stream is not None else None
