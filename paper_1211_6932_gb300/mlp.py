"""Python front end of the warm-start network (include/lbm_mlp.h).  Marshalling only: the
forward, backward and Adam steps run in the CUDA library."""
import ctypes

import numpy as np

from . import _lib as C
from .lattice import LbmError, _device_of, _stream_ptr

NPARAMS = C.LBM_MLP_NPARAMS
N_IN, N_OUT = 4, 5


def _f32(a, n):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.shape != (n,):
        raise ValueError("expected %d floats, got shape %s" % (n, a.shape))
    return a


def _rows(a, cols):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != cols:
        raise ValueError("expected an (n, %d) array, got shape %s" % (cols, a.shape))
    return a


def _fp(a):
    return a.ctypes.data_as(C.fptr)


def _dp(a):
    return a.ctypes.data_as(C.dptr)


class Mlp:
    """The 4 -> 64 -> 64 -> 5 GELU network (lbm_mlp_create ... lbm_mlp_destroy).

    params: initial master weights (NPARAMS floats, packed W1, b1, W2, b2, W3, b3)."""

    def __init__(self, params, max_rows=4096, stream=None, device=None):
        self._L = C.lib()
        self._h = None
        h = ctypes.c_void_p()
        p = _f32(params, NPARAMS)
        rc = self._L.lbm_mlp_create(ctypes.byref(h), _fp(p), int(max_rows), _stream_ptr(stream),
                                    _device_of(stream, device))
        if rc != 0:
            raise LbmError(rc, self._L.lbm_mlp_last_error(None).decode())
        self._h = h
        self.max_rows = int(max_rows)

    def _check(self, rc):
        if rc != 0:
            raise LbmError(rc, self._L.lbm_mlp_last_error(self._h).decode())

    def close(self):
        if self._h is not None:
            self._L.lbm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_scaling(self, in_mean, in_scale, out_mean, out_scale):
        arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in
                (in_mean, in_scale, out_mean, out_scale)]
        self._check(self._L.lbm_mlp_set_scaling(self._h, *[_dp(a) for a in arrs]))

    def fit_scaling(self, x, t):
        x, t = _rows(x, N_IN), _rows(t, N_OUT)
        self._check(self._L.lbm_mlp_fit_scaling(self._h, _dp(x), _dp(t), x.shape[0]))

    def set_data(self, x, t):
        x, t = _rows(x, N_IN), _rows(t, N_OUT)
        if x.shape[0] != t.shape[0]:
            raise ValueError("x and t differ in rows")
        self._check(self._L.lbm_mlp_set_data(self._h, _dp(x), _dp(t), x.shape[0]))

    def train(self, steps, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """Full-batch Adam updates; returns the loss before each update."""
        opt = C.lbm_adam(lr, beta1, beta2, eps)
        losses = np.empty(max(int(steps), 0), dtype=np.float32)
        self._check(self._L.lbm_mlp_train(self._h, int(steps), ctypes.byref(opt),
                                          _fp(losses) if steps > 0 else None))
        return losses

    def gradient(self):
        g = np.empty(NPARAMS, dtype=np.float32)
        L = ctypes.c_float()
        self._check(self._L.lbm_mlp_gradient(self._h, _fp(g), ctypes.byref(L)))
        return L.value, g

    def predict(self, x):
        x = _rows(x, N_IN)
        y = np.empty((x.shape[0], N_OUT))
        self._check(self._L.lbm_mlp_predict(self._h, _dp(x), x.shape[0], _dp(y)))
        return y

    def params(self, which="master"):
        k = {"master": 0, "bf16": 1, "m": 2, "v": 3}[which]
        out = np.empty(NPARAMS, dtype=np.float32)
        self._check(self._L.lbm_mlp_get_params(self._h, k, _fp(out)))
        return out

    def set_params(self, values, which="master"):
        k = {"master": 0, "m": 2, "v": 3}[which]
        v = _f32(values, NPARAMS)
        self._check(self._L.lbm_mlp_set_params(self._h, k, _fp(v)))

    @property
    def update_count(self):
        return int(self._L.lbm_mlp_update_count(self._h))
