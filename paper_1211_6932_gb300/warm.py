"""Python front end of the warm-start helpers (include/lbm_warm.h).  Marshalling only."""
import ctypes
import dataclasses

import numpy as np

from . import _lib as C
from .lattice import Eos, LbmError


@dataclasses.dataclass
class WarmParams:
    """Equilibrium quantities of one run (definitions in include/lbm_warm.h)."""
    rho_l: float
    rho_v: float
    width: float
    shift: float = 0.0
    curvature: float = 0.0

    def c(self):
        return C.lbm_warm_params(self.rho_l, self.rho_v, self.width, self.shift, self.curvature)

    @classmethod
    def of(cls, w):
        return cls(w.rho_l, w.rho_v, w.width, w.shift, w.curvature)


def _field(rho):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if rho.ndim != 2:
        raise ValueError("rho must be (ny, nx)")
    return rho


def _ok(rc, what):
    if rc != 0:
        raise LbmError(rc, what)


def measure_film(rho):
    rho = _field(rho)
    out = C.lbm_warm_params()
    _ok(C.lib().lbm_measure_film(rho.ctypes.data_as(C.dptr), rho.shape[1], rho.shape[0],
                                 ctypes.byref(out)), "film measurement failed")
    return WarmParams.of(out)


def measure_droplet(rho, eos: Eos):
    """(rho_in, rho_out, equimolar radius, Laplace-law surface tension) of a centred
    droplet."""
    rho = _field(rho)
    v = [ctypes.c_double() for _ in range(4)]
    _ok(C.lib().lbm_measure_droplet(rho.ctypes.data_as(C.dptr), rho.shape[1], rho.shape[0],
                                    eos.c(), *[ctypes.byref(x) for x in v]),
        "droplet measurement failed")
    return tuple(x.value for x in v)


def encode(eos: Eos, p: WarmParams):
    y = np.empty(5)
    _ok(C.lib().lbm_warm_encode(eos.c(), ctypes.byref(p.c()), y.ctypes.data_as(C.dptr)),
        "encode failed")
    return y


def decode(eos: Eos, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = C.lbm_warm_params()
    _ok(C.lib().lbm_warm_decode(eos.c(), y.ctypes.data_as(C.dptr), ctypes.byref(out)),
        "decode failed")
    return WarmParams.of(out)


def vapour_law(r1, ro1, r2, ro2):
    """(rho_v, curvature) of rho_out(R) = rho_v (1 + curvature / R) through two droplets."""
    rv, k = ctypes.c_double(), ctypes.c_double()
    _ok(C.lib().lbm_vapour_law(float(r1), float(ro1), float(r2), float(ro2), ctypes.byref(rv),
                               ctypes.byref(k)), "vapour law needs two distinct radii")
    return rv.value, k.value


def curved_densities(eos: Eos, p: WarmParams, kappa):
    """(rho_in, rho_out) around droplets of mean curvature kappa."""
    ri, ro = ctypes.c_double(), ctypes.c_double()
    _ok(C.lib().lbm_curved_densities(eos.c(), ctypes.byref(p.c()), float(kappa),
                                     ctypes.byref(ri), ctypes.byref(ro)),
        "curved-interface densities failed")
    return ri.value, ro.value
