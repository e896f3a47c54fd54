"""FP64 CPU oracle for the improved MRT pseudopotential LB method (arXiv:1211.6932).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this package.  It shares no code with the CUDA library.

Contents
--------
``Params``                       -- one run's physical and numerical parameters.
``run(params, f, nsteps)``       -- advance populations (Q, ny, nx) by nsteps (Eqs. 1-7, 25).
``fields(params, f)``            -- rho, v (Eq. 6), psi (Eq. 24), F (Eq. 7) at the current time.
``equilibrium(rho, ux, uy)``     -- f = M^{-1} m_eq (Eq. 3).
``tables()``                     -- the oracle's own lattice tables.
``thermo``                       -- CS EOS, Maxwell rule, mechanical stability, Lamb period.
"""
import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build
from . import thermo  # noqa: F401  (re-exported)

Q = 9
_LIB = None


class _CParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("T", ctypes.c_double), ("G", ctypes.c_double), ("sigma", ctypes.c_double),
        ("s", ctypes.c_double * Q), ("visc_mode", ctypes.c_int),
        ("nu_l", ctypes.c_double), ("nu_v", ctypes.c_double), ("rho_c", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double), ("walls", ctypes.c_int),
    ]


VISC_CONST, VISC_STEP, VISC_LINEAR = 0, 1, 2


@dataclasses.dataclass
class Params:
    """Parameters of one lattice (lattice units, c = delta_t = 1)."""
    nx: int
    ny: int
    a: float = 0.25
    b: float = 4.0
    R: float = 1.0
    T: float = 0.0
    G: float = -1.0
    sigma: float = 0.0
    s: tuple = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)
    visc_mode: int = VISC_CONST
    nu_l: float = 0.0
    nu_v: float = 0.0
    rho_c: float = 0.0
    rho_l: float = 0.0
    rho_v: float = 0.0
    walls: bool = False

    def to_c(self) -> _CParams:
        c = _CParams()
        for k in ("nx", "ny", "visc_mode"):
            setattr(c, k, int(getattr(self, k)))
        for k in ("a", "b", "R", "T", "G", "sigma", "nu_l", "nu_v", "rho_c", "rho_l", "rho_v"):
            setattr(c, k, float(getattr(self, k)))
        c.walls = int(bool(self.walls))
        if len(self.s) != Q:
            raise ValueError("s must have 9 rates")
        for i in range(Q):
            c.s[i] = float(self.s[i])
        return c


def lib():
    """Load (building first if needed) the oracle's shared object.  LBM_ORACLE_LIB, when
    set, names another build of it to load instead (the mutation check of the pins loads
    altered copies this way)."""
    global _LIB
    if _LIB is None:
        path = os.environ.get("LBM_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_run.argtypes = [ctypes.POINTER(_CParams), dp, dp, ctypes.c_int]
        L.oracle_run.restype = ctypes.c_int
        L.oracle_fields.argtypes = [ctypes.POINTER(_CParams), dp, dp, dp, dp, dp, dp, dp]
        L.oracle_fields.restype = ctypes.c_int
        L.oracle_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.oracle_equilibrium.restype = ctypes.c_int
        L.oracle_tables.argtypes = [ip, ip, ip, dp, dp]
        L.oracle_tables.restype = None
        L.oracle_p_eos.argtypes = [ctypes.c_double] * 5
        L.oracle_p_eos.restype = ctypes.c_double
        L.oracle_psi.argtypes = [ctypes.c_double] * 6
        L.oracle_psi.restype = ctypes.c_double
        L.oracle_threads.argtypes = []
        L.oracle_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def run(params: Params, f, nsteps: int):
    """Advance populations f (Q, ny, nx) by ``nsteps`` steps; returns a new array."""
    f = _c64(f, (Q, params.ny, params.nx))
    out = np.empty_like(f)
    cp = params.to_c()
    rc = lib().oracle_run(ctypes.byref(cp), _dptr(f), _dptr(out), int(nsteps))
    if rc != 0:
        raise RuntimeError("oracle_run failed with %d" % rc)
    return out


def fields(params: Params, f):
    """Return dict rho, ux, uy, psi, Fx, Fy (each (ny, nx)) at the current time."""
    f = _c64(f, (Q, params.ny, params.nx))
    names = ("rho", "ux", "uy", "psi", "Fx", "Fy")
    out = {k: np.empty((params.ny, params.nx)) for k in names}
    cp = params.to_c()
    rc = lib().oracle_fields(ctypes.byref(cp), _dptr(f), *[_dptr(out[k]) for k in names])
    if rc != 0:
        raise RuntimeError("oracle_fields failed with %d" % rc)
    return out


def equilibrium(rho, ux=None, uy=None):
    """Populations whose moments are the equilibria of Eq. 3, shape (Q, ny, nx)."""
    rho = _c64(rho)
    ny, nx = rho.shape
    ux = np.zeros_like(rho) if ux is None else _c64(ux, rho.shape)
    uy = np.zeros_like(rho) if uy is None else _c64(uy, rho.shape)
    f = np.empty((Q, ny, nx))
    rc = lib().oracle_equilibrium(nx, ny, _dptr(rho), _dptr(ux), _dptr(uy), _dptr(f))
    if rc != 0:
        raise RuntimeError("oracle_equilibrium failed with %d" % rc)
    return f


def tables():
    """The oracle's velocities, opposite map, force weights w and matrix M."""
    ex = (ctypes.c_int * Q)()
    ey = (ctypes.c_int * Q)()
    opp = (ctypes.c_int * Q)()
    w = (ctypes.c_double * Q)()
    m = (ctypes.c_double * (Q * Q))()
    lib().oracle_tables(ex, ey, opp, w, m)
    return {
        "ex": np.array(ex[:], dtype=np.int64), "ey": np.array(ey[:], dtype=np.int64),
        "opp": np.array(opp[:], dtype=np.int64), "w": np.array(w[:]),
        "M": np.array(m[:]).reshape(Q, Q),
    }


def p_eos(rho, a, b, R, T):
    """Carnahan-Starling pressure (Eq. 30), evaluated by the C oracle."""
    return lib().oracle_p_eos(float(rho), a, b, R, T)


def psi(rho, a, b, R, T, G):
    """Pseudopotential of Eq. 24, evaluated by the C oracle."""
    return lib().oracle_psi(float(rho), a, b, R, T, G)


def threads() -> int:
    return lib().oracle_threads()


def rates_for(tau_nu, s_e=1.1, s_zeta=1.1, s_q=1.1):
    """Rate vector of Eq. 2 with s_rho = s_j = 1 and the stress rate 1/tau_nu."""
    sn = 1.0 / tau_nu
    return (1.0, s_e, s_zeta, 1.0, s_q, 1.0, s_q, sn, sn)


__all__ = ["Params", "run", "fields", "equilibrium", "tables", "p_eos", "psi", "thermo",
           "threads", "rates_for", "VISC_CONST", "VISC_STEP", "VISC_LINEAR", "Q"]
