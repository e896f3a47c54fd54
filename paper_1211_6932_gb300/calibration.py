"""Calibration of the improved forcing's sigma against the Maxwell rule.

Two routes, both against the vapour density of Eq. 22 (the sensitive branch):

* ``sigma_eq21``: the continuum route, lbm_sigma_consistent: the sigma for which the
  mechanical-stability condition (Eq. 21 with eps of Eq. 29) gives the Maxwell vapour
  density.  Host only, fast.
* ``sigma_lattice``: the lattice route: flat films (4 x 128, rates of Sec. IV A with
  tau_nu = 0.8) in one batch per round, `k` trial sigmas per (a, T/Tc) inside the current
  bracket; a trial's film vapour density (window-averaged after `steps` steps) above the
  Maxwell value moves the upper end of the bracket down, below moves the lower end up
  (the film vapour density rises with sigma).  The result interpolates ln(rho_v/rho_v^M)
  linearly between the final bracket ends.  Below T/Tc ~ 0.7 the two routes part: the
  interfaces are a few nodes wide and the lattice no longer follows the continuum
  condition.

This module sequences library calls; all arithmetic runs in the library.
"""
import dataclasses
import math

import numpy as np

from . import workloads as wl
from .coexistence import rates
from .lattice import Batch, Eos, Instance, maxwell, sigma_consistent
from .warm import measure_film


def sigma_eq21(a, t_over_tc, G=-1.0):
    return sigma_consistent(Eos(a=a, T=t_over_tc * wl.t_crit(a)), G)


@dataclasses.dataclass
class Calibration:
    a: float
    t_over_tc: float
    sigma: float        # interpolated root (nan if never bracketed)
    lo: float           # largest trial sigma with the film vapour below Maxwell
    hi: float           # smallest trial sigma with the film vapour above Maxwell
    h_lo: float         # ln(rho_v / rho_v^M) at lo
    h_hi: float         # ... at hi


def _film_vapour_logratio(trials, tau_nu, steps, avg_samples, avg_stride, stream):
    """trials: (a, t_over_tc, sigma); ln(film rho_v / Maxwell rho_v) per trial (nan when
    the film went unstable)."""
    insts, fields, mv = [], [], []
    for a, tr, sig in trials:
        eos = Eos(a=a, T=tr * wl.t_crit(a))
        rl, rv = maxwell(eos)
        mv.append(rv)
        insts.append(Instance(nx=4, ny=128, eos=eos, sigma=sig, s=rates(tau_nu),
                              visc_mode="const", rho_l=rl, rho_v=rv))
        fields.append(wl.flat_film(4, 128, rl, rv, 5.0, 64.0))
    b = Batch(insts, precision="fp32", stream=stream)
    try:
        for i, f in enumerate(fields):
            b.init_fields(i, f)
        b.step(steps)
        acc = [np.zeros((128, 4)) for _ in insts]
        for _ in range(avg_samples):
            b.step(avg_stride)
            for i in range(len(insts)):
                acc[i] += b.density(i)
        diag = b.diagnostics()
    finally:
        b.close()
    out = []
    for i in range(len(insts)):
        h = float("nan")
        if diag[i]["nonfinite"] == 0:
            try:
                h = math.log(measure_film(acc[i] / avg_samples).rho_v / mv[i])
            except Exception:
                pass
        out.append(h)
    return out


GRID = (0.06, 0.08, 0.09, 0.10, 0.11, 0.12, 0.13, 0.15, 0.18, 0.22)


def sigma_lattice(points, grid=GRID, k=4, rounds=4, tau_nu=0.8, steps=40000, avg_samples=10,
                  avg_stride=100, stream=None):
    """points: (a, t_over_tc) pairs; returns one Calibration per point.  A first batch
    runs every grid sigma for every point (small sigmas blow up at low temperatures:
    those trials are left out); the bracket is the sign change among the stable ones."""
    st = [Calibration(a, tr, float("nan"), float("nan"), float("nan"), float("nan"),
                      float("nan")) for a, tr in points]
    hs = _film_vapour_logratio([(c.a, c.t_over_tc, g) for c in st for g in grid],
                               tau_nu, steps, avg_samples, avg_stride, stream)
    for j, c in enumerate(st):
        ok = [(g, h) for g, h in zip(grid, hs[j * len(grid):(j + 1) * len(grid)])
              if not math.isnan(h)]
        for (g0, h0), (g1, h1) in zip(ok[:-1], ok[1:]):
            if h0 < 0.0 <= h1:
                c.lo, c.h_lo, c.hi, c.h_hi = g0, h0, g1, h1
                break
    for _ in range(rounds):
        live = [c for c in st if c.h_lo < 0.0 < c.h_hi]
        if not live:
            break
        trials = []
        for c in live:
            trials += [(c.a, c.t_over_tc, c.lo + (c.hi - c.lo) * (i + 1) / (k + 1))
                       for i in range(k)]
        hs = _film_vapour_logratio(trials, tau_nu, steps, avg_samples, avg_stride, stream)
        for j, c in enumerate(live):
            for (_, _, sig), h in zip(trials[j * k:(j + 1) * k], hs[j * k:(j + 1) * k]):
                if math.isnan(h):
                    continue
                if h < 0.0 and sig > c.lo:
                    c.lo, c.h_lo = sig, h
                elif h >= 0.0 and sig < c.hi:
                    c.hi, c.h_hi = sig, h
    for c in st:
        if c.h_lo < 0.0 < c.h_hi:
            c.sigma = c.lo + (c.hi - c.lo) * (-c.h_lo) / (c.h_hi - c.h_lo)
    return st
