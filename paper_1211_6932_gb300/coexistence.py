"""Coexistence curves of the original and the improved forcing scheme (Sec. IV A, Fig. 1).

Flat films (x-uniform, liquid in the middle half) at a range of reduced temperatures,
for each forcing (sigma = 0: the original scheme; sigma > 0: Eq. 25) and each stress
relaxation time, all advance together in one batch (lbm_batch_*).  After a fixed number
of steps the density is averaged over a window and the film and vapour centre densities
are read off (lbm_measure_film).  Instances whose density became non-finite are reported
unstable: the lowest stable reduced temperature of each scheme is the paper's measure of
its reach.  The paper reads its curve off stationary droplets; flat films give the
flat-interface coexistence that the Maxwell rule (Eq. 22) and the mechanical-stability
condition (Eq. 21) describe, without a Laplace shift.

This module sequences library calls; all arithmetic runs in the library.
"""
import dataclasses

import numpy as np

from . import workloads as wl
from .lattice import Batch, Eos, Instance, maxwell
from .warm import measure_film

T_OVER_TC = (0.49, 0.5, 0.55, 0.6, 0.65, 0.7, 0.75, 0.8, 0.85, 0.9, 0.95)


def rates(tau_nu, s_e=1.1, s_zeta=1.1, s_q=1.1):
    """Relaxation rates of Sec. IV A: tau_rho = tau_j = 1, s_e = s_zeta = s_q = 1.1 and
    the stress rates 1 / tau_nu."""
    sn = 1.0 / tau_nu
    return (1.0, s_e, s_zeta, 1.0, s_q, 1.0, s_q, sn, sn)


@dataclasses.dataclass
class Point:
    sigma: float
    tau_nu: float
    t_over_tc: float
    stable: bool
    rho_l: float       # film centre (nan when unstable)
    rho_v: float       # vapour centre (nan when unstable)
    maxwell_l: float
    maxwell_v: float


def sweep(a=0.5, t_over_tc=T_OVER_TC, sigmas=(0.0, 0.11), taus=(0.6, 0.8), nx=4, ny=128,
          width=5.0, steps=40000, avg_samples=10, avg_stride=100, precision="fp32",
          stream=None):
    """One film per (sigma, tau_nu, T/Tc); returns the Points in that nesting order."""
    keys, insts, fields = [], [], []
    for sig in sigmas:
        for tau in taus:
            for tr in t_over_tc:
                eos = Eos(a=a, T=tr * wl.t_crit(a))
                rl, rv = maxwell(eos)
                keys.append((sig, tau, tr, rl, rv))
                insts.append(Instance(nx=nx, ny=ny, eos=eos, sigma=sig, s=rates(tau),
                                      visc_mode="const", rho_l=rl, rho_v=rv))
                fields.append(wl.flat_film(nx, ny, rl, rv, width, ny / 2.0))
    b = Batch(insts, precision=precision, stream=stream)
    try:
        for i, f in enumerate(fields):
            b.init_fields(i, f)
        b.step(steps)
        acc = [np.zeros((ny, nx)) for _ in insts]
        for _ in range(avg_samples):
            b.step(avg_stride)
            for i in range(len(insts)):
                acc[i] += b.density(i)
        diag = b.diagnostics()
    finally:
        b.close()
    out = []
    for i, (sig, tau, tr, rl, rv) in enumerate(keys):
        ok = diag[i]["nonfinite"] == 0 and np.all(np.isfinite(acc[i]))
        fl = fv = float("nan")
        if ok:
            try:
                m = measure_film(acc[i] / avg_samples)
                fl, fv = m.rho_l, m.rho_v
            except Exception:  # no longer a film (the interfaces merged or vanished)
                ok = False
        out.append(Point(sig, tau, tr, bool(ok), fl, fv, rl, rv))
    return out


def lowest_stable(points, sigma, tau):
    """Lowest reduced temperature from which on every warmer film of (sigma, tau) stayed
    stable."""
    pts = sorted((p for p in points if p.sigma == sigma and p.tau_nu == tau),
                 key=lambda p: p.t_over_tc)
    low = None
    for p in reversed(pts):
        if not p.stable:
            break
        low = p.t_over_tc
    return low
