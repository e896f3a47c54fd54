"""Physics checks of the dynamics on the GPU path (Sec. IV A-C): the Laplace law, the
oscillation period of an elliptic droplet against Lamb's Eq. 32, and the spread of a
splash against the power law r/D = C sqrt(U t / D).

Each function runs library calls (single lattices or one batch) and reduces the density
fields it reads back; the reductions are measurements, not part of the step.
"""
import dataclasses
import math

import numpy as np

from . import workloads as wl
from .lattice import Batch, Eos, Instance, Lattice, maxwell
from .warm import measure_droplet

RATES_TAU08 = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25)  # Sec. IV A, tau_nu = 0.8


@dataclasses.dataclass
class LaplaceFit:
    radii: np.ndarray     # equimolar radii
    dp: np.ndarray        # p(rho_in) - p(rho_out)
    gamma: float          # slope of dp against 1/R
    intercept: float
    r2: float


def laplace_law(a=0.25, t_over_tc=0.7, sigma=0.114, radii=(15.0, 20.0, 25.0, 30.0, 40.0),
                tol=1e-6, max_steps=80000, stream=None):
    """Droplets of several radii (128^2 boxes up to R = 30, 256^2 above) in one batch, run
    until their densities settle; dp against 1/R by least squares."""
    return laplace_law_at(Eos(a=a, T=t_over_tc * wl.t_crit(a)), sigma, radii, tol, max_steps,
                          stream)


def laplace_law_at(eos, sigma, radii=(15.0, 20.0, 25.0, 30.0, 40.0), tol=1e-6,
                   max_steps=80000, stream=None):
    rl, rv = maxwell(eos)
    insts, fields = [], []
    for r in radii:
        n = 128 if r <= 30 else 256
        insts.append(Instance(nx=n, ny=n, eos=eos, sigma=sigma, s=RATES_TAU08, rho_l=rl,
                              rho_v=rv))
        fields.append(wl.droplet(n, n, rl, rv, r, 4.0))
    b = Batch(insts, precision="fp32", stream=stream)
    try:
        for i, f in enumerate(fields):
            b.init_fields(i, f)
        b.run_to_equilibrium(tol, 100, max_steps)
        meas = [measure_droplet(b.density(i), eos) for i in range(len(insts))]
    finally:
        b.close()
    R = np.array([m[2] for m in meas])
    dp = np.array([m[3] / m[2] for m in meas])
    x = 1.0 / R
    A = np.column_stack([x, np.ones_like(x)])
    (g, c), *_ = np.linalg.lstsq(A, dp, rcond=None)
    pred = A @ np.array([g, c])
    r2 = 1.0 - np.sum((dp - pred) ** 2) / np.sum((dp - dp.mean()) ** 2)
    return LaplaceFit(R, dp, float(g), float(c), float(r2))


@dataclasses.dataclass
class Oscillation:
    period: float        # measured, in steps (mean spacing of upward zero crossings)
    lamb: float          # Eq. 32, n = 2, with R0 = sqrt(ax ay), the centre liquid density
    r0: float
    rho_l: float
    gamma: float
    crossings: int
    signal: np.ndarray   # I_xx - I_yy of the liquid excess, every `every` steps


def ellipse_period(n=200, ax=30.0, ay=27.0, a=0.5, t_over_tc=0.5, tc=0.047, sigma=0.11,
                   nu_l=0.05, nu_v=0.3, visc_mode="step", steps=10400, every=20, gamma=None,
                   stream=None):
    """An elliptic droplet (semi-axes ax along x, ay along y) at the domain centre; the
    n = 2 mode makes I_xx - I_yy of the liquid-excess mass oscillate.  The period (mean
    spacing of its upward zero crossings about the late mean) is compared with Eq. 32 at
    R0 = sqrt(ax ay) (the paper's equilibrium radius), the centre density and gamma (by
    default the Laplace-law slope at the same state).  Defaults: the test of Sec. IV A
    (200^2, 30 x 27, a = 0.5, T/Tc = 0.5 with the printed T_c = 0.047, sigma = 0.11,
    nu_l = 0.05, nu_v = 0.3, rates of Sec. IV A)."""
    eos = Eos(a=a, T=t_over_tc * tc)
    rl, rv = maxwell(eos)
    if gamma is None:
        gamma = laplace_law_at(eos, sigma, stream=stream).gamma
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    c = (n - 1) / 2.0
    dxy = (x - c) ** 2 - (y - c) ** 2
    sig = []
    rates = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)
    with Lattice(n, n, eos, sigma=sigma, s=rates, nu_l=nu_l, nu_v=nu_v, visc_mode=visc_mode,
                 stream=stream) as L:
        L.init_fields(wl.ellipse(n, n, rl, rv, ax, ay, 4.0))
        rho = None
        for _ in range(steps // every):
            L.step(every)
            rho = L.moments()["rho"]
            w = np.clip(rho - rv, 0.0, None)
            sig.append(float(np.sum(w * dxy) / np.sum(w)))
        ri = float(rho[n // 2, n // 2])
    s = np.array(sig)
    s0 = s - np.mean(s[len(s) // 2:])
    up = [i for i in range(1, len(s0)) if s0[i - 1] < 0.0 <= s0[i]]
    period = float(np.mean(np.diff(up))) * every if len(up) >= 2 else float("nan")
    r0 = math.sqrt(ax * ay)
    lamb = 2.0 * math.pi / math.sqrt(2 * 3 * gamma / (ri * r0 ** 3))
    return Oscillation(period, lamb, r0, ri, float(gamma), len(up), s)


@dataclasses.dataclass
class Spread:
    c: float             # fitted C of r / D = C sqrt(U t / D)
    t_star: np.ndarray
    r_over_d: np.ndarray


def splash_spread(nx=2048, ny=512, film=32, d=160.0, u=0.05, re=200.0, ratio=15.0, a=0.25,
                  t_over_tc=0.5, sigma=0.114, t_max=1.0, samples=20, stream=None):
    """The 2048 x 512 splash workload (walls, step viscosity, s_e = s_zeta = 0.8): the
    spread radius r(t), half the x-extent of liquid (rho above the mean of the phase
    densities) on the row one film thickness plus one above the wall, against t* = U t / D
    from the first contact; C by least squares of r/D on sqrt(t*)."""
    eos = Eos(a=a, T=t_over_tc * wl.t_crit(a))
    rl, rv = maxwell(eos)
    nu_l = u * d / re
    mid = 0.5 * (rl + rv)
    row = film + 1
    per = int(round(t_max * d / u / samples))
    ts, rs = [], []
    with Lattice(nx, ny, eos, sigma=sigma, s=(1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0),
                 nu_l=nu_l, nu_v=ratio * nu_l, visc_mode="step", bc="walls",
                 stream=stream) as L:
        rho, ux, uy = wl.splash(nx, ny, rl, rv, 4.0, film, d, u)
        L.init_fields(rho, ux, uy)
        # contact: the droplet's lowest liquid node reaches the probe row
        t0 = None
        n = 0
        while n < int(3 * d / u):
            L.step(20)
            n += 20
            liquid = np.nonzero(L.moments()["rho"][row] > mid)[0]
            if liquid.size:
                t0 = n
                break
        if t0 is None:
            return Spread(float("nan"), np.array([]), np.array([]))
        for k in range(1, samples + 1):
            L.step(per)
            liquid = np.nonzero(L.moments()["rho"][row] > mid)[0]
            ts.append(k * per * u / d)
            rs.append(0.5 * (liquid.max() - liquid.min() + 1) / d if liquid.size else 0.0)
    t = np.array(ts)
    r = np.array(rs)
    c = float(np.sum(r * np.sqrt(t)) / np.sum(t))
    return Spread(c, t, r)
