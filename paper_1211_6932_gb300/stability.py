"""Lowest stable liquid viscosity against the vapour/liquid viscosity ratio (Sec. IV C,
Fig. 4), by batched multi-section search on the splash problem.

The problem is that of Sec. IV C: a 600 x 250 lattice, walls at the top and bottom
(halfway bounce-back), periodic in x, a liquid film of 1/10 of the height on the bottom
wall, a droplet of radius 50 moving down at U = 0.125; a = 0.25, T/Tc = 0.5 with the
printed T_c = 0.0235, sigma = 0.114, s_e = s_zeta = 0.8, viscosity nu_l where rho >= rho_c
and nu_v = ratio * nu_l below (the step rule of Sec. IV C).  The paper does not state its
stability test; here a run is stable if after `t_star` = U t / D its density is finite
and positive everywhere.

Search: for every ratio the stable/unstable boundary in nu_l is bracketed in log space;
each round puts `k` trial viscosities per ratio, evenly spaced in log nu_l inside the
bracket, into one batch, and shrinks the bracket to the interval where stability
switches (stability is taken to be monotone in nu_l).  This module sequences library
calls; all arithmetic runs in the library.
"""
import dataclasses
import math

import numpy as np

from . import workloads as wl
from .lattice import Batch, Eos, Instance, maxwell

NX, NY, FILM, D, U = 600, 250, 25, 100.0, 0.125
A, TR, TC, SIGMA = 0.25, 0.5, 0.0235, 0.114
RATES = (1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)  # s_e = s_zeta = 0.8 (Sec. IV C)


@dataclasses.dataclass
class Bracket:
    ratio: float
    stable: float    # smallest nu_l seen stable
    unstable: float  # largest nu_l seen unstable (below `stable`)


# Criteria of a stable run (the paper states none):
#   "finite"     density finite and positive everywhere at t* (the default)
#   "umax"       also the largest |v| (Eq. 6) stays below U_MAX_RUN at every check
#   "psi_real"   also no node ever reaches the density where 2 (p_EOS - rho/3) / G turns
#                negative (so psi of Eq. 24 stays real without the clamp at zero)
U_MAX_RUN = 0.3  # about half the lattice speed of sound
CHECK_EVERY = 100


def psi_real_limit(eos, G=-1.0):
    """Smallest density above the liquid density where 2 (p_EOS - rho/3) / G < 0 (Eqs. 24,
    30), by bisection on the library's psi evaluation."""
    import ctypes
    from . import _lib as C
    rl, _ = maxwell(eos)
    lo, hi = rl, 4.0 / eos.b * (1.0 - 1e-9)

    def psi2(r):
        out = ctypes.c_double()
        rc = C.lib().lbm_eos_psi2(eos.c(), float(G), float(r), ctypes.byref(out))
        if rc != 0:
            raise RuntimeError("lbm_eos_psi2 failed")
        return out.value

    if psi2(hi) >= 0:
        return hi
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if psi2(mid) >= 0:
            lo = mid
        else:
            hi = mid
    return hi


def stable_flags(trials, t_star=3.0, precision="fp32", stream=None, criterion="finite",
                 velocity="fraction", gap=None):
    """trials: list of (nu_l, ratio); one bool per trial (all run in one batch).
    criterion, velocity and gap select the readings described above and in
    workloads.splash."""
    eos = Eos(a=A, T=TR * TC)
    rl, rv = maxwell(eos)
    rho, ux, uy = wl.splash(NX, NY, rl, rv, 4.0, FILM, D, U, velocity=velocity, gap=gap)
    insts = [Instance(nx=NX, ny=NY, eos=eos, sigma=SIGMA, s=RATES, nu_l=nu, nu_v=r * nu,
                      visc_mode="step", bc="walls", rho_l=rl, rho_v=rv) for nu, r in trials]
    steps = int(round(t_star * D / U))
    rho_lim = psi_real_limit(eos) if criterion == "psi_real" else None
    ok = [True] * len(insts)
    b = Batch(insts, precision=precision, stream=stream)
    try:
        for i in range(len(insts)):
            b.init_fields(i, rho, ux, uy)
        if criterion == "finite":
            b.step(steps)
        else:
            done = 0
            while done < steps:
                n = min(CHECK_EVERY, steps - done)
                b.step(n)
                done += n
                diag = b.diagnostics()
                for i in range(len(insts)):
                    if not ok[i]:
                        continue
                    if criterion == "umax" and not diag[i]["max_u"] < U_MAX_RUN:
                        ok[i] = False
                    elif criterion == "psi_real" and not float(b.density(i).max()) < rho_lim:
                        ok[i] = False
        diag = b.diagnostics()
        out = []
        for i in range(len(insts)):
            good = ok[i] and diag[i]["nonfinite"] == 0
            if good:
                d = b.density(i)
                good = bool(np.all(np.isfinite(d)) and d.min() > 0.0)
            out.append(good)
    finally:
        b.close()
    return out


def lowest_stable_viscosity(ratios=(1.0, 2.0, 5.0, 10.0, 15.0, 20.0, 35.0, 50.0),
                            nu_lo=1e-3, nu_hi=0.3, nu_v_max=1.0, k=4, rounds=4, t_star=3.0,
                            stream=None, **reading):
    """Returns a Bracket per ratio: the boundary lies between `unstable` and `stable`.
    The search starts from [nu_lo, min(nu_hi, nu_v_max / ratio)]: a vapour viscosity far
    above 1 (tau_v > 3.5) is a different instability, outside the question.  `reading`
    passes criterion / velocity / gap to stable_flags."""
    br = [Bracket(r, min(nu_hi, nu_v_max / r), nu_lo) for r in ratios]
    # the ends of the search interval, once
    flags = stable_flags([(b.stable, b.ratio) for b in br] + [(nu_lo, r) for r in ratios],
                         t_star, stream=stream, **reading)
    n = len(ratios)
    for j, b in enumerate(br):
        if not flags[j]:
            b.stable = float("nan")  # unstable even at the top of the interval
        if flags[n + j]:
            b.stable = nu_lo          # stable down to nu_lo
            b.unstable = float("nan")
    for _ in range(rounds):
        live = [b for b in br if not math.isnan(b.stable) and not math.isnan(b.unstable)]
        if not live:
            break
        trials = []
        for b in live:
            lo, hi = math.log(b.unstable), math.log(b.stable)
            trials += [(math.exp(lo + (hi - lo) * (i + 1) / (k + 1)), b.ratio) for i in range(k)]
        flags = stable_flags(trials, t_star, stream=stream, **reading)
        for j, b in enumerate(live):
            pts = trials[j * k:(j + 1) * k]
            ok = flags[j * k:(j + 1) * k]
            for (nu, _), f in zip(pts, ok):
                if f:
                    b.stable = min(b.stable, nu)
            for (nu, _), f in zip(pts, ok):
                if not f and nu < b.stable:
                    b.unstable = max(b.unstable, nu)
    return br
