"""Helpers that build the same lattice on both sides: the CUDA library (through its
Python binding) and the FP64 oracle."""
import numpy as np

import oracle
from oracle import thermo
from paper_1211_6932_gb300 import workloads as wl

B, R = 4.0, 1.0
RATES_TAU1 = (1.0, 1.0, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)


def case(nx, ny, a=0.25, tr=0.7, sigma=0.114, s=None, visc="const", nu_l=0.0, nu_v=0.0,
         walls=False, G=-1.0):
    """A dict describing one lattice; T = tr * 0.3773 a / b."""
    T = tr * wl.t_crit(a, B, R)
    return dict(nx=nx, ny=ny, a=a, T=T, sigma=sigma, s=tuple(s or oracle.rates_for(0.8)),
                visc=visc, nu_l=nu_l, nu_v=nu_v, walls=walls, G=G)


def maxwell(c):
    rl, rv, _ = thermo.maxwell(c["a"], B, R, c["T"])
    return rl, rv


def oracle_params(c):
    vm = {"const": oracle.VISC_CONST, "step": oracle.VISC_STEP,
          "linear": oracle.VISC_LINEAR}[c["visc"]]
    rl, rv = maxwell(c)
    return oracle.Params(nx=c["nx"], ny=c["ny"], a=c["a"], b=B, R=R, T=c["T"], G=c["G"],
                         sigma=c["sigma"], s=c["s"], visc_mode=vm, nu_l=c["nu_l"],
                         nu_v=c["nu_v"], rho_c=0.5218 / B, rho_l=rl, rho_v=rv,
                         walls=c["walls"])


def gpu_lattice(c, precision="fp64", **kw):
    from paper_1211_6932_gb300 import Eos, Lattice
    rl, rv = maxwell(c)
    return Lattice(c["nx"], c["ny"], Eos(a=c["a"], T=c["T"], b=B, R=R), G=c["G"],
                   sigma=c["sigma"], s=c["s"], nu_l=c["nu_l"], nu_v=c["nu_v"],
                   precision=precision, visc_mode=c["visc"],
                   bc="walls" if c["walls"] else "periodic", rho_c=0.5218 / B, rho_l=rl,
                   rho_v=rv, **kw)


def droplet_state(c, r0=None, W=4.0, seed=0, vel=0.0):
    """Equilibrium populations (oracle) of a droplet with a little seeded noise/velocity."""
    rl, rv = maxwell(c)
    nx, ny = c["nx"], c["ny"]
    r0 = r0 if r0 is not None else 0.3 * min(nx, ny)
    rho = wl.droplet(nx, ny, rl, rv, r0, W)
    rng = np.random.default_rng(seed)
    ux = vel * rng.uniform(-1, 1, rho.shape)
    uy = vel * rng.uniform(-1, 1, rho.shape)
    return oracle.equilibrium(rho, ux, uy)


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
