"""Error of the FP32 production path over the stated runs, measured against the FP64 mode.

The FP32 path stores populations as deviations from t_q rho_ref and computes in FP32; the
FP64 mode stores and computes in double precision and matches the FP64 oracle to 1e-12
per step, so over runs too long for the host oracle it stands in for the oracle as the
reference.  For each workload both precisions start from the same density (and velocity)
field through the library's equilibrium initialisation, advance the same number of steps,
and their density fields are compared:

  max_rel_density   max over nodes of |rho_32 - rho_64| / rho_64
  liquid / vapour   mean density over the bulk liquid nodes (rho_64 above
                    rho_l - 0.05 (rho_l - rho_v), Maxwell densities) and the bulk vapour
                    nodes (rho_64 below 1.25 rho_v), the same node sets for both fields:
                    the coexistence densities, and their relative FP32 error

A second FP64 run, started from the same fields rounded once to float32 (all arithmetic
and storage still double), gives the sensitivity floor of the flow itself: how far a
perturbation of the size of one float rounding of the start drifts over the same steps.
Where the flow amplifies perturbations, no FP32 path can stay closer to the FP64 run
than this floor.

Workloads (the configurations the FP32 tolerances are stated for):
  ellipse_1024   1024^2 periodic, a = 0.25, T/Tc = 0.6, 240 x 160 ellipse with +-1e-4
                 uniform density noise (seed 2), nu_l = 0.05, nu_v = 0.5, tau linear in
                 rho; 20000 steps
  splash_2048    2048 x 512, walls in y, a = 0.25, T/Tc = 0.5, film 32, D = 160,
                 U = 0.05, Re = U D / nu_l = 200, nu_v / nu_l = 15, step viscosity,
                 s_e = s_zeta = 0.8; 30000 steps
  splash_2048_linear   the same with tau linear in rho between the Maxwell densities
                 (the step rule switches a node's viscosity on an arbitrarily small change
                 of its density, so there the flow is not a continuous function of its
                 start)
  field_4096     the 4096^2 field of 64 droplets (a = 0.25, T/Tc = 0.6, sigma = 0.114,
                 nu 0.05 / 0.5 linear); a few thousand steps

This module sequences library calls; every step runs in the library's kernels.  The
comparison itself is a host-side reduction of the read-back fields.
"""
import dataclasses

import numpy as np

from . import workloads as wl
from .lattice import Eos, Lattice, maxwell

RATES = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)
SPLASH_RATES = (1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)  # s_e = s_zeta = 0.8


@dataclasses.dataclass
class Setup:
    name: str
    nx: int
    ny: int
    steps: int
    eos: Eos
    kwargs: dict          # Lattice keyword arguments besides precision and tiling
    fields: tuple         # (rho, ux, uy) host arrays (ux, uy may be None)
    rho_l: float          # Maxwell densities (phase classification)
    rho_v: float


def setup(name, steps=None):
    """The named workload's lattice arguments and initial fields."""
    if name == "ellipse_1024":
        eos = Eos(a=0.25, T=0.6 * wl.t_crit(0.25))
        rl, rv = maxwell(eos)
        rho = wl.ellipse(1024, 1024, rl, rv, 240, 160, 4.0, noise=1e-4, seed=2)
        kw = dict(sigma=0.114, s=RATES, nu_l=0.05, nu_v=0.5, visc_mode="linear")
        return Setup(name, 1024, 1024, steps or 20000, eos, kw, (rho, None, None), rl, rv)
    if name in ("splash_2048", "splash_2048_linear"):
        eos = Eos(a=0.25, T=0.5 * wl.t_crit(0.25))
        rl, rv = maxwell(eos)
        nu_l = 0.05 * 160 / 200.0
        fields = wl.splash(2048, 512, rl, rv, 4.0, 32, 160, 0.05)
        kw = dict(sigma=0.114, s=SPLASH_RATES, nu_l=nu_l, nu_v=15 * nu_l, visc_mode="step",
                  bc="walls")
        if name == "splash_2048_linear":
            kw.update(visc_mode="linear", rho_l=rl, rho_v=rv)
        return Setup(name, 2048, 512, steps or 30000, eos, kw, fields, rl, rv)
    if name == "field_4096":
        eos = Eos(a=0.25, T=0.6 * wl.t_crit(0.25))
        rl, rv = maxwell(eos)
        rho, _, _ = wl.multi_droplets(4096, 4096, rl, rv, 4.0, 64, 40.0, 200.0, seed=5)
        kw = dict(sigma=0.114, s=RATES, nu_l=0.05, nu_v=0.5, visc_mode="linear")
        return Setup(name, 4096, 4096, steps or 2000, eos, kw, (rho, None, None), rl, rv)
    raise ValueError("unknown workload %r" % name)


def _lattice(su: Setup, precision, round_start=False, stream=None):
    """A lattice of the workload in the given precision, initialised; round_start=True
    starts from the fields rounded to float32 (passed as float64)."""
    fields = su.fields
    if round_start:
        fields = tuple(None if f is None else np.asarray(f, np.float32).astype(np.float64)
                       for f in fields)
    L = Lattice(su.nx, su.ny, su.eos, precision=precision, stream=stream, **su.kwargs)
    try:
        L.init_fields(*fields)
    except Exception:
        L.close()
        raise
    return L


@dataclasses.dataclass
class Errors:
    max_rel_density: float   # max |a - b| / b over nodes
    liquid_rel: float        # |mean_l(a) - mean_l(b)| / mean_l(b)
    vapour_rel: float
    liquid: float            # mean_l(b), mean_v(b)
    vapour: float
    n_liquid: int
    n_vapour: int


def compare_fields(a, b, rho_l, rho_v):
    """Errors of density field a against reference field b (phase sets from b)."""
    liq = b > rho_l - 0.05 * (rho_l - rho_v)
    vap = b < 1.25 * rho_v
    ml_a, ml_b = float(a[liq].mean()), float(b[liq].mean())
    mv_a, mv_b = float(a[vap].mean()), float(b[vap].mean())
    return Errors(float(np.max(np.abs(a - b) / b)), abs(ml_a - ml_b) / ml_b,
                  abs(mv_a - mv_b) / mv_b, ml_b, mv_b, int(liq.sum()), int(vap.sum()))


def fp32_error(name, steps=None, checkpoints=1, floor=True, stream=None):
    """FP32 against FP64 on the named workload, compared at `checkpoints` evenly spaced
    step counts up to `steps`; with floor=True also FP64 from the float32-rounded start
    against FP64.  Returns a dict (JSON-ready); its top-level errors are those at the
    last step, `history` has one entry per checkpoint."""
    su = setup(name, steps)
    names = ["fp64", "fp32"] + (["floor"] if floor else [])
    lats = {}
    try:
        for k in names:
            lats[k] = _lattice(su, "fp32" if k == "fp32" else "fp64", k == "floor", stream)
        done, hist = 0, []
        for c in range(1, checkpoints + 1):
            target = su.steps * c // checkpoints
            for L in lats.values():
                L.step(target - done)
            done = target
            diag = {k: L.diagnostics() for k, L in lats.items()}
            bad = {k: d["nonfinite"] for k, d in diag.items()}
            rec = {"step": done, "nonfinite": bad}
            if not any(bad.values()):
                rho = {k: L.moments()["rho"] for k, L in lats.items()}
                rec.update(dataclasses.asdict(compare_fields(rho["fp32"], rho["fp64"],
                                                             su.rho_l, su.rho_v)))
                rec["mass_rel"] = abs(diag["fp32"]["mass"] - diag["fp64"]["mass"]) / \
                    diag["fp64"]["mass"]
                rec["density_ratio"] = float(rho["fp64"].max() / rho["fp64"].min())
                if floor:
                    f = compare_fields(rho["floor"], rho["fp64"], su.rho_l, su.rho_v)
                    rec["fp64_floor"] = {"max_rel_density": f.max_rel_density,
                                         "liquid_rel": f.liquid_rel,
                                         "vapour_rel": f.vapour_rel}
            hist.append(rec)
    finally:
        for L in lats.values():
            L.close()
    out = {"workload": name, "grid": [su.nx, su.ny], "steps": su.steps}
    out.update(hist[-1])
    out["history"] = hist
    return out
