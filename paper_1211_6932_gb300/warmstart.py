"""Learned warm start, end to end, on top of the library's entry points.

1. ``equilibria``: per parameter draw one flat film and two droplets (radii 20 and 40)
   advance together in one batch (lbm_batch_*) until every instance's density changes by
   less than `tol` per check interval (or a step limit); then the densities are averaged
   over a window and measured (lbm_measure_film / lbm_measure_droplet).  The film gives
   rho_l, the width and the shift; the two droplets' far vapour densities give the vapour
   law rho_out(R) = rho_v (1 + curvature / R) (lbm_vapour_law).  Rows are encoded with
   lbm_warm_encode.
2. ``Surrogate``: networks of lbm_mlp.h trained on those rows by full-batch Adam on
   the GPU; their mean prediction decoded (lbm_warm_decode) gives the warm-start
   parameters.
3. ``relax``: a droplet field initialised on the device (lbm_init_droplets), stepped,
   with the phase-averaged densities (lbm_phase_stats) recorded at every check.  The
   warm start uses the network's parameters with the vapour curvature law
   (LBM_WARM_CURVATURE) and a force-balanced start (LBM_WARM_BALANCED, u0 = -F/(2 rho)),
   which removes the start-up impulse that otherwise rings through the liquid.
4. ``settling_step``: the first check after which the phase densities stay within a
   tolerance of reference values.

Everything numerical runs in the library (CUDA kernels, or host C++ for the small
measurements); this module sequences the calls.
"""
import dataclasses
import math

import numpy as np

from . import workloads as wl
from .lattice import Batch, Eos, Instance, Lattice, maxwell
from .mlp import Mlp
from .warm import WarmParams, decode, encode, measure_droplet, measure_film, vapour_law

# Relaxation rates of Eq. 2 used by the warm-start runs (s_e = s_zeta = s_q = 1.1 as in
# Sec. IV A; the stress rates follow the density through the linear viscosity mode).
RATES = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)
W_PLAIN = 5.0  # the tanh width of Eq. 31 used in Sec. IV A
DROP_RADII = (20.0, 40.0)  # the two droplets of each draw, in boxes of side 4 R + 8


def features(a, t_over_tc, sigma, visc_ratio):
    return np.array([a, t_over_tc, sigma, visc_ratio], dtype=np.float64)


def eos_of(a, t_over_tc):
    return Eos(a=a, T=t_over_tc * wl.t_crit(a))


@dataclasses.dataclass
class Dataset:
    x: np.ndarray          # (m, 4) features
    y: np.ndarray          # (m, 5) encoded targets
    raw: np.ndarray        # (m, 12) film rho_l, rho_v, width, shift; per droplet rho_in,
                           # rho_out, equimolar radius, Laplace-law surface tension
    draws: list            # the draws kept, in row order
    steps: np.ndarray      # (m, 3) steps film / droplets took to meet the tolerance (-1: not)
    dropped: list          # (draw index, reason) of draws left out


def equilibria(draws, nu_l=0.05, tol=1e-6, check_every=100, max_steps=60000, avg_samples=20,
               avg_stride=200, stream=None):
    """Training rows from equilibrated film + two droplets, one triple per draw."""
    insts, fields, eoses = [], [], []
    for d in draws:
        e = eos_of(d["a"], d["T_over_Tc"])
        rl, rv = maxwell(e)
        eoses.append(e)
        kw = dict(eos=e, sigma=d["sigma"], s=RATES, nu_l=nu_l, nu_v=nu_l * d["visc_ratio"],
                  visc_mode="linear", rho_l=rl, rho_v=rv)
        insts.append(Instance(nx=d["nx"], ny=d["ny"], **kw))
        fields.append(wl.flat_film(d["nx"], d["ny"], rl, rv, W_PLAIN, d["ny"] / 2.0))
        for r in DROP_RADII:
            n = int(4 * r) + 8
            insts.append(Instance(nx=n, ny=n, **kw))
            fields.append(wl.droplet(n, n, rl, rv, r, W_PLAIN))
    b = Batch(insts, precision="fp32", stream=stream)
    try:
        for i, f in enumerate(fields):
            b.init_fields(i, f)
        _, steps = b.run_to_equilibrium(tol, check_every, max_steps)
        # average the density over a window (instances that met the tolerance are frozen
        # and contribute a constant)
        acc = [np.zeros((insts[i].ny, insts[i].nx)) for i in range(len(insts))]
        for _ in range(avg_samples):
            b.step(avg_stride)
            for i in range(len(insts)):
                acc[i] += b.density(i)
        diag = b.diagnostics()
    finally:
        b.close()
    xs, ys, raw, kept, st, dropped = [], [], [], [], [], []
    for k, d in enumerate(draws):
        idx = [3 * k, 3 * k + 1, 3 * k + 2]
        if any(diag[i]["nonfinite"] for i in idx):
            dropped.append((k, "unstable"))
            continue
        try:
            p = measure_film(acc[idx[0]] / avg_samples)
            m1 = measure_droplet(acc[idx[1]] / avg_samples, eoses[k])
            m2 = measure_droplet(acc[idx[2]] / avg_samples, eoses[k])
            film_rho_v = p.rho_v
            p.rho_v, p.curvature = vapour_law(m1[2], m1[1], m2[2], m2[1])
            y = encode(eoses[k], p)
        except Exception as ex:  # the run did not settle, or the vapour law is not positive
            dropped.append((k, "measure: %s" % ex))
            continue
        xs.append(features(d["a"], d["T_over_Tc"], d["sigma"], d["visc_ratio"]))
        ys.append(y)
        raw.append((p.rho_l, film_rho_v, p.width, p.shift) + tuple(m1) + tuple(m2))
        kept.append(d)
        st.append(tuple(steps[i] for i in idx))
    return Dataset(np.array(xs), np.array(ys), np.array(raw), kept, np.array(st), dropped)


class Surrogate:
    """The warm-start networks trained on a Dataset: `members` networks of lbm_mlp.h,
    initialised from seeds seed, seed + 1, ..., each trained by full-batch Adam on the
    GPU; a prediction is the mean of their encoded outputs.  One network's prediction at a
    given point moves by about 1 % in rho_v from one seed (or one rounding-level change of
    the training rows) to the next; the mean over members takes that scatter out."""

    def __init__(self, seed=0, max_rows=4096, stream=None, members=16):
        self.nets = []
        try:
            for k in range(members):
                self.nets.append(Mlp(wl.mlp_init(seed + k), max_rows=max_rows, stream=stream))
        except Exception:
            self.close()
            raise
        self.losses = None

    def close(self):
        for n in self.nets:
            n.close()
        self.nets = []

    def fit(self, data: Dataset, steps=4000, lr=3e-3):
        """Train every member; returns the members' mean loss before each update."""
        curves = []
        for n in self.nets:
            n.fit_scaling(data.x, data.y)
            n.set_data(data.x, data.y)
            curves.append(n.train(steps, lr=lr))
        self.losses = np.mean(curves, axis=0)
        return self.losses

    def predict(self, a, t_over_tc, sigma, visc_ratio) -> WarmParams:
        x = features(a, t_over_tc, sigma, visc_ratio)[None, :]
        y = np.mean([n.predict(x)[0] for n in self.nets], axis=0)
        return decode(eos_of(a, t_over_tc), y)


def plain_params(eos: Eos) -> WarmParams:
    """Eq. 31 with the Maxwell densities and W = 5."""
    rl, rv = maxwell(eos)
    return WarmParams(rl, rv, W_PLAIN, 0.0, 0.0)


@dataclasses.dataclass
class Relaxation:
    steps: np.ndarray  # check steps
    vap: np.ndarray    # mean vapour-phase density at each check
    liq: np.ndarray    # mean liquid-phase density at each check
    thresholds: tuple  # (rho_vap_max, rho_liq_min)


def relax(lat: Lattice, drops, params: WarmParams, curvature, thresholds, check_every, horizon,
          balanced=False):
    """Initialise lat with the droplets, then step to `horizon`, recording the phase
    densities every check_every steps (including step 0)."""
    lat.init_droplets(drops, params, curvature=curvature, balanced=balanced)
    steps, vap, liq = [0], [], []
    v, _, l_, _ = lat.phase_stats(*thresholds)
    vap.append(v)
    liq.append(l_)
    n = 0
    while n < horizon:
        lat.step(check_every)
        n += check_every
        v, _, l_, _ = lat.phase_stats(*thresholds)
        steps.append(n)
        vap.append(v)
        liq.append(l_)
    return Relaxation(np.array(steps), np.array(vap), np.array(liq), tuple(thresholds))


def settling_step(rel: Relaxation, ref_vap, ref_liq, tol_vap, tol_liq):
    """First check step from which on every later check has both phase densities within
    the relative tolerances of the references (None if the last check does not)."""
    ok = (np.abs(rel.vap / ref_vap - 1.0) <= tol_vap) & (np.abs(rel.liq / ref_liq - 1.0) <= tol_liq)
    if not ok[-1]:
        return None
    bad = np.nonzero(~ok)[0]
    k = 0 if len(bad) == 0 else bad[-1] + 1
    return int(rel.steps[k])


def phase_thresholds(p: WarmParams):
    """Vapour nodes: rho below 1.25 rho_v; liquid nodes: rho above rho_l minus 5 % of
    the density gap."""
    return (1.25 * p.rho_v, p.rho_l - 0.05 * (p.rho_l - p.rho_v))


def drops_array(centres, radii):
    return np.column_stack([centres[:, 0], centres[:, 1], radii])


def tail_mean(x, frac=0.2):
    k = max(1, int(math.ceil(frac * len(x))))
    return float(np.mean(x[-k:]))
