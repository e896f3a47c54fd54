"""Interface width and spurious currents against the EOS parameter a (Sec. IV B, Fig. 3
and Table I).

For each a and reduced temperature, one flat film (for the width: the integral width of
lbm_measure_film, the W of Eq. 31 for a tanh profile) and one stationary droplet
(Sec. IV A: 200 x 200, r0 = 50, Eq. 31 start with W = 5; for the largest velocity
magnitude of Eq. 6 at the end, the spurious current) advance together in one batch.
sigma per a: 0.11 for a >= 0.5 and 0.114 for a = 0.25 (the paper's values; the sigma0
rule of workloads.py in between).  Rates as in Sec. IV A with tau_nu = 0.8.  T_c is the
value the paper prints for a = 1, 0.5, 0.25 (0.094, 0.047, 0.0235: a / 10.601 rounded),
else 0.3773 a / b.

This module sequences library calls; all arithmetic runs in the library.
"""
import dataclasses


from . import workloads as wl
from .coexistence import rates
from .lattice import Batch, Eos, Instance, maxwell
from .warm import measure_film


PAPER_TC = {1.0: 0.094, 0.5: 0.047, 0.25: 0.0235}


def t_crit(a):
    return PAPER_TC.get(a, wl.t_crit(a))


@dataclasses.dataclass
class Row:
    a: float
    t_over_tc: float
    sigma: float
    width: float          # film integral width (nan when unstable)
    max_u: float          # droplet's largest |v| at the end (nan when unstable)
    density_ratio: float  # droplet centre / far-point density
    stable: bool


def study(a_values=(1.0, 0.5, 0.25), t_over_tc=(0.5, 0.55), tau_nu=0.8, film_ny=128, n=200,
          r0=50.0, steps=30000, precision="fp32", stream=None):
    keys, insts, fields = [], [], []
    for a in a_values:
        sig = wl.sigma0(a)
        for tr in t_over_tc:
            eos = Eos(a=a, T=tr * t_crit(a))
            rl, rv = maxwell(eos)
            kw = dict(eos=eos, sigma=sig, s=rates(tau_nu), visc_mode="const", rho_l=rl, rho_v=rv)
            keys.append((a, tr, sig))
            insts.append(Instance(nx=4, ny=film_ny, **kw))
            fields.append(wl.flat_film(4, film_ny, rl, rv, 5.0, film_ny / 2.0))
            insts.append(Instance(nx=n, ny=n, **kw))
            fields.append(wl.droplet(n, n, rl, rv, r0, 5.0))
    b = Batch(insts, precision=precision, stream=stream)
    try:
        for i, f in enumerate(fields):
            b.init_fields(i, f)
        b.step(steps)
        diag = b.diagnostics()
        films = [b.density(2 * k) for k in range(len(keys))]
        drops = [b.density(2 * k + 1) for k in range(len(keys))]
    finally:
        b.close()
    out = []
    for k, (a, tr, sig) in enumerate(keys):
        ok = diag[2 * k]["nonfinite"] == 0 and diag[2 * k + 1]["nonfinite"] == 0
        w = mu = ratio = float("nan")
        if ok:
            try:
                w = measure_film(films[k]).width
            except Exception:
                ok = False
            d = drops[k]
            mu = diag[2 * k + 1]["max_u"]
            ratio = float(d[n // 2, n // 2] / d[0, 0])
        out.append(Row(a, tr, sig, w, mu, ratio, bool(ok)))
    return out
