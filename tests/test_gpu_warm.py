"""Warm-start device kernels against the oracle: the droplet-field fill (with the
Laplace-raised liquid density per droplet) and the phase-averaged densities."""
import numpy as np
import pytest

import oracle
from oracle import thermo
from oracle import warm as ow
from paper_1211_6932_gb300 import workloads as wl
from tests import pairs

pytestmark = pytest.mark.gpu

A = 0.25
T = 0.6 * wl.t_crit(A)


def lattice(nx, ny, precision):
    rl, rv, _ = thermo.maxwell(A, 4.0, 1.0, T)
    c = dict(nx=nx, ny=ny, a=A, T=T, sigma=0.114, s=(1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0),
             visc="linear", nu_l=0.05, nu_v=0.5, walls=False, G=-1.0)
    return pairs.gpu_lattice(c, precision), rl, rv


DROPS = np.array([[30.0, 40.0, 18.0], [150.5, 100.25, 25.0], [5.0, 140.0, 12.0]])


@pytest.mark.parametrize("curvature", [False, True])
def test_init_droplets_matches_oracle_field(curvature):
    """FP64 lattice: populations = equilibrium of the oracle's droplet field, with the
    phase densities of the droplets' mean curvature when asked; droplets wrap across the
    periodic edges."""
    from paper_1211_6932_gb300.warm import WarmParams
    ctx, rl, rv = lattice(180, 150, "fp64")
    p = WarmParams(rl * 0.999, rv * 0.94, 4.6, 0.35, 24.0)
    d = dict(rho_l=p.rho_l, rho_v=p.rho_v, curvature=p.curvature)
    kappa = float(np.mean(1.0 / DROPS[:, 2]))
    rin, rout = ow.curved_densities(d, kappa, A, 4.0, 1.0, T) if curvature else (p.rho_l, p.rho_v)
    ref = ow.droplet_field(180, 150, DROPS, [rin] * len(DROPS), rout, p.width, p.shift)
    with ctx as L:
        L.init_droplets(DROPS, p, curvature=curvature)
        got = L.get_populations()
        assert L.step_count == 0
    f_ref = oracle.equilibrium(ref, np.zeros_like(ref), np.zeros_like(ref))
    assert np.max(np.abs(got - f_ref)) <= 1e-14


def test_init_droplets_plain_is_eq31():
    """No flags, shift 0: each droplet is Eq. 31 (the recipe of workloads.multi_droplets,
    which evaluates each droplet only within its bounding box: differences are tanh tails
    below 1e-6 of the density gap)."""
    from paper_1211_6932_gb300.warm import WarmParams
    ctx, rl, rv = lattice(256, 256, "fp64")
    rho, cs, rs = wl.multi_droplets(256, 256, rl, rv, 5.0, 3, 20.0, 40.0, seed=3)
    with ctx as L:
        L.init_droplets(np.column_stack([cs, rs]), WarmParams(rl, rv, 5.0))
        got = L.moments()["rho"]
    assert np.max(np.abs(got - rho)) <= 1e-6 * (rl - rv)


def test_init_droplets_rejects_bad_arguments():
    from paper_1211_6932_gb300 import LbmError
    from paper_1211_6932_gb300.warm import WarmParams
    ctx, rl, rv = lattice(64, 64, "fp32")
    with ctx as L:
        for p, drops in ((WarmParams(rl, rv, -1.0), DROPS[:1]), (WarmParams(rv, rl, 5.0), DROPS[:1]),
                         (WarmParams(rl, rv, 5.0), np.array([[1.0, 1.0, -3.0]]))):
            with pytest.raises(LbmError) as ei:
                L.init_droplets(drops, p)
            assert ei.value.code == -1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_phase_stats_matches_density_field(precision):
    """Counts are exact; means agree with numpy's over the same densities to summation
    order."""
    from paper_1211_6932_gb300.warm import WarmParams
    ctx, rl, rv = lattice(300, 200, precision)
    with ctx as L:
        L.init_droplets(DROPS, WarmParams(rl, rv, 5.0))
        L.step(40)
        rho = L.moments()["rho"]
        vmax, lmin = 1.25 * rv, rl - 0.05 * (rl - rv)
        v, nv, l_, nl = L.phase_stats(vmax, lmin)
    assert nv == int(np.sum(rho < vmax)) and nl == int(np.sum(rho > lmin))
    assert v == pytest.approx(rho[rho < vmax].mean(), rel=1e-12)
    assert l_ == pytest.approx(rho[rho > lmin].mean(), rel=1e-12)
    assert nv > 0 and nl > 0


def test_balanced_start_has_zero_force_corrected_velocity():
    """LBM_WARM_BALANCED: populations at the equilibrium of u0 = -F/(2 rho), so the
    velocity of Eq. 6 is zero everywhere at t = 0; the populations equal the oracle's
    equilibrium at the oracle's u0."""
    from paper_1211_6932_gb300.warm import WarmParams
    ctx, rl, rv = lattice(180, 150, "fp64")
    p = WarmParams(rl, rv, 4.5, 0.3, 0.0)
    ref_rho = ow.droplet_field(180, 150, DROPS, [rl] * len(DROPS), rv, 4.5, 0.3)
    with ctx as L:
        L.init_droplets(DROPS, p, balanced=True)
        m = L.moments()
        got = L.get_populations()
    assert np.max(np.abs(m["ux"])) < 1e-15 and np.max(np.abs(m["uy"])) < 1e-15
    c = dict(nx=180, ny=150, a=A, T=T, sigma=0.114, s=(1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0),
             visc="linear", nu_l=0.05, nu_v=0.5, walls=False, G=-1.0)
    fl = oracle.fields(pairs.oracle_params(c), oracle.equilibrium(ref_rho))
    u0x, u0y = -0.5 * fl["Fx"] / ref_rho, -0.5 * fl["Fy"] / ref_rho
    assert np.max(np.abs(got - oracle.equilibrium(ref_rho, u0x, u0y))) <= 1e-14
