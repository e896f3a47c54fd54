"""Coexistence curves of the original (sigma = 0) and improved (Eq. 25) forcing on flat
films, run as one batch (Sec. IV A, Fig. 1: a = 0.5, sigma = 0.11, tau_nu = 0.6 and 0.8),
against the Maxwell rule (Eq. 22) and the mechanical-stability condition (Eq. 21), and the
batch's FP64 film against the oracle."""
import pytest

import oracle
from oracle import thermo
from oracle import warm as ow
from paper_1211_6932_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

A = 0.5


@pytest.fixture(scope="module")
def curve():
    from paper_1211_6932_gb300 import coexistence as cx
    return cx.sweep(a=A, steps=40000)


def eq21(p):
    return thermo.mechanical_stability(A, 4.0, 1.0, p.t_over_tc * wl.t_crit(A), -1.0,
                                       thermo.epsilon_from_sigma(p.sigma))


def test_reach_of_the_two_schemes(curve):
    """The improved forcing holds flat films down to T/Tc = 0.49 (density ratio ~900);
    the original scheme fails below T/Tc ~ 0.8 (Sec. IV A)."""
    from paper_1211_6932_gb300 import coexistence as cx
    for tau in (0.6, 0.8):
        assert cx.lowest_stable(curve, 0.11, tau) == 0.49
        low0 = cx.lowest_stable(curve, 0.0, tau)
        assert low0 is not None and 0.8 <= low0 <= 0.85
    p = [q for q in curve if q.sigma == 0.11 and q.t_over_tc == 0.49][0]
    assert p.rho_l / p.rho_v > 800


def test_improved_forcing_tracks_maxwell(curve):
    """Liquid branch within 1e-3 of Maxwell for the improved scheme, off by about 1 % for
    the original one; in the vapour branch the original scheme is off by far more."""
    for p in curve:
        if not p.stable:
            continue
        dl = abs(p.rho_l / p.maxwell_l - 1)
        if p.sigma == 0.11:
            assert dl < 1e-3, p
        elif p.t_over_tc <= 0.9:
            assert dl > 8e-3, p
    for tr in (0.85, 0.9):
        for tau in (0.6, 0.8):
            imp, org = [[q for q in curve if q.sigma == s and q.tau_nu == tau
                         and q.t_over_tc == tr][0] for s in (0.11, 0.0)]
            assert abs(org.rho_v / org.maxwell_v - 1) > 5 * abs(imp.rho_v / imp.maxwell_v - 1)


def test_films_follow_mechanical_stability(curve):
    """Eq. 21 with eps from Eq. 29 predicts the films: the original scheme to 1e-4 (it is
    Eq. 21 with eps = 0), the improved one to 1 % at T/Tc >= 0.7 (at lower temperatures the
    interfaces are a few nodes wide and the lattice departs from the continuum condition)."""
    for p in curve:
        if not p.stable:
            continue
        ml, mv, _ = eq21(p)
        if p.sigma == 0.0:
            assert abs(p.rho_l / ml - 1) < 1e-4 and abs(p.rho_v / mv - 1) < 1e-3, p
        elif p.t_over_tc >= 0.7:
            assert abs(p.rho_l / ml - 1) < 1e-3 and abs(p.rho_v / mv - 1) < 1e-2, p


def test_fp64_film_matches_oracle():
    """The batch's FP64 film after 3001 steps against the oracle's (a = 0.5, T/Tc = 0.8,
    improved forcing, 3 x 64), measured the same way."""
    from paper_1211_6932_gb300 import coexistence as cx
    pts = cx.sweep(a=A, t_over_tc=(0.8,), sigmas=(0.11,), taus=(0.8,), nx=3, ny=64, steps=3000,
                   avg_samples=1, avg_stride=1, precision="fp64")
    T = 0.8 * wl.t_crit(A)
    rl, rv, _ = thermo.maxwell(A, 4.0, 1.0, T)
    p = oracle.Params(nx=3, ny=64, a=A, T=T, sigma=0.11, s=cx.rates(0.8))
    f = oracle.run(p, oracle.equilibrium(wl.flat_film(3, 64, rl, rv, 5.0, 32.0)), 3001)
    m = ow.measure_film(oracle.fields(p, f)["rho"])
    assert pts[0].stable
    assert abs(pts[0].rho_l / m["rho_l"] - 1) < 1e-10 and abs(pts[0].rho_v / m["rho_v"] - 1) < 1e-10
