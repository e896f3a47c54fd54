"""The library's host solvers of the mechanical-stability condition (Eq. 21) and the
sigma calibration against the oracle's independent quadrature solver (no GPU)."""
import math

import pytest

from oracle import thermo
from paper_1211_6932_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    from paper_1211_6932_gb300 import build, _lib
    build.build()
    return _lib.load()


@pytest.mark.parametrize("a,tr,sigma", [(0.25, 0.9, 0.114), (0.25, 0.7, 0.114), (0.5, 0.8, 0.11),
                                        (1.0, 0.85, 0.05), (0.5, 0.55, 0.12)])
def test_mechanical_stability_matches_oracle(lib, a, tr, sigma):
    from paper_1211_6932_gb300.lattice import Eos, mechanical_stability
    T = tr * wl.t_crit(a)
    rl, rv = mechanical_stability(Eos(a=a, T=T), sigma)
    ol, ov, _ = thermo.mechanical_stability(a, 4.0, 1.0, T, -1.0, thermo.epsilon_from_sigma(sigma))
    assert rl == pytest.approx(ol, rel=1e-10) and rv == pytest.approx(ov, rel=1e-9)


def test_no_solution_is_reported_like_the_oracle(lib):
    """The original scheme (sigma = 0) has no positive-pressure coexistence at
    T/Tc = 0.6 for a = 0.5 (where its films also blow up)."""
    from paper_1211_6932_gb300 import LbmError
    from paper_1211_6932_gb300.lattice import Eos, mechanical_stability
    T = 0.6 * wl.t_crit(0.5)
    with pytest.raises(ValueError):
        thermo.mechanical_stability(0.5, 4.0, 1.0, T, -1.0, 0.0)
    with pytest.raises(LbmError):
        mechanical_stability(Eos(a=0.5, T=T), 0.0)


@pytest.mark.parametrize("a,tr", [(0.25, 0.6), (0.5, 0.8), (1.0, 0.5)])
def test_consistent_sigma_reproduces_maxwell_in_the_oracle(lib, a, tr):
    """At the library's calibrated sigma the oracle's Eq. 21 gives the Maxwell vapour
    density; sigma falls with a (Sec. IV B: 0.114 at a = 0.25, 0.11 at a = 0.5)."""
    from paper_1211_6932_gb300.lattice import Eos, sigma_consistent
    T = tr * wl.t_crit(a)
    s = sigma_consistent(Eos(a=a, T=T))
    _, ov, _ = thermo.mechanical_stability(a, 4.0, 1.0, T, -1.0, thermo.epsilon_from_sigma(s))
    _, mv, _ = thermo.maxwell(a, 4.0, 1.0, T)
    assert abs(math.log(ov / mv)) < 1e-9
    assert 0.09 < s < 0.13


def test_consistent_sigma_falls_with_a(lib):
    from paper_1211_6932_gb300.lattice import Eos, sigma_consistent
    s = [sigma_consistent(Eos(a=a, T=0.8 * wl.t_crit(a))) for a in (0.25, 0.5, 1.0)]
    assert s[0] > s[1] > s[2]
