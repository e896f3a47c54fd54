"""Lowest stable liquid viscosity against the viscosity ratio (Sec. IV C, Fig. 4) by
batched multi-section on the splash problem."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_lower_viscosity_limit_falls_with_viscosity_ratio():
    """A larger vapour/liquid viscosity ratio lets the liquid viscosity go lower (Sec.
    IV C); each bracket is consistent and narrow."""
    from paper_1211_6932_gb300 import stability as st
    br = st.lowest_stable_viscosity(ratios=(1.0, 5.0, 20.0), rounds=3)
    for b in br:
        assert not math.isnan(b.stable) and not math.isnan(b.unstable)
        assert b.unstable < b.stable < 1.2 * b.unstable
    s = [b.stable for b in br]
    assert s[0] > s[1] > s[2] and s[0] / s[2] > 2.0
    # the verdicts at the bracket ends hold when rerun
    flags = st.stable_flags([(b.stable, b.ratio) for b in br] + [(b.unstable, b.ratio) for b in br])
    assert flags == [True] * 3 + [False] * 3


def test_stability_verdict_does_not_depend_on_precision():
    """FP32 deviation storage and FP64 give the same verdicts near the boundary."""
    from paper_1211_6932_gb300 import stability as st
    trials = [(0.0045, 1.0), (0.006, 1.0), (0.0017, 20.0), (0.0025, 20.0)]
    assert st.stable_flags(trials, precision="fp32") == st.stable_flags(trials, precision="fp64")


def test_stability_verdicts_match_oracle():
    """The FP64 oracle, run on the host from its own initial state (Maxwell densities of
    its quadrature rule, equilibrium populations of Eq. 3), gives the GPU's verdict at both
    ends of the GPU's bracket for viscosity ratios 1 and 20 on the 600 x 250 splash at
    t* = 3: stable at the bracket's upper end, unstable at its lower end.  This rules out
    the GPU step as the cause of the distance between these brackets and Fig. 4."""
    import numpy as np

    import oracle
    from oracle import thermo
    from paper_1211_6932_gb300 import stability as st
    from paper_1211_6932_gb300 import workloads as wl

    br = st.lowest_stable_viscosity(ratios=(1.0, 20.0), rounds=2)
    T = st.TR * st.TC
    rl, rv, _ = thermo.maxwell(st.A, 4.0, 1.0, T)
    rho, ux, uy = wl.splash(st.NX, st.NY, rl, rv, 4.0, st.FILM, st.D, st.U)
    f0 = oracle.equilibrium(rho, ux, uy)
    steps = int(round(3.0 * st.D / st.U))
    for b in br:
        assert b.unstable < b.stable
        verdicts = []
        for nu in (b.stable, b.unstable):
            p = oracle.Params(nx=st.NX, ny=st.NY, a=st.A, T=T, sigma=st.SIGMA, s=st.RATES,
                              visc_mode=oracle.VISC_STEP, nu_l=nu, nu_v=b.ratio * nu,
                              rho_c=0.5218 / 4.0, walls=True)
            d = oracle.fields(p, oracle.run(p, f0, steps))["rho"]
            verdicts.append(bool(np.all(np.isfinite(d)) and d.min() > 0.0))
        assert verdicts == [True, False], (b, verdicts)


def test_psi_clamp_does_not_decide_stability():
    """Reading check for Fig. 4: at both ends of the ratio-1 bracket, a run that must also
    keep the argument of Eq. 24's square root non-negative everywhere at every check (no
    use of the clamp at zero) gets the same verdict as the finite-density criterion; the
    splash blows up before any node is compressed to the density where the clamp would
    act."""
    from paper_1211_6932_gb300 import stability as st
    br = st.lowest_stable_viscosity(ratios=(1.0,), rounds=2)[0]
    trials = [(br.stable, 1.0), (br.unstable, 1.0)]
    assert st.stable_flags(trials) == [True, False]
    assert st.stable_flags(trials, criterion="psi_real") == [True, False]
