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
