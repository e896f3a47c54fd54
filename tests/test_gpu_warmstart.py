"""What the trained network gains: the 4096^2 field of 64 droplets (radii 40..200) at
a = 0.25, T = 0.6 T_c, sigma = 0.114, viscosity ratio 10, started from the warm start
(the network's parameters with the vapour curvature law and a force-balanced start)
settles its phase densities in fewer steps than the same force-balanced start without the
network (Eq. 31 with the Maxwell densities), and settles to the same values.  The control
arm differs from the warm start only in the parameters the network supplies, so the
difference in steps is what the network adds.

The training set is the benchmark's: 256 draws over the whole parameter box of the
batched workload, one film and two droplets each (about 20 s on the GPU)."""
import pytest

from paper_1211_6932_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

A, TR, SIGMA, RATIO = 0.25, 0.6, 0.114, 10.0


@pytest.fixture(scope="module")
def surrogate():
    from paper_1211_6932_gb300 import warmstart as ws
    ds = ws.equilibria(wl.warm_draws(256, seed=6), max_steps=60000)
    assert len(ds.x) >= 240, ds.dropped
    sur = ws.Surrogate(seed=0)
    losses = sur.fit(ds, steps=4000, lr=3e-3)
    assert losses[-1] < 1e-2 * losses[0]
    yield sur
    sur.close()


def test_warm_start_settles_sooner_to_the_same_state(surrogate):
    from paper_1211_6932_gb300 import Lattice
    from paper_1211_6932_gb300 import warmstart as ws
    eos = ws.eos_of(A, TR)
    plain = ws.plain_params(eos)
    warm = surrogate.predict(A, TR, SIGMA, RATIO)
    # the network's profile parameters are physical: a few lattice units wide, vapour
    # density below Maxwell's at this sigma, liquid density within 0.1 % of Maxwell's
    assert 3.0 < warm.width < 6.0 and 0.0 < warm.shift < 1.0 and warm.curvature > 0
    assert 0.5 * plain.rho_v < warm.rho_v < plain.rho_v
    assert abs(warm.rho_l / plain.rho_l - 1) < 1e-3
    cs, rs = wl.droplet_layout(4096, 4096, 64, 40.0, 200.0, seed=5, gap=20.0)
    drops = ws.drops_array(cs, rs)
    thr = ws.phase_thresholds(plain)
    with Lattice(4096, 4096, eos, sigma=SIGMA, s=ws.RATES, nu_l=0.05, nu_v=0.05 * RATIO,
                 precision="fp32", visc_mode="linear") as L:
        rp = ws.relax(L, drops, plain, False, thr, 100, 30000)
        rb = ws.relax(L, drops, plain, False, thr, 100, 30000, balanced=True)
        rw = ws.relax(L, drops, warm, True, thr, 100, 30000, balanced=True)
    ref_v, ref_l = ws.tail_mean(rp.vap), ws.tail_mean(rp.liq)
    for tv, tl in ((0.01, 0.002), (0.005, 0.001)):
        sp = ws.settling_step(rp, ref_v, ref_l, tv, tl)
        sb = ws.settling_step(rb, ref_v, ref_l, tv, tl)
        sw = ws.settling_step(rw, ref_v, ref_l, tv, tl)
        assert sp is not None and sb is not None and sw is not None
        # the network against the same start without it, and against the paper's start
        assert sw < 0.5 * sb, (tv, tl, sw, sb)
        assert sw < 0.5 * sp, (tv, tl, sw, sp)
    # the starting vapour is much closer to where the field settles
    assert abs(rw.vap[0] / ref_v - 1) < 0.5 * abs(rp.vap[0] / ref_v - 1)
    # same final state
    assert abs(ws.tail_mean(rw.vap) / ref_v - 1) < 2e-3
    assert abs(ws.tail_mean(rw.liq) / ref_l - 1) < 2e-4
