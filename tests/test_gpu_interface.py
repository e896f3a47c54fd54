"""Interface width and spurious currents against the EOS parameter a (Sec. IV B): the
width ratios of Fig. 3 and the spurious velocities of Table I, from one batch of films
and 200^2 droplets."""
import pytest

from tests import golden_io

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rows():
    from paper_1211_6932_gb300 import interface as itf
    out = itf.study(t_over_tc=(0.5, 0.55), steps=30000)
    assert all(r.stable for r in out)
    return {(r.a, r.t_over_tc): r for r in out}


@pytest.mark.parametrize("tr", [0.5, 0.55])
def test_width_scales_like_one_over_sqrt_a(rows, tr):
    """W(0.25)/W(1) ~ 1.9 and W(0.5)/W(1) ~ 1.4 (Sec. IV B), within 6 %."""
    w1 = rows[(1.0, tr)].width
    assert rows[(0.25, tr)].width / w1 == pytest.approx(1.9, rel=0.06)
    assert rows[(0.5, tr)].width / w1 == pytest.approx(1.4, rel=0.06)


@pytest.mark.parametrize("tr", [0.5, 0.55])
def test_spurious_velocities_match_table_i(rows, tr):
    """Largest |v| of the equilibrated droplet against Table I: within 15 % for every a,
    and reduced 12-22 fold from a = 1 to a = 0.25 (the paper: 15-20)."""
    ref = golden_io.load("table_i_spurious.txt")["%.2f" % tr]
    for a, u in zip((1.0, 0.5, 0.25), ref[1:]):
        assert rows[(a, tr)].max_u == pytest.approx(u, rel=0.15), (a, tr)
    assert 12 < rows[(1.0, tr)].max_u / rows[(0.25, tr)].max_u < 22
    # the density ratio of the a = 0.25 droplet is the printed one to 10 %
    assert rows[(0.25, tr)].density_ratio == pytest.approx(ref[0], rel=0.1)
