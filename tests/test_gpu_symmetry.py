"""Invariances of the GPU step: the conserved-moment rates s_rho, s_j do not matter,
a centred droplet keeps its mirror symmetries, and an x-uniform film does not depend on
the strip width."""
import numpy as np
import pytest

from oracle import thermo
from paper_1211_6932_gb300 import workloads as wl
from tests import pairs

pytestmark = pytest.mark.gpu

A = 0.25
T = 0.7 * wl.t_crit(A)


def test_conserved_moment_rates_have_no_effect():
    c = pairs.case(60, 44, tr=0.7, sigma=0.114)
    f = pairs.droplet_state(c, vel=0.01)
    outs = []
    for s0, s3 in ((1.0, 1.0), (0.7, 1.3), (1.9, 0.4)):
        s = list(c["s"])
        s[0], s[3], s[5] = s0, s3, s3
        with pairs.gpu_lattice(dict(c, s=tuple(s)), "fp64") as L:
            L.set_populations(f)
            L.step(6)
            outs.append(L.get_populations())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_centred_droplet_stays_mirror_symmetric(precision, tol):
    from paper_1211_6932_gb300 import Eos, Lattice
    rl, rv, _ = thermo.maxwell(A, 4.0, 1.0, T)
    n = 128
    with Lattice(n, n, Eos(a=A, T=T), sigma=0.114,
                 s=(1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25), precision=precision) as L:
        L.init_fields(wl.droplet(n, n, rl, rv, 30.0, 4.0))
        L.step(300)
        r = L.moments()["rho"]
    for m in (r[:, ::-1], r[::-1, :], r.T):
        assert np.max(np.abs(r - m)) <= tol * rl


def test_x_uniform_film_does_not_depend_on_width():
    from paper_1211_6932_gb300 import Eos, Lattice
    rl, rv, _ = thermo.maxwell(A, 4.0, 1.0, T)
    cols = []
    for nx in (3, 300):
        with Lattice(nx, 64, Eos(a=A, T=T), sigma=0.114,
                     s=(1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25), precision="fp64") as L:
            L.init_fields(wl.flat_film(nx, 64, rl, rv, 4.0, 32))
            L.step(200)
            r = L.moments()["rho"]
            assert np.max(np.abs(r - r[:, :1])) < 1e-15
            cols.append(r[:, 0])
    assert np.max(np.abs(cols[0] - cols[1])) < 1e-14
