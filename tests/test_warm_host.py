"""Warm-start definitions: the oracle against closed forms, and the library's host
functions (no GPU needed) against the oracle."""
import math

import numpy as np
import pytest

from oracle import thermo
from oracle import warm as ow
from paper_1211_6932_gb300 import workloads as wl

A, B, R = 0.25, 4.0, 1.0
T = 0.6 * wl.t_crit(A)


def tanh_film(nx, ny, W, h, rl, rv):
    return wl.flat_film(nx, ny, rl, rv, W, h)


@pytest.mark.parametrize("ny,W,h", [(64, 5.0, 32), (65, 4.0, 30.5), (128, 7.5, 64), (97, 3.0, 40)])
def test_oracle_film_recovers_tanh_parameters(ny, W, h):
    """For the tanh profile of Eq. 31 the integral width gives W, the shift is 0 (the
    profile is odd about its centre, so the centroid of g (1 - g) is the Gibbs surface) and
    the bulk values are the profile at the film and vapour centres, interpolated linearly
    between the rows next to them (rows c -/+ 1/2 when c = (ny-1)/2 is not a row)."""
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    m = ow.measure_film(tanh_film(3, ny, W, h, rl, rv))
    c = (ny - 1) / 2
    prof = lambda y: wl.tanh_profile(abs(y - c) - h / 2, rl, rv, W)  # noqa: E731
    assert m["rho_l"] == pytest.approx(0.5 * (prof(math.floor(c)) + prof(math.ceil(c))), rel=1e-12)
    assert m["rho_v"] == pytest.approx(0.5 * (prof(0) + prof(ny - 1)), rel=1e-12)
    assert m["rho_l"] == pytest.approx(rl, rel=1e-4) and m["rho_v"] == pytest.approx(rv, rel=1e-3)
    # the row sum of a smooth decaying function is spectrally accurate; the normalisation by
    # the bulk values of a finite film costs a relative error of about exp(-2 h / W)
    assert m["width"] == pytest.approx(W, rel=1e-4)
    assert abs(m["shift"]) < 1e-4  # finite-film tails, exp(-2 (ny - h) / (2 W)) in size


def test_oracle_film_shift_of_a_shifted_tanh():
    """A tanh film whose centre sits at c + h/2 + s0 but whose bulk densities are fixed:
    the Gibbs surface moves with the profile, so the shift stays 0; the centroid of
    g (1 - g) is the profile centre."""
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    ny, h, W = 128, 60.0, 5.0
    for s0 in (-0.3, 0.0, 0.45):
        m = ow.measure_film(tanh_film(2, ny, W, h + 2 * s0, rl, rv))
        assert abs(m["shift"]) < 1e-6


def test_oracle_film_shift_of_two_sided_tanh():
    """A profile with vapour-side width Wv and liquid-side width Wl about d = 0.  Per unit
    area the vapour tail carries an excess (Wv/4) ln 2 and the liquid side a deficit
    (Wl/4) ln 2, so the Gibbs surface lies (Wv - Wl) ln 2 / 4 beyond d = 0.  The weights of
    g (1 - g) are W/8 on each side with first moments +-(W^2/16) ln 2, so the centroid lies
    (Wv - Wl) ln 2 / 2 beyond d = 0.  Hence shift = (Wv - Wl) ln 2 / 4 (the kink at d = 0
    costs the row sums their spectral accuracy: 2 % tolerance)."""
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    ny = 256
    y = np.arange(ny, dtype=float)
    for Wv, Wl in ((8.0, 3.0), (3.0, 6.0)):
        d = np.abs(y - (ny - 1) / 2) - 64.0
        W = np.where(d > 0, Wv, Wl)
        prof = 0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2 * d / W)
        m = ow.measure_film(np.tile(prof[:, None], (1, 2)))
        assert m["shift"] == pytest.approx((Wv - Wl) * math.log(2) / 4, rel=2e-2)


@pytest.mark.parametrize("r0,W", [(20.0, 5.0), (31.5, 4.0), (12.0, 3.0)])
def test_oracle_droplet_equimolar_radius(r0, W):
    """For the tanh droplet the equimolar radius obeys R^2 = r0^2 + pi^2 W^2 / 48 (the
    first moment of 1 - tanh over the half line is pi^2/24)."""
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    n = 128
    rho = wl.droplet(n, n, rl, rv, r0, W)
    ri, ro, Rg, lap = ow.measure_droplet(rho, A, B, R, T)
    assert ri == pytest.approx(rl, rel=1e-6) and ro == pytest.approx(rv, rel=1e-6)
    assert Rg == pytest.approx(math.sqrt(r0 ** 2 + math.pi ** 2 * W ** 2 / 48), rel=2e-4)
    # Maxwell end densities have equal pressure: no jump
    dp = thermo.p_eos(ri, A, B, R, T) - thermo.p_eos(ro, A, B, R, T)
    assert lap == pytest.approx(dp * Rg, rel=1e-12, abs=1e-18)
    # p(rl) = p(rv) for the Maxwell pair: the jump comes only from the profile's tails at
    # the measuring points, first order in their offsets from rl and rv
    bound = Rg * (abs(thermo.dp_drho(rl, A, B, R, T) * (ri - rl))
                  + abs(thermo.dp_drho(rv, A, B, R, T) * (ro - rv)))
    assert abs(lap) <= 1.01 * bound + 1e-15


def test_oracle_curved_densities_first_order():
    """The liquid follows the vapour's pressure rise to first order: p(rho_in) - p(rho_l)
    = p(rho_out) - p(rho_v) up to a residual second order in the curvature; zero
    curvature returns the flat pair."""
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    p = {"rho_l": rl, "rho_v": rv, "curvature": 25.0}
    assert ow.curved_densities(p, 0.0, A, B, R, T) == (rl, rv)
    res = []
    for kappa in (1 / 50.0, 1 / 100.0, 1 / 200.0):
        ri, ro = ow.curved_densities(p, kappa, A, B, R, T)
        assert ro == pytest.approx(rv * (1 + 25.0 * kappa), rel=1e-15)
        res.append(thermo.p_eos(ri, A, B, R, T) - thermo.p_eos(rl, A, B, R, T)
                   - (thermo.p_eos(ro, A, B, R, T) - thermo.p_eos(rv, A, B, R, T)))
    assert abs(res[1] / res[0]) == pytest.approx(0.25, rel=0.1)
    assert abs(res[2] / res[1]) == pytest.approx(0.25, rel=0.1)


def test_oracle_encode_decode_roundtrip():
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    p = {"rho_l": rl * 1.003, "rho_v": rv * 0.93, "width": 4.7, "shift": -0.2, "curvature": 30.0}
    y = ow.encode(p, A, B, R, T)
    assert y[0] == pytest.approx(0.003) and y[1] == pytest.approx(math.log(0.93))
    assert y[4] == pytest.approx(math.log(30.0))
    q = ow.decode(y, A, B, R, T)
    for k in p:
        assert q[k] == pytest.approx(p[k], rel=1e-14)


def test_oracle_vapour_law_recovers_a_1_over_r_law():
    rv, k = 2.5e-3, 18.0
    got = ow.vapour_law(20.0, rv * (1 + k / 20.0), 40.0, rv * (1 + k / 40.0))
    assert got[0] == pytest.approx(rv, rel=1e-12) and got[1] == pytest.approx(k, rel=1e-12)


def test_oracle_droplet_field_is_eq31_for_one_droplet():
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    f = ow.droplet_field(40, 30, [((40 - 1) / 2, (30 - 1) / 2, 9.0)], [rl], rv, 5.0)
    assert np.allclose(f, wl.droplet(40, 30, rl, rv, 9.0, 5.0), rtol=0, atol=1e-15)


# --- library host functions against the oracle (CPU only) ---------------------------

@pytest.fixture(scope="module")
def lib():
    from paper_1211_6932_gb300 import build, _lib
    build.build()
    return _lib.load()


def noisy(field, seed, amp):
    return field + amp * np.random.default_rng(seed).uniform(-1, 1, field.shape)


@pytest.mark.parametrize("ny,W,h,seed", [(64, 5.0, 32, 0), (97, 4.0, 48, 1), (200, 6.0, 100, 2)])
def test_library_film_measure_matches_oracle(lib, ny, W, h, seed):
    from paper_1211_6932_gb300 import warm
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    rho = noisy(tanh_film(7, ny, W, h, rl, rv), seed, 1e-5)
    m = warm.measure_film(rho)
    o = ow.measure_film(rho)
    for k in ("rho_l", "rho_v", "width", "shift"):
        assert getattr(m, k) == pytest.approx(o[k], rel=1e-11, abs=1e-12), k
    assert m.curvature == 0.0


@pytest.mark.parametrize("nx,ny,r0,seed", [(64, 64, 16, 0), (77, 120, 19.5, 1), (200, 90, 22, 2)])
def test_library_droplet_measure_matches_oracle(lib, nx, ny, r0, seed):
    from paper_1211_6932_gb300 import Eos, warm
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    rho = noisy(wl.droplet(nx, ny, rl * 1.002, rv * 1.05, r0, 4.5), seed, 1e-6)
    got = warm.measure_droplet(rho, Eos(a=A, T=T))
    ref = ow.measure_droplet(rho, A, B, R, T)
    for g, r in zip(got, ref):
        assert g == pytest.approx(r, rel=1e-10)


def test_library_encode_decode_and_curvature_match_oracle(lib):
    from paper_1211_6932_gb300 import Eos, warm
    e = Eos(a=A, T=T)
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    p = warm.WarmParams(rl * 0.998, rv * 1.07, 4.2, 0.3, 22.0)
    d = dict(rho_l=p.rho_l, rho_v=p.rho_v, width=p.width, shift=p.shift, curvature=p.curvature)
    assert np.allclose(warm.encode(e, p), ow.encode(d, A, B, R, T), rtol=1e-9, atol=1e-12)
    q = warm.decode(e, warm.encode(e, p))
    assert q.rho_l == pytest.approx(p.rho_l, rel=1e-14) and q.rho_v == pytest.approx(p.rho_v, rel=1e-14)
    for kappa in (0.0, 1 / 30.0, 1 / 120.0):
        got = warm.curved_densities(e, p, kappa)
        ref = ow.curved_densities(d, kappa, A, B, R, T)
        assert got[0] == pytest.approx(ref[0], rel=1e-13) and got[1] == pytest.approx(ref[1], rel=1e-14)


def test_library_vapour_law_matches_oracle(lib):
    from paper_1211_6932_gb300 import LbmError, warm
    for args in ((20.0, 3.3e-3, 40.0, 2.9e-3), (19.7, 4.1e-2, 41.3, 3.8e-2), (40.0, 1e-3, 20.0, 1.2e-3)):
        got = warm.vapour_law(*args)
        ref = ow.vapour_law(*args)
        assert got[0] == pytest.approx(ref[0], rel=1e-12) and got[1] == pytest.approx(ref[1], rel=1e-10)
    with pytest.raises(LbmError):
        warm.vapour_law(20.0, 1e-3, 20.0, 2e-3)


def test_library_measure_rejects_bad_input(lib):
    from paper_1211_6932_gb300 import Eos, LbmError, warm
    with pytest.raises(LbmError):
        warm.measure_film(np.full((32, 4), 0.1))
    with pytest.raises(LbmError):
        warm.measure_droplet(np.full((32, 32), 0.1), Eos(a=A, T=T))
