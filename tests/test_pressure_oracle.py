"""Pins of the discrete pressure tensor oracle (Eq. 18) against closed forms."""
import numpy as np
import pytest

import oracle
from oracle import pressure as op
from oracle import thermo
from paper_1211_6932_gb300 import workloads as wl

A, B, R = 0.25, 4.0, 1.0


def test_uniform_state_gives_the_equation_of_state():
    """sum_a w e_a e_a = I for the weights of Eq. 7, so a uniform state has
    P = rho/3 + (G/2) psi^2 = p_EOS (Eq. 24) on the diagonal and no shear."""
    T = 0.7 * wl.t_crit(A)
    for rho0 in (0.01, 0.13, 0.35):
        rho = np.full((5, 6), rho0)
        psi = np.full_like(rho, thermo.psi(rho0, A, B, R, T))
        pxx, pyy, pxy = op.pressure_tensor_from_psi(rho, psi, -1.0)
        p = thermo.p_eos(rho0, A, B, R, T)
        assert np.allclose(pxx, p, rtol=1e-13, atol=1e-16) and np.allclose(pyy, p, rtol=1e-13)
        assert np.all(pxy == 0.0)


def test_quadratic_psi_gives_eq19_exactly():
    """For psi quadratic in x and y the Taylor expansion (Eq. 19) terminates:
    P = (rho/3 + G/2 psi^2 + G/12 psi lap psi) I + G/6 psi grad grad psi, using the fourth
    moment sum w e_a e_b e_c e_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/3 of Eq. 7's weights.
    Interior nodes of a walled grid (no wrap)."""
    ny, nx = 12, 14
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    c = dict(c0=0.3, cx=0.01, cy=-0.02, cxx=1e-3, cyy=2e-3, cxy=-1.5e-3)
    psi = c["c0"] + c["cx"] * x + c["cy"] * y + c["cxx"] * x * x + c["cyy"] * y * y + c["cxy"] * x * y
    rho = 0.1 + 0.001 * x
    G = -1.0
    pxx, pyy, pxy = op.pressure_tensor_from_psi(rho, psi, G, walls=True)
    lap = 2 * c["cxx"] + 2 * c["cyy"]
    iso = rho / 3 + G / 2 * psi ** 2 + G / 12 * psi * lap
    s = (slice(1, ny - 1), slice(1, nx - 1))
    assert np.allclose(pxx[s], (iso + G / 6 * psi * 2 * c["cxx"])[s], rtol=0, atol=1e-15)
    assert np.allclose(pyy[s], (iso + G / 6 * psi * 2 * c["cyy"])[s], rtol=0, atol=1e-15)
    assert np.allclose(pxy[s], (G / 6 * psi * c["cxy"])[s], rtol=0, atol=1e-15)


def test_sigma_term_is_two_sigma_force_over_psi_squared():
    """The isotropic extra term equals 2 sigma |F/psi|^2 with F of the oracle's own step
    (Eq. 7), on a droplet state."""
    T = 0.7 * wl.t_crit(A)
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    p = oracle.Params(nx=40, ny=30, a=A, b=B, R=R, T=T, sigma=0.114, s=oracle.rates_for(0.8))
    f = oracle.equilibrium(wl.droplet(40, 30, rl, rv, 9.0, 4.0))
    a0 = op.pressure_tensor(p, f)
    a1 = op.pressure_tensor(p, f, include_sigma=True)
    fl = oracle.fields(p, f)
    g2 = (fl["Fx"] ** 2 + fl["Fy"] ** 2) / fl["psi"] ** 2
    # the difference of two O(p) numbers: absolute rounding ~1e-18
    assert np.allclose(a1[0] - a0[0], 2 * 0.114 * g2, rtol=1e-12, atol=1e-16)
    assert np.allclose(a1[1] - a0[1], 2 * 0.114 * g2, rtol=1e-12, atol=1e-16)
    assert np.array_equal(a1[2], a0[2])


def test_walls_tensor_equals_the_mirrored_periodic_tensor():
    """With walls, psi at a ghost row equals psi of the adjacent fluid row (the halfway
    wall of the step), so the walled tensor equals, on the original rows, the periodic
    tensor of the field extended by its mirror image in y."""
    T = 0.7 * wl.t_crit(A)
    rng = np.random.default_rng(3)
    rho = 0.05 + 0.3 * rng.uniform(size=(9, 7))
    psi = np.vectorize(lambda r: thermo.psi(r, A, B, R, T))(rho)
    walled = op.pressure_tensor_from_psi(rho, psi, -1.0, walls=True, sigma=0.114)
    ext = lambda a: np.concatenate([a, a[::-1]], axis=0)  # noqa: E731
    periodic = op.pressure_tensor_from_psi(ext(rho), ext(psi), -1.0, sigma=0.114)
    for w, q in zip(walled, periodic):
        assert np.allclose(w, q[:9], rtol=1e-14, atol=1e-17)


def test_film_tensor_is_x_uniform_and_symmetric():
    """An x-uniform film has no shear and x-uniform components; rotating the film by 90
    degrees swaps pxx and pyy."""
    T = 0.7 * wl.t_crit(A)
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    rho = wl.flat_film(6, 40, rl, rv, 4.0, 20)
    psi = np.vectorize(lambda r: thermo.psi(r, A, B, R, T))(rho)
    pxx, pyy, pxy = op.pressure_tensor_from_psi(rho, psi, -1.0)
    assert np.all(pxy == 0.0)
    assert np.allclose(pxx, pxx[:, :1]) and np.allclose(pyy, pyy[:, :1])
    qxx, qyy, _ = op.pressure_tensor_from_psi(rho.T.copy(), psi.T.copy(), -1.0)
    assert np.allclose(qxx, pyy.T, rtol=1e-14) and np.allclose(qyy, pxx.T, rtol=1e-14)
    # bulk rows carry p_EOS; the interfaces carry a positive excess of P_n - P_t
    assert op.surface_tension_film(pxx, pyy) > 0


def test_film_surface_tension_is_the_integral_over_one_interface():
    """A constructed x-uniform film whose P_yy - P_xx is two Gaussian bumps of integral g0
    each (one per interface; sampled at the nodes their sums equal g0 to rounding) gives
    the per-interface tension g0; exchanging P_xx and P_yy flips its sign, and a part of
    P_xx that varies in x with zero mean over x leaves it unchanged."""
    import math
    ny, nx, g0 = 64, 6, 0.0123
    y = np.arange(ny, dtype=float)

    def bump(y0, s=2.0):
        return np.exp(-0.5 * ((y - y0) / s) ** 2) / (s * math.sqrt(2.0 * math.pi))
    pxx = np.full((ny, nx), 0.05)
    pyy = pxx + g0 * (bump(16.0) + bump(48.0))[:, None]
    assert op.surface_tension_film(pxx, pyy) == pytest.approx(g0, rel=1e-12)
    assert op.surface_tension_film(pyy, pxx) == pytest.approx(-g0, rel=1e-12)
    wiggle = 1e-3 * np.cos(2.0 * np.pi * np.arange(nx) / nx)[None, :]
    assert op.surface_tension_film(pxx + wiggle, pyy + wiggle) == pytest.approx(g0, rel=1e-12)
