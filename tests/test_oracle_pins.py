"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test states what it pins.  None re-types the oracle's own formula: the lattice
identities come from the textbook D2Q9 definitions, the EOS from the constants the paper
prints, the step from special cases (BGK with Guo forcing, the closed form of the sigma
term of Eq. 25, exact Taylor expansion of Eq. 7), conservation, symmetry and the
thermodynamics the paper reports (Table II, Eq. 21 with Eq. 29, Sec. IV B).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import thermo
from paper_1211_6932_gb300 import workloads as wl
from tests import textbook as tb

A, B, R = 0.25, 4.0, 1.0


def tc(a):
    return wl.t_crit(a, B, R)


def smooth_field(nx, ny, seed, base=0.2, amp=0.05):
    rng = np.random.default_rng(seed)
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    rho = np.full((ny, nx), base)
    for _ in range(3):
        kx, ky = rng.integers(1, 3, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        rho += amp / 3 * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny) + ph)
    ux = 0.02 * np.sin(2 * np.pi * y / ny + rng.uniform(0, 6))
    uy = 0.02 * np.cos(2 * np.pi * x / nx + rng.uniform(0, 6))
    return rho, ux, uy


# ---------------------------------------------------------------------------- lattice
def test_lattice_tables_match_textbook():
    """Oracle velocity set, opposites, force weights (Eq. 7: w(1)=1/3, w(2)=1/12) and the
    moment matrix equal the textbook D2Q9 / Lallemand-Luo definitions."""
    t = oracle.tables()
    assert np.array_equal(t["ex"], tb.EX) and np.array_equal(t["ey"], tb.EY)
    for a in range(9):
        assert t["ex"][t["opp"][a]] == -t["ex"][a] and t["ey"][t["opp"][a]] == -t["ey"][a]
    assert np.allclose(t["w"], tb.W_FORCE, rtol=0, atol=1e-16)
    assert np.array_equal(t["M"], tb.moment_basis())


def test_force_weights_isotropy():
    """sum w e e = I and sum w e_x^4 = 3 sum w e_x^2 e_y^2 (fourth-order isotropy)."""
    w = oracle.tables()["w"]
    ex, ey = tb.EX, tb.EY
    assert math.isclose((w * ex * ex).sum(), 1.0) and math.isclose((w * ey * ey).sum(), 1.0)
    assert abs((w * ex * ey).sum()) < 1e-16
    assert math.isclose((w * ex ** 4).sum(), 3 * (w * ex ** 2 * ey ** 2).sum())


def test_moment_matrix_orthogonal():
    M = oracle.tables()["M"]
    assert np.array_equal(M @ M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))


def test_equilibrium_moments_are_eq3():
    """M applied to the textbook second-order equilibrium gives Eq. 3, and the oracle's
    equilibrium (built as M^-1 m_eq) equals the textbook equilibrium."""
    rng = np.random.default_rng(1)
    M = oracle.tables()["M"]
    rho = rng.uniform(0.01, 0.5, (4, 5))
    ux = rng.uniform(-0.1, 0.1, (4, 5))
    uy = rng.uniform(-0.1, 0.1, (4, 5))
    feq = tb.feq(rho, ux, uy)
    m = np.tensordot(M, feq, axes=1)
    v2 = ux ** 2 + uy ** 2
    expect = np.array([rho, rho * (-2 + 3 * v2), rho * (1 - 3 * v2), rho * ux, -rho * ux,
                       rho * uy, -rho * uy, rho * (ux ** 2 - uy ** 2), rho * ux * uy])
    assert np.allclose(m, expect, rtol=0, atol=1e-15)
    assert np.allclose(oracle.equilibrium(rho, ux, uy), feq, rtol=0, atol=1e-16)


def test_guo_forcing_in_moment_space_is_eq9():
    """The moment-space forcing of Eq. 9 is M applied to Guo's velocity-space term."""
    rng = np.random.default_rng(2)
    M = oracle.tables()["M"]
    ux, uy, Fx, Fy = rng.uniform(-0.1, 0.1, 4)
    S = tb.guo_source(ux, uy, Fx, Fy)
    vF = ux * Fx + uy * Fy
    expect = [0, 6 * vF, -6 * vF, Fx, -Fx, Fy, -Fy, 2 * (ux * Fx - uy * Fy), ux * Fy + uy * Fx]
    assert np.allclose(M @ S, expect, rtol=0, atol=1e-16)


# ------------------------------------------------------------------------------- EOS
def test_cs_critical_point_matches_printed_constants(golden):
    """Critical point of the oracle's Eq. 30 (dp/drho = d2p/drho2 = 0, found from the
    C oracle's p_EOS by finite differences) reproduces rho_c = 0.5218/b, a = 10.601 R T_c
    (b = 4) and p_c = 0.070663 a/b^2 printed in Sec. IV."""
    g = golden["paper_constants"]
    rc, Tc, pc = thermo.critical_point(1.0, B, R)
    # The C oracle's pressure has a van der Waals loop just below T_c and none above.
    grid = np.linspace(0.02, 0.6, 3001)

    def monotone(T):
        p = np.array([oracle.p_eos(r, 1.0, B, R, T) for r in grid])
        return bool(np.all(np.diff(p) > 0))

    assert monotone(Tc * 1.0005) and not monotone(Tc * 0.9995)
    assert math.isclose(oracle.p_eos(rc, 1.0, B, R, Tc), pc, rel_tol=1e-12)
    assert math.isclose(rc * B, g["rho_c_times_b"][0], rel_tol=2e-4)
    assert math.isclose(1.0 / (R * Tc), g["a_over_RTc_b4"][0], rel_tol=2e-4)
    assert math.isclose(pc * B * B / 1.0, g["pc_b2_over_a"][0], rel_tol=2e-4)
    for key, a in (("Tc_a1", 1.0), ("Tc_a05", 0.5), ("Tc_a025", 0.25)):
        assert math.isclose(thermo.critical_point(a, B, R)[1], g[key][0], rel_tol=4e-3)
    # Eq. 33 / App. B constants
    assert math.isclose(B * rc / 4, g["bx_coeff_eq33"][0], rel_tol=2e-4)
    assert math.isclose(rc * R * Tc / pc, g["eq33_prefactor"][0], rel_tol=2e-4)
    assert math.isclose(1.0 * rc / (R * Tc), g["eq33_attraction"][0], rel_tol=2e-4)


def test_psi_reproduces_eos_through_eq11():
    """With psi from Eq. 24 the LB equation of state of Eq. 11 equals p_EOS."""
    for rho in (1e-4, 3e-3, 0.05, 0.13, 0.3, 0.45):
        for T in (0.5 * tc(A), 0.9 * tc(A)):
            psi = oracle.psi(rho, A, B, R, T, -1.0)
            p_lb = rho / 3.0 + (-1.0) / 2.0 * psi ** 2
            assert math.isclose(p_lb, oracle.p_eos(rho, A, B, R, T), rel_tol=1e-12,
                                abs_tol=1e-18)


def test_psi_clamps_a_negative_argument_to_zero():
    """Reading of Eq. 24 (G < 0): where p_EOS exceeds rho c_s^2, which the CS EOS does at
    liquid densities well above coexistence (here rho >= 0.7 at T = 0.7 T_c), the square
    root's argument is negative; psi is taken as zero there, by the C step and the Python
    thermodynamics alike, and stays positive below that density."""
    T = 0.7 * tc(A)
    for rho in (0.7, 0.8, 0.95):
        assert oracle.p_eos(rho, A, B, R, T) > rho / 3.0
        assert oracle.psi(rho, A, B, R, T, -1.0) == 0.0
        assert thermo.psi(rho, A, B, R, T, -1.0) == 0.0
    for rho in (0.01, 0.3, 0.6):
        assert oracle.psi(rho, A, B, R, T, -1.0) > 0.0


def test_maxwell_matches_table_ii(golden):
    """Maxwell construction (Eq. 22) against the Maxwell column of Table II (a = 0.25,
    T_c = 0.0235, Sec. IV C).  Liquid within the printed digits; vapour within 0.5 %
    (the T/Tc = 0.55 entry is 0.4 % off the exact construction at the rounded T_c)."""
    for key, (rl_p, rv_p) in golden["table_ii_maxwell"].items():
        rl, rv, p0 = thermo.maxwell(A, B, R, float(key) * 0.0235)
        assert abs(rl - rl_p) <= 6e-4, (key, rl, rl_p)
        assert abs(rv - rv_p) / rv_p <= 5e-3, (key, rv, rv_p)
        # the construction: equal pressures
        assert math.isclose(oracle.p_eos(rl, A, B, R, float(key) * 0.0235),
                            oracle.p_eos(rv, A, B, R, float(key) * 0.0235), rel_tol=1e-9)


def test_maxwell_equal_chemical_potential_closed_form():
    """Independent check of the quadrature Maxwell solver: the CS free energy gives
    int p/rho^2 = R T [ln rho + (4x - 3x^2)/(1-x)^2] - a rho, so equal areas mean
    p0 (1/rho_v - 1/rho_l) = Phi(rho_l) - Phi(rho_v)."""
    for a in (0.125, 0.5, 1.0):
        for tr in (0.5, 0.7, 0.9):
            T = tr * tc(a)
            rl, rv, p0 = thermo.maxwell(a, B, R, T)

            def phi(r):
                x = B * r / 4
                return R * T * (math.log(r) + (4 * x - 3 * x * x) / (1 - x) ** 2) - a * r

            lhs = p0 * (1 / rv - 1 / rl)
            assert math.isclose(lhs, phi(rl) - phi(rv), rel_tol=1e-9)


def test_epsilon_sigma_relation(golden):
    """Eq. 29 with G = -1, alpha = 0, beta = 3: the (sigma, epsilon) pairs of the paper."""
    g = golden["paper_constants"]
    for key in ("eps_sigma_0125", "eps_sigma_011", "eps_sigma_0114"):
        sig, eps = g[key]
        assert math.isclose(thermo.epsilon_from_sigma(sig, -1.0), eps, rel_tol=1e-12)


# ------------------------------------------------------------------------------ step
def psi_fn(a, T, G=-1.0):
    return lambda r: oracle.psi(r, a, B, R, T, G)


def test_bgk_guo_special_case():
    """All rates equal 1/tau and sigma = 0: the MRT step is BGK with Guo forcing, written
    here in velocity space from the textbook form."""
    nx, ny = 7, 6
    T = 0.8 * tc(A)
    rho, ux, uy = smooth_field(nx, ny, 3)
    f = tb.feq(rho, ux, uy) * (1 + 0.01 * np.random.default_rng(4).standard_normal((9, ny, nx)))
    for tau in (0.6, 1.0, 1.7):
        p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, G=-1.0, sigma=0.0,
                          s=(1 / tau,) * 9)
        got = oracle.run(p, f, 1)
        ref = tb.bgk_guo_step(f, tau, psi_fn(A, T), -1.0)
        assert np.max(np.abs(got - ref)) < 1e-15, tau


def test_velocity_space_mrt_brute_force():
    """Eq. 1 in velocity space with Lambda_bar = M^-1 Lambda M (M built from its polynomial
    definition, inverted numerically) agrees with the oracle's moment-space step on tiny
    grids, for several rate vectors, sigma values and steps."""
    T = 0.7 * tc(A)
    for (nx, ny) in ((4, 4), (5, 3)):
        rho, ux, uy = smooth_field(nx, ny, 5, base=0.15)
        f = tb.feq(rho, ux, uy)
        for s, sig in (((1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25), 0.114),
                       ((0.9, 1.3, 0.7, 1.2, 1.5, 0.8, 1.1, 1.6, 0.9), 0.05)):
            p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, sigma=sig, s=s)
            g = f.copy()
            got = oracle.run(p, f, 10)
            for _ in range(10):
                g = tb.velocity_space_mrt_step(g, s, sig, psi_fn(A, T), -1.0)
            assert np.max(np.abs(got - g)) < 1e-13


def test_sigma_term_closed_form():
    """Eq. 25 minus Eq. 9, after (I - Lambda/2), changes the post-collision moments by
    exactly +s_e 12 sigma |F|^2/psi^2 (energy) and -s_zeta 12 sigma |F|^2/psi^2
    (energy square), because (1 - s/2)/(tau - 1/2) = s.  Check on the streamed result."""
    nx, ny = 9, 8
    T = 0.7 * tc(A)
    rho, ux, uy = smooth_field(nx, ny, 6, base=0.12, amp=0.1)
    f = oracle.equilibrium(rho, ux, uy)
    s = (1.0, 1.3, 0.8, 1.0, 1.1, 1.0, 1.1, 1.2, 1.2)
    sig = 0.11
    p0 = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, sigma=0.0, s=s)
    p1 = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, sigma=sig, s=s)
    diff = oracle.run(p1, f, 1) - oracle.run(p0, f, 1)
    fl = oracle.fields(p0, f)
    X = 12 * sig * (fl["Fx"] ** 2 + fl["Fy"] ** 2) / fl["psi"] ** 2
    M = tb.moment_basis()
    dm = np.zeros((9,) + X.shape)
    dm[1] = s[1] * X
    dm[2] = -s[2] * X
    df = np.tensordot(np.linalg.inv(M), dm, axes=1)
    expect = tb.stream_periodic(df)
    assert np.max(np.abs(diff - expect)) < 1e-16 + 1e-12 * np.max(np.abs(expect))
    assert np.max(np.abs(expect)) > 1e-8


def test_force_matches_taylor_expansion_for_cubic_psi():
    """For psi cubic in (x, y), Eq. 7 with w(1) = 1/3, w(2) = 1/12 equals the expansion of
    Eq. 8, -G psi [grad psi + (1/6) grad(lap psi)], exactly (the next term is fifth
    order).  psi is set by inverting Eq. 24 on the vapour branch."""
    T = 0.7 * tc(A)
    G = -1.0
    nx, ny = 24, 24
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    cx, cy = 11.5, 11.5
    X, Y = (x - cx) / 12.0, (y - cy) / 12.0
    psi_t = 0.06 + 0.01 * (X + 0.5 * Y + 0.3 * X * X - 0.2 * X * Y + 0.4 * X ** 3
                            + 0.3 * X * Y * Y - 0.2 * Y ** 3)
    # invert psi(rho) on the vapour branch (monotone on (0, spinodal))
    from scipy.optimize import brentq
    s1 = thermo._spinodals(A, B, R, T)[0]
    rho = np.vectorize(lambda t: brentq(lambda r: oracle.psi(r, A, B, R, T, G) - t,
                                        1e-12, s1, xtol=1e-17, rtol=1e-15))(psi_t)
    f = oracle.equilibrium(rho)
    fl = oracle.fields(oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, G=G), f)
    assert np.max(np.abs(fl["psi"] - psi_t)) < 1e-14
    s = 1.0 / 12.0
    px = 0.01 * s * (1 + 0.6 * X - 0.2 * Y + 1.2 * X * X + 0.3 * Y * Y)
    py = 0.01 * s * (0.5 - 0.2 * X + 0.6 * X * Y - 0.6 * Y * Y)
    # lap psi = 0.01 s^2 (0.6 + 2.4 X + 0.6 X - 1.2 Y) ; its gradient:
    lx = 0.01 * s ** 3 * (2.4 + 0.6)
    ly = 0.01 * s ** 3 * (-1.2)
    Fx = -G * psi_t * (px + lx / 6.0)
    Fy = -G * psi_t * (py + ly / 6.0)
    inner = (slice(3, ny - 3), slice(3, nx - 3))
    assert np.max(np.abs(fl["Fx"][inner] - Fx[inner])) < 1e-15
    assert np.max(np.abs(fl["Fy"][inner] - Fy[inner])) < 1e-15


def test_uniform_state_is_fixed_point():
    for sig in (0.0, 0.114):
        p = oracle.Params(nx=5, ny=4, a=A, b=B, R=R, T=0.6 * tc(A), sigma=sig)
        f = oracle.equilibrium(np.full((4, 5), 0.3))
        assert np.max(np.abs(oracle.run(p, f, 20) - f)) < 1e-15


@pytest.mark.parametrize("walls", [False, True])
def test_mass_and_momentum_conservation(walls):
    """Mass is conserved (periodic or walls); total momentum sum e f changes by sum F
    per step, which is zero in a periodic domain (pairwise antisymmetry of Eq. 7)."""
    nx, ny = 16, 12
    rho, ux, uy = smooth_field(nx, ny, 7, base=0.2, amp=0.08)
    p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=0.7 * tc(A), sigma=0.114,
                      s=oracle.rates_for(0.8), walls=walls)
    f0 = oracle.equilibrium(rho, ux, uy)
    f1 = oracle.run(p, f0, 50)
    assert math.isclose(f1.sum(), f0.sum(), rel_tol=1e-13)
    if not walls:
        for e in (tb.EX, tb.EY):
            m0 = np.tensordot(e, f0, axes=1).sum()
            m1 = np.tensordot(e, f1, axes=1).sum()
            assert abs(m1 - m0) < 1e-13 * f0.sum()


def test_translation_invariance_is_exact():
    nx, ny = 12, 10
    rho, ux, uy = smooth_field(nx, ny, 8)
    p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=0.7 * tc(A), sigma=0.114)
    f = oracle.equilibrium(rho, ux, uy)
    a = oracle.run(p, f, 5)
    b = oracle.run(p, np.roll(f, (3, -4), axis=(1, 2)), 5)
    assert np.array_equal(np.roll(a, (3, -4), axis=(1, 2)), b)


def test_rotation_by_90_degrees():
    """Rotating the initial state by 90 degrees rotates the result (x -> y, y -> -x maps
    velocity a to rot[a]).  Catches x/y and sign mix-ups in Eqs. 6, 7, 9, 25."""
    n = 10
    rho, ux, uy = smooth_field(n, n, 9)
    s = (1.0, 1.1, 1.2, 1.0, 1.3, 1.0, 1.3, 1.25, 1.25)
    p = oracle.Params(nx=n, ny=n, a=A, b=B, R=R, T=0.7 * tc(A), sigma=0.114, s=s)
    f = oracle.equilibrium(rho, ux, uy)
    # np.rot90 maps node (x, y) to (y, n-1-x): a clockwise quarter turn, under which
    # e_a becomes e_rot[a].
    rot = [0, 4, 1, 2, 3, 8, 5, 6, 7]

    def rotate(g):
        out = np.empty_like(g)
        for a in range(9):
            out[rot[a]] = np.rot90(g[a], k=1)
        return out

    a1 = rotate(oracle.run(p, f, 4))
    a2 = oracle.run(p, rotate(f), 4)
    assert np.max(np.abs(a1 - a2)) < 1e-14


@pytest.mark.parametrize("visc", ["const", "linear"])
def test_axis_exchange_on_a_rectangular_lattice(visc):
    """Exchanging x and y (node (x, y) -> (y, x), velocity e_a -> its mirror image in the
    diagonal) maps the update of an nx x ny lattice onto that of the ny x nx lattice: the
    symmetry that lets a batch store an instance transposed.  A reflection, not a
    rotation: it flips the sign of p_xx, so a wrong sign or a mixed-up rate of the p_xx
    row of Eqs. 3, 25 fails it where the quarter turn above would not."""
    nx, ny = 11, 7
    rho, ux, uy = smooth_field(nx, ny, 10)
    s = (1.0, 1.1, 1.2, 1.0, 1.3, 1.0, 1.3, 1.25, 1.25)
    kw = dict(a=A, b=B, R=R, T=0.7 * tc(A), sigma=0.114, s=s)
    if visc == "linear":
        rl, rv, _ = thermo.maxwell(A, B, R, 0.7 * tc(A))
        kw.update(visc_mode=oracle.VISC_LINEAR, nu_l=0.05, nu_v=0.2, rho_l=rl, rho_v=rv)
    p = oracle.Params(nx=nx, ny=ny, **kw)
    pt = oracle.Params(nx=ny, ny=nx, **kw)
    f = oracle.equilibrium(rho, ux, uy)
    mirror = [0, 2, 1, 4, 3, 5, 8, 7, 6]  # (ex, ey) -> (ey, ex)

    def exchange(g):
        return np.stack([g[mirror[a]].T for a in range(9)])

    a1 = exchange(oracle.run(p, f, 6))
    a2 = oracle.run(pt, exchange(f), 6)
    assert a2.shape == (9, nx, ny)
    assert np.max(np.abs(a1 - a2)) < 1e-14


@pytest.mark.parametrize("mode,rho0", [("const", 0.4), ("step", 0.4), ("step", 0.005),
                                       ("linear", 0.32), ("linear", 0.4)])
def test_shear_wave_decay_gives_viscosity(mode, rho0):
    """Single-phase shear wave u_x = U sin(2 pi y / ny) decays at exp(-nu k^2 t), with nu
    from Eq. 10 (nu = (tau - 1/2)/3) and the viscosity mode's choice of tau (Sec. IV C).
    Densities lie outside the spinodal region, so the uniform state is stable."""
    nx, ny, U, steps = 4, 32, 1e-5, 400
    T = 0.7 * tc(A)
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    if mode == "const":
        tau = 0.9
        p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, s=oracle.rates_for(tau))
    elif mode == "step":
        nu_l, nu_v = 0.05, 0.2
        tau = 3 * (nu_l if rho0 >= 0.5218 / B else nu_v) + 0.5
        p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, visc_mode=oracle.VISC_STEP,
                          nu_l=nu_l, nu_v=nu_v, rho_c=0.5218 / B)
    else:
        nu_l, nu_v = 0.05, 0.2
        fr = min(max((rho0 - rv) / (rl - rv), 0.0), 1.0)
        tau = (3 * nu_v + 0.5) + fr * ((3 * nu_l + 0.5) - (3 * nu_v + 0.5))
        p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, visc_mode=oracle.VISC_LINEAR,
                          nu_l=nu_l, nu_v=nu_v, rho_l=rl, rho_v=rv)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    k = 2 * np.pi / ny
    f = oracle.equilibrium(np.full((ny, nx), rho0), U * np.sin(k * y), np.zeros((ny, nx)))
    f = oracle.run(p, f, steps)
    u = oracle.fields(p, f)["ux"][:, 0]
    amp = 2 * np.mean(u * np.sin(k * np.arange(ny)))
    nu = (tau - 0.5) / 3
    assert math.isclose(amp / U, math.exp(-nu * k * k * steps), rel_tol=5e-3)


def test_walls_no_slip_shear_wave():
    """Between halfway bounce-back walls at y = -1/2 and ny - 1/2 the mode
    sin(pi (y + 1/2)/ny) vanishes on the walls and decays at exp(-nu (pi/ny)^2 t)."""
    nx, ny, U, steps, tau = 4, 24, 1e-5, 400, 0.9
    T = 0.7 * tc(A)
    p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, s=oracle.rates_for(tau), walls=True)
    yy = (np.arange(ny) + 0.5)[:, None] * np.ones((1, nx))
    k = np.pi / ny
    f = oracle.equilibrium(np.full((ny, nx), 0.4), U * np.sin(k * yy), np.zeros((ny, nx)))
    f = oracle.run(p, f, steps)
    u = oracle.fields(p, f)["ux"][:, 0]
    amp = 2 * np.mean(u * np.sin(k * (np.arange(ny) + 0.5)))
    assert math.isclose(amp / U, math.exp(-(tau - 0.5) / 3 * k * k * steps), rel_tol=1e-2)


def test_walls_film_equals_mirrored_periodic_film():
    """An x-uniform film on a bottom wall is the mirror image of a periodic domain twice
    as tall (bounce-back equals specular reflection there; the ghost psi mirrors)."""
    nx, ny = 3, 24
    T = 0.7 * tc(A)
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    prof = wl.tanh_profile(np.arange(ny) - 7.5, rl, rv, 4.0)
    rho_w = np.repeat(prof[:, None], nx, axis=1)
    rho_p = np.vstack([rho_w[::-1], rho_w])  # rows -ny..-1 mirror rows 0..ny-1
    s = oracle.rates_for(0.8)
    pw = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=T, sigma=0.114, s=s, walls=True)
    pp = oracle.Params(nx=nx, ny=2 * ny, a=A, b=B, R=R, T=T, sigma=0.114, s=s)
    fw = oracle.run(pw, oracle.equilibrium(rho_w), 200)
    fp = oracle.run(pp, oracle.equilibrium(rho_p), 200)
    assert np.max(np.abs(fw - fp[:, ny:, :])) < 1e-13


# --------------------------------------------------------------------- thermodynamics
def film_equilibrium(a, tr, sigma, tau=0.8, ny=128, steps=20000, W=5.0):
    T = tr * tc(a)
    rl, rv, _ = thermo.maxwell(a, B, R, T)
    rho = wl.flat_film(3, ny, rl, rv, W, ny / 2)
    p = oracle.Params(nx=3, ny=ny, a=a, b=B, R=R, T=T, sigma=sigma, s=oracle.rates_for(tau))
    f = oracle.run(p, oracle.equilibrium(rho), steps)
    r = oracle.fields(p, f)["rho"][:, 0]
    return r, (r[ny // 2], r[0]), (rl, rv)


@pytest.mark.parametrize("sigma", [0.0, 0.114])
def test_flat_film_follows_mechanical_stability(sigma):
    """Flat-film coexistence densities of the full step agree with the mechanical-
    stability condition of Eq. 21 with epsilon from Eq. 29 (epsilon = -16 G sigma).
    T/Tc = 0.9, a = 0.25."""
    _, (l, v), _ = film_equilibrium(A, 0.9, sigma)
    ml, mv, _ = thermo.mechanical_stability(A, B, R, 0.9 * tc(A), -1.0,
                                            thermo.epsilon_from_sigma(sigma))
    assert abs(l - ml) / ml < 2e-3 and abs(v - mv) / mv < 5e-3


def test_improved_forcing_is_thermodynamically_consistent():
    """Sec. III-IV A: with sigma = 0.114 (a = 0.25) the film coexistence densities match
    the Maxwell construction, while the original scheme (sigma = 0) misses the vapour
    density by far more (T/Tc = 0.85)."""
    _, (l1, v1), (rl, rv) = film_equilibrium(A, 0.85, 0.114)
    _, (l0, v0), _ = film_equilibrium(A, 0.85, 0.0)
    assert abs(l1 - rl) / rl < 2e-3 and abs(v1 - rv) / rv < 2e-2
    assert abs(v0 - rv) / rv > 5 * abs(v1 - rv) / rv


def table_ii_droplet(a, tr, sigma, tc_value, steps, n=200, r0=50):
    """The stationary-droplet run behind Table II; returns (rho_centre, rho_corner)."""
    T = tr * tc_value
    rl, rv, _ = thermo.maxwell(a, B, R, T)
    p = oracle.Params(nx=n, ny=n, a=a, b=B, R=R, T=T, sigma=sigma, s=oracle.rates_for(0.8))
    f = oracle.run(p, oracle.equilibrium(wl.droplet(n, n, rl, rv, r0, 5.0)), steps)
    r = oracle.fields(p, f)["rho"]
    return r[n // 2, n // 2], r[0, 0]


@pytest.mark.slow
def test_table_ii_numerical_droplet(golden):
    """The oracle's stationary droplet (a = 0.25, T/Tc = 0.6, sigma = 0.114) reproduces the
    numerical column of Table II to the printed digits."""
    l_p, v_p = golden["table_ii_numerical"]["a0.25_0.60"]
    l, v = table_ii_droplet(0.25, 0.6, 0.114, 0.0235, 20000)
    assert abs(l - l_p) <= 1e-4 and abs(v - v_p) / v_p <= 5e-3, (l, v)


def fitted_width(profile):
    from scipy.optimize import curve_fit
    ny = profile.size
    y = np.arange(ny, dtype=float)
    half = slice(0, ny // 2)  # lower interface
    rl, rv = profile.max(), profile.min()

    def model(yy, y0, W, lo, hi):
        return 0.5 * (hi + lo) + 0.5 * (hi - lo) * np.tanh(2 * (yy - y0) / W)

    p, _ = curve_fit(model, y[half], profile[half], p0=[ny / 4, 5.0, rv, rl])
    return abs(p[1])


def test_interface_width_scales_like_inverse_sqrt_a(golden):
    """Sec. IV B / Fig. 3: widths at a = 0.25 and 0.5 are about 1.9 and 1.4 times the
    width at a = 1 (T/Tc = 0.7); checked within 10 %."""
    g = golden["width_ratios"]
    widths = {}
    for a in (1.0, 0.5, 0.25):
        prof, _, _ = film_equilibrium(a, 0.7, wl.sigma0(a), ny=96, steps=12000)
        widths[a] = fitted_width(prof)
    assert math.isclose(widths[0.25] / widths[1.0], g["a_025"][0], rel_tol=0.1)
    assert math.isclose(widths[0.5] / widths[1.0], g["a_05"][0], rel_tol=0.1)


@pytest.mark.slow
def test_laplace_law():
    """Droplets of several radii: the pressure jump (Eq. 11 pressure = p_EOS at the
    centre minus far field) grows linearly with 1/R (positive slope = surface tension).
    The radii here (9-19 nodes, interface width ~4) are small enough that curvature
    corrections leave an intercept of ~25 % of the smallest jump; the GPU suite repeats
    this with radii up to 40."""
    n = 64
    T = 0.7 * tc(A)
    rl, rv, _ = thermo.maxwell(A, B, R, T)
    inv_r, dp = [], []
    for r0 in (10, 13, 16, 19):
        p = oracle.Params(nx=n, ny=n, a=A, b=B, R=R, T=T, sigma=0.114, s=oracle.rates_for(1.0))
        f = oracle.run(p, oracle.equilibrium(wl.droplet(n, n, rl, rv, r0, 4.0)), 6000)
        rho = oracle.fields(p, f)["rho"]
        pin = oracle.p_eos(rho[n // 2, n // 2], A, B, R, T)
        pout = oracle.p_eos(rho[0, 0], A, B, R, T)
        mass_excess = (rho - rho[0, 0]).sum() / (rho[n // 2, n // 2] - rho[0, 0])
        inv_r.append(1.0 / math.sqrt(mass_excess / math.pi))
        dp.append(pin - pout)
    slope, icpt = np.polyfit(inv_r, dp, 1)
    fit = np.polyval([slope, icpt], inv_r)
    r2 = 1 - np.sum((dp - fit) ** 2) / np.sum((dp - np.mean(dp)) ** 2)
    assert slope > 0 and r2 > 0.98 and abs(icpt) < 0.35 * min(dp)


def test_conserved_moment_rates_have_no_effect():
    """s_rho, s_j relax conserved moments (m - m_eq = 0 for rho and j): any values give
    bitwise the same run."""
    nx, ny = 14, 11
    rho, ux, uy = smooth_field(nx, ny, 9, base=0.2, amp=0.08)
    f0 = oracle.equilibrium(rho, ux, uy)
    outs = []
    for s0, s3 in ((1.0, 1.0), (0.7, 1.3), (1.9, 0.4)):
        s = list(oracle.rates_for(0.8))
        s[0], s[3], s[5] = s0, s3, s3
        p = oracle.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=0.7 * tc(A), sigma=0.114, s=tuple(s))
        outs.append(oracle.run(p, f0, 6))
    # M^-1 applied to the same post-collision moments: equal to rounding of the back
    # transformation (the relaxed conserved moments equal their equilibria exactly)
    assert np.max(np.abs(outs[1] - outs[0])) < 1e-15 and np.max(np.abs(outs[2] - outs[0])) < 1e-15


def test_centred_droplet_stays_mirror_symmetric():
    """A droplet centred on the domain keeps its x and y mirror symmetry (Sec. IV A's
    stationary droplet): to 1e-13 after 200 steps."""
    n = 40
    rl, rv, _ = thermo.maxwell(A, B, R, 0.7 * tc(A))
    p = oracle.Params(nx=n, ny=n, a=A, b=B, R=R, T=0.7 * tc(A), sigma=0.114,
                      s=oracle.rates_for(0.8))
    f = oracle.run(p, oracle.equilibrium(wl.droplet(n, n, rl, rv, 10.0, 4.0)), 200)
    r = oracle.fields(p, f)["rho"]
    assert np.max(np.abs(r - r[:, ::-1])) < 1e-13 and np.max(np.abs(r - r[::-1, :])) < 1e-13
    assert np.max(np.abs(r - r.T)) < 1e-13


def test_x_uniform_film_is_independent_of_nx():
    """An x-uniform film evolves the same on a 3-wide strip and an 8-wide one."""
    rl, rv, _ = thermo.maxwell(A, B, R, 0.7 * tc(A))
    outs = []
    for nx in (3, 8):
        p = oracle.Params(nx=nx, ny=40, a=A, b=B, R=R, T=0.7 * tc(A), sigma=0.114,
                          s=oracle.rates_for(0.8))
        f = oracle.run(p, oracle.equilibrium(wl.flat_film(nx, 40, rl, rv, 4.0, 20)), 100)
        outs.append(oracle.fields(p, f)["rho"])
    assert np.max(np.abs(outs[0][:, 0] - outs[1][:, 5])) < 1e-14


# ---------------------------------------------------------------------- Eq. 32 (Lamb)
def _energy_method_omega2(n, gamma, rho_l, r0, eps=1e-3, m=4096):
    """omega^2 of mode n of an inviscid 2D liquid cylinder by Rayleigh's energy method,
    computed by quadrature and finite differences, not from Eq. 32.

    Shape r(theta) = c(e) (1 + e cos n theta), with c(e) chosen so the enclosed area stays
    pi r0^2 exactly.  Potential energy = gamma * (perimeter - 2 pi r0), both integrals by
    the periodic trapezoid rule (spectrally accurate); its second derivative in e at 0 by
    central differences with Richardson extrapolation.  Kinetic energy = rho/2 * surface integral of phi dphi/dr for
    the interior potential phi = (r0^2 de/dt / n) (r/r0)^n cos n theta whose normal
    velocity at r = r0 is r0 de/dt cos n theta; its coefficient of (de/dt)^2 by the same
    quadrature."""
    th = 2.0 * np.pi * np.arange(m) / m
    cosn, sinn = np.cos(n * th), np.sin(n * th)
    dth = 2.0 * np.pi / m

    def perimeter(e):
        g = 1.0 + e * cosn
        c = r0 / math.sqrt(0.5 * np.sum(g * g) * dth / math.pi)  # area = pi r0^2
        r, dr = c * g, -c * e * n * sinn
        return float(np.sum(np.sqrt(r * r + dr * dr)) * dth)

    def d2(h):
        return (perimeter(h) - 2.0 * perimeter(0.0) + perimeter(-h)) / (h * h)

    d2pe = gamma * (4.0 * d2(eps / 2.0) - d2(eps)) / 3.0  # Richardson: O(eps^4) error
    # KE = (rho/2) * int phi phi_r r0 dtheta with phi = (r0^2/n) cos, phi_r = r0 cos per
    # unit de/dt: coefficient of (de/dt)^2 doubled gives the effective mass
    mass = rho_l * float(np.sum((r0 * r0 / n) * cosn * r0 * cosn * r0) * dth)
    return d2pe / mass


@pytest.mark.parametrize("n", [2, 3, 5])
def test_lamb_period_matches_energy_method(n):
    """Eq. 32 against Rayleigh's energy method for the same cylinder, worked out by
    numerical quadrature of the perimeter and of the flow's kinetic energy (no closed form
    shared with the oracle): the periods agree to 1e-6 for modes 2, 3 and 5 at two
    radii, tensions and densities."""
    for gamma, rho_l, r0 in ((0.011, 0.4, 28.46), (0.0052, 0.2, 60.0)):
        om2 = _energy_method_omega2(n, gamma, rho_l, r0)
        expect = 2.0 * math.pi / math.sqrt(om2)
        assert thermo.lamb_period(gamma, rho_l, r0, n) == pytest.approx(expect, rel=1e-6)


def test_lamb_period_planar_capillary_limit():
    """For large n the interface is locally flat: Eq. 32 must tend to the planar
    capillary-wave dispersion omega^2 = gamma k^3 / rho_l with k = n / R0, the
    relative difference falling like 1 / (2 n^2)."""
    gamma, rho_l, r0 = 0.005, 0.41, 40.0
    for n in (20, 200, 2000):
        k = n / r0
        planar = 2.0 * math.pi / math.sqrt(gamma * k ** 3 / rho_l)
        rel = thermo.lamb_period(gamma, rho_l, r0, n) / planar - 1.0
        assert rel == pytest.approx(0.5 / n ** 2, rel=0.02)
