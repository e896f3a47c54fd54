"""Thermodynamics of the Carnahan-Starling fluid, FP64 (test infrastructure only).

Each function restates one relation of Li, Luo & Li (arXiv:1211.6932):

  p_eos                 Eq. 30, the Carnahan-Starling equation of state.
  psi                   Eq. 24, the pseudopotential that reproduces p_eos (c = 1).
  critical_point        the point where dp/drho = d2p/drho2 = 0 (Sec. IV A, App. B).
  maxwell               Eq. 22, the Maxwell equal-area rule, by adaptive quadrature.
  epsilon_from_sigma    Eq. 29: eps = -2 (alpha + 24 G sigma) / beta, alpha = 0, beta = 3.
  mechanical_stability  Eq. 21, the coexistence densities the LB model selects.
  lamb_period           Eq. 32, the 2D droplet oscillation period.

Lattice units, c_s^2 = 1/3.  numpy and scipy only.
"""
import math

from scipy import integrate, optimize

CS2 = 1.0 / 3.0


def _Z(x):
    """Compressibility factor of Eq. 30: (1 + x + x^2 - x^3) / (1 - x)^3."""
    return (1.0 + x + x * x - x ** 3) / (1.0 - x) ** 3


def _Z_derivs(x):
    """Z, dZ/dx and d2Z/dx2 by differentiating numerator N and (1 - x)^-3 term by term."""
    N = 1.0 + x + x * x - x ** 3
    N1 = 1.0 + 2.0 * x - 3.0 * x * x
    N2 = 2.0 - 6.0 * x
    u = 1.0 - x
    Z = N / u ** 3
    Z1 = N1 / u ** 3 + 3.0 * N / u ** 4
    Z2 = N2 / u ** 3 + 6.0 * N1 / u ** 4 + 12.0 * N / u ** 5
    return Z, Z1, Z2


def p_eos(rho, a, b, R, T):
    """Eq. 30."""
    x = b * rho / 4.0
    return rho * R * T * _Z(x) - a * rho * rho


def dp_drho(rho, a, b, R, T):
    x = b * rho / 4.0
    Z, Z1, _ = _Z_derivs(x)
    return R * T * (Z + x * Z1) - 2.0 * a * rho


def psi(rho, a, b, R, T, G=-1.0):
    """Eq. 24 with c = 1; a negative argument is clamped to zero."""
    arg = 2.0 * (p_eos(rho, a, b, R, T) - rho * CS2) / G
    return math.sqrt(max(arg, 0.0))


def dpsi_drho(rho, a, b, R, T, G=-1.0):
    """psi' from 2 psi psi' = 2 (p' - c_s^2) / G."""
    return (dp_drho(rho, a, b, R, T) - CS2) / (G * psi(rho, a, b, R, T, G))


def critical_point(a, b, R=1.0):
    """(rho_c, T_c, p_c) where dp/drho = d2p/drho2 = 0.

    With x = b rho / 4 the two conditions give R T = 2a / ((b/4)(2 Z' + x Z'')) and
    Z + x Z' = x (2 Z' + x Z''), a single equation for x on (0, 1).
    """
    def g(x):
        Z, Z1, Z2 = _Z_derivs(x)
        return (Z + x * Z1) - x * (2.0 * Z1 + x * Z2)

    xc = optimize.brentq(g, 0.01, 0.5, xtol=1e-15, rtol=1e-15, maxiter=200)
    _, Z1, Z2 = _Z_derivs(xc)
    Tc = 2.0 * a / ((b / 4.0) * (2.0 * Z1 + xc * Z2)) / R
    rho_c = 4.0 * xc / b
    return rho_c, Tc, p_eos(rho_c, a, b, R, Tc)


def _spinodals(a, b, R, T):
    """Densities where dp/drho = 0 (below T_c), found by bracketing on a fine grid."""
    rmax = 4.0 / b
    n = 4000
    grid = [rmax * (i + 0.5) / n for i in range(n)]
    vals = [dp_drho(r, a, b, R, T) for r in grid]
    roots = []
    for i in range(n - 1):
        if vals[i] == 0.0 or (vals[i] > 0) != (vals[i + 1] > 0):
            roots.append(optimize.brentq(dp_drho, grid[i], grid[i + 1], args=(a, b, R, T),
                                         xtol=1e-16, rtol=1e-15, maxiter=200))
    if len(roots) < 2:
        raise ValueError("temperature is not below the critical temperature")
    return roots[0], roots[1]


def _outer_roots(p0, a, b, R, T, s1, s2):
    """Vapour root on (0, s1) and liquid root on (s2, 4/b) of p_eos(rho) = p0."""
    f = lambda r: p_eos(r, a, b, R, T) - p0  # noqa: E731
    rv = optimize.brentq(f, 1e-300, s1, xtol=1e-18, rtol=1e-15, maxiter=500)
    hi = 4.0 / b * (1.0 - 1e-12)
    rl = optimize.brentq(f, s2, hi, xtol=1e-18, rtol=1e-15, maxiter=500)
    return rv, rl


def _coexistence(weight, a, b, R, T):
    """Solve int_{rho_v}^{rho_l} (p0 - p_eos) weight(rho) drho = 0 for p0 (Eqs. 21, 22)."""
    s1, s2 = _spinodals(a, b, R, T)
    p_hi = p_eos(s1, a, b, R, T)
    p_lo = max(p_eos(s2, a, b, R, T), 0.0)
    span = p_hi - p_lo

    def area(p0):
        rv, rl = _outer_roots(p0, a, b, R, T, s1, s2)
        # Integrate in u = ln(rho) (d rho = rho du), piecewise between the roots and the
        # spinodals; the absolute tolerance is scaled by the size of the pieces because
        # the signed total vanishes at the solution.
        def g(u):
            r = math.exp(u)
            return (p0 - p_eos(r, a, b, R, T)) * weight(r) * r

        edges = [math.log(r) for r in [rv] + [r for r in (s1, s2) if rv < r < rl] + [rl]]
        pieces = list(zip(edges[:-1], edges[1:]))
        scale = sum(abs(integrate.quad(g, u, v, epsabs=0.0, epsrel=1e-6, limit=200)[0])
                    for u, v in pieces)
        total = sum(integrate.quad(g, u, v, epsabs=1e-14 * scale, epsrel=1e-11,
                                   limit=500)[0] for u, v in pieces)
        return total / scale if scale > 0 else 0.0

    lo = p_lo + 1e-6 * span if p_lo > 0 else p_hi * 1e-9
    hi = p_hi - 1e-6 * span
    f_lo, f_hi = area(lo), area(hi)
    if (f_lo > 0) == (f_hi > 0):
        raise ValueError("no coexistence solution with a positive pressure at this state")
    p0 = optimize.brentq(area, lo, hi, xtol=1e-20, rtol=1e-15, maxiter=500)
    rv, rl = _outer_roots(p0, a, b, R, T, s1, s2)
    return rl, rv, p0


def maxwell(a, b, R, T):
    """Eq. 22: coexistence (rho_l, rho_v, p0) by the Maxwell equal-area rule."""
    return _coexistence(lambda r: 1.0 / (r * r), a, b, R, T)


def epsilon_from_sigma(sigma, G=-1.0, alpha=0.0, beta=3.0):
    """Eq. 29 (nearest-neighbour interactions: alpha = 0, beta = 3)."""
    return -2.0 * (alpha + 24.0 * G * sigma) / beta


def mechanical_stability(a, b, R, T, G=-1.0, eps=0.0):
    """Eq. 21: coexistence (rho_l, rho_v, p0) selected by mechanical stability.

    The bracket of Eq. 21 equals p0 - p_eos because of Eq. 24; the weight is
    psi' / psi^(1 + eps).
    """
    w = lambda r: dpsi_drho(r, a, b, R, T, G) / psi(r, a, b, R, T, G) ** (1.0 + eps)  # noqa
    return _coexistence(w, a, b, R, T)


def lamb_period(gamma, rho_l, R0, n=2):
    """Eq. 32: T_a = 2 pi [n (n^2 - 1) gamma / (rho_l R0^3)]^(-1/2)."""
    return 2.0 * math.pi / math.sqrt(n * (n * n - 1) * gamma / (rho_l * R0 ** 3))
