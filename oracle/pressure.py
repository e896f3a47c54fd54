"""FP64 oracle of the discrete pressure tensor (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.  It shares no code with the CUDA library.

  pressure_tensor_from_psi  Eq. 18 written out for given rho and psi fields:
                            P = rho c_s^2 I + (G/2) psi(x) sum_a w(|e_a|^2) psi(x + e_a) e_a e_a,
                            nearest-neighbour weights w(1) = 1/3, w(2) = 1/12 (Eq. 7), with
                            the optional isotropic 2 G^2 sigma |grad psi|^2 of Eq. 26 taken
                            with the force stencil's gradient, grad psi = sum_a w psi e_a.
  pressure_tensor           the same for an oracle state (rho and psi from fields()).
  surface_tension_film      integral of (P_n - P_t) across the interfaces of an x-uniform
                            film, per interface (the mechanical definition).
"""
import numpy as np

from . import fields

# the eight moving D2Q9 velocities and Eq. 7's weights by |e|^2
_E = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
_W = {1: 1.0 / 3.0, 2: 1.0 / 12.0}


def _shifted(a, ex, ey, walls):
    """a(x + ex, y + ey): periodic in x; in y periodic, or clamped to the edge rows."""
    out = np.roll(a, -ex, axis=1)
    if not walls:
        return np.roll(out, -ey, axis=0)
    ny = a.shape[0]
    idx = np.clip(np.arange(ny) + ey, 0, ny - 1)
    return out[idx, :]


def pressure_tensor_from_psi(rho, psi, G, walls=False, sigma=0.0):
    rho = np.asarray(rho, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    sxx = np.zeros_like(rho)
    syy = np.zeros_like(rho)
    sxy = np.zeros_like(rho)
    gx = np.zeros_like(rho)
    gy = np.zeros_like(rho)
    for ex, ey in _E:
        wp = _W[ex * ex + ey * ey] * _shifted(psi, ex, ey, walls)
        sxx += wp * ex * ex
        syy += wp * ey * ey
        sxy += wp * ex * ey
        gx += wp * ex
        gy += wp * ey
    iso = rho / 3.0 + 2.0 * sigma * G * G * (gx * gx + gy * gy)
    half = 0.5 * G * psi
    return iso + half * sxx, iso + half * syy, half * sxy


def pressure_tensor(params, f, include_sigma=False):
    fl = fields(params, f)
    return pressure_tensor_from_psi(fl["rho"], fl["psi"], params.G, params.walls,
                                    params.sigma if include_sigma else 0.0)


def surface_tension_film(pxx, pyy):
    """Per-interface integral of P_n - P_t = P_yy - P_xx over one period of an x-uniform
    film with two interfaces (mean over x, sum over rows, halved)."""
    return 0.5 * float(np.sum(np.mean(np.asarray(pyy) - np.asarray(pxx), axis=1)))
