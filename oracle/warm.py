"""FP64 CPU oracle of the warm-start definitions (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.  It shares no code with the CUDA library.

The paper has no warm start.  Each function writes out one definition of the warm-start
quantities, for fields given as (ny, nx) arrays:

  profile_at        the mean-over-x profile at a real row position, linear between rows.
  measure_film      bulk densities at the film and vapour centres, the integral width
                    4 * integral of g (1 - g) per interface, g the normalised profile (the W
                    of Eq. 31 for a tanh profile), and the shift of the centroid of
                    g (1 - g) across the upper interface from the equimolar (Gibbs) surface.
  measure_droplet   centre and far-point densities, equimolar radius from the mass, and
                    the Laplace coefficient (p(rho_in) - p(rho_out)) R with p of Eq. 30.
  encode / decode   the network targets relative to the Maxwell densities (Eq. 22).
  vapour_law        intercept and relative slope of the far vapour density against 1/R
                    through two droplets.
  curved_densities  the vapour density around droplets of mean curvature kappa,
                    rho_v (1 + curvature kappa), and the liquid at that vapour's pressure
                    to first order.
  droplet_field     the initial density: the largest over droplets of the tanh profile of
                    Eq. 31 about each droplet's half-density circle.
"""
import math

import numpy as np

from . import thermo


def profile_at(prof, y):
    n = len(prof)
    f = math.floor(y)
    w = y - f
    return (1 - w) * prof[int(f) % n] + w * prof[(int(f) + 1) % n]


def measure_film(rho):
    """dict(rho_l, rho_v, width, shift) of an x-uniform film centred on y = (ny-1)/2."""
    rho = np.asarray(rho, dtype=np.float64)
    ny = rho.shape[0]
    prof = rho.mean(axis=1)
    c = (ny - 1) / 2.0
    rl = profile_at(prof, c)
    rv = profile_at(prof, ny - 0.5)
    d = rl - rv
    g = (prof - rv) / d
    L = float(np.sum(g))                  # liquid excess of both interfaces, in rows
    width = 4.0 * float(np.sum(g * (1.0 - g))) / 2.0
    yg = c + L / 2.0
    ys = math.floor(c) + np.arange(1, ny // 2 + 1)  # the upper interface, unwrapped rows
    gu = g[ys % ny]
    yc = float(np.sum(ys * gu * (1 - gu)) / np.sum(gu * (1 - gu)))
    return {"rho_l": rl, "rho_v": rv, "width": width, "shift": yc - yg}


def measure_droplet(rho, a, b, R, T):
    """(rho_in, rho_out, radius, laplace) of a droplet centred on ((nx-1)/2, (ny-1)/2)."""
    rho = np.asarray(rho, dtype=np.float64)
    ny, nx = rho.shape

    def mean_at(px, py):
        """Mean of the four corners of the unit square around (px, py) (a node at
        integer coordinates is its own corners)."""
        xw = [math.floor(px) % nx, math.ceil(px) % nx]
        yw = [math.floor(py) % ny, math.ceil(py) % ny]
        return float(np.mean([rho[y, x] for y in yw for x in xw]))

    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    ri = mean_at(cx, cy)
    ro = mean_at(cx + nx / 2.0, cy + ny / 2.0)
    M = float(rho.sum())
    Rg = math.sqrt((M - nx * ny * ro) / (math.pi * (ri - ro)))
    lap = (thermo.p_eos(ri, a, b, R, T) - thermo.p_eos(ro, a, b, R, T)) * Rg
    return ri, ro, Rg, lap


def encode(p, a, b, R, T):
    ml, mv, _ = thermo.maxwell(a, b, R, T)
    return np.array([p["rho_l"] / ml - 1.0, math.log(p["rho_v"] / mv), p["width"],
                     p["shift"], math.log(p["curvature"])])


def decode(y, a, b, R, T):
    ml, mv, _ = thermo.maxwell(a, b, R, T)
    return {"rho_l": ml * (1.0 + y[0]), "rho_v": mv * math.exp(y[1]), "width": y[2],
            "shift": y[3], "curvature": math.exp(y[4])}


def vapour_law(r1, ro1, r2, ro2):
    """Solve ro_i = rho_v + (rho_v k) / r_i for (rho_v, k)."""
    M = np.array([[1.0, 1.0 / r1], [1.0, 1.0 / r2]])
    rv, s = np.linalg.solve(M, np.array([ro1, ro2]))
    return float(rv), float(s / rv)


def curved_densities(p, kappa, a, b, R, T):
    """(rho_in, rho_out) around droplets of mean curvature kappa."""
    ro = p["rho_v"] * (1.0 + p["curvature"] * kappa)
    dp = thermo.p_eos(ro, a, b, R, T) - thermo.p_eos(p["rho_v"], a, b, R, T)
    return p["rho_l"] + dp / thermo.dp_drho(p["rho_l"], a, b, R, T), ro


def droplet_field(nx, ny, drops, rho_in, rho_v, width, shift=0.0):
    """max over droplets k of the tanh profile between rho_in[k] and rho_v (the vapour
    density everywhere away from droplets) about the
    circle of radius drops[k][2] + shift centred on (drops[k][0], drops[k][1]); periodic
    distances; every droplet evaluated at every node."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    out = np.full((ny, nx), rho_v, dtype=np.float64)
    for (cx, cy, r), ri in zip(drops, rho_in):
        dx = np.abs(x - cx)
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(y - cy)
        dy = np.minimum(dy, ny - dy)
        s = np.hypot(dx, dy) - (r + shift)
        prof = 0.5 * (ri + rho_v) - 0.5 * (ri - rho_v) * np.tanh(2.0 * s / width)
        out = np.maximum(out, prof)
    return out
