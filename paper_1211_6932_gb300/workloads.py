"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method itself: it only lays out initial density
and velocity fields (droplets, films, ellipses) from given phase densities, and draws the
parameters of the batched workload.  Phase densities come from the caller (the library's
Maxwell solver on the product side, the oracle's on the test side).

The interface profile is the tanh form of Eq. 31,
    rho = (rho_l + rho_v)/2 - (rho_l - rho_v)/2 * tanh(2 d / W),
with d the signed distance from the interface (positive on the vapour side).
Node (x, y) sits at coordinates (x, y); the domain centre is ((nx-1)/2, (ny-1)/2).
"""
import math

import numpy as np

TC_COEFF = 0.3773  # T_c = 0.3773 a / (b R), the rounded critical temperature of the workloads


def t_crit(a, b=4.0, R=1.0):
    return TC_COEFF * a / (b * R)


def tanh_profile(d, rho_l, rho_v, W):
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * d / W)


def grid(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx]
    return x.astype(np.float64), y.astype(np.float64)


def droplet(nx, ny, rho_l, rho_v, r0, W, cx=None, cy=None):
    """Circular droplet (liquid inside), periodic distance to the centre."""
    x, y = grid(nx, ny)
    cx = (nx - 1) / 2.0 if cx is None else cx
    cy = (ny - 1) / 2.0 if cy is None else cy
    dx = np.abs(x - cx)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(y - cy)
    dy = np.minimum(dy, ny - dy)
    return tanh_profile(np.hypot(dx, dy) - r0, rho_l, rho_v, W)


def flat_film(nx, ny, rho_l, rho_v, W, thickness, yc=None):
    """Liquid slab of the given thickness centred on row yc (x-uniform)."""
    x, y = grid(nx, ny)
    yc = (ny - 1) / 2.0 if yc is None else yc
    return tanh_profile(np.abs(y - yc) - thickness / 2.0, rho_l, rho_v, W)


def ellipse(nx, ny, rho_l, rho_v, ax, ay, W, noise=0.0, seed=0):
    """Elliptical droplet with semi-axes ax (x) and ay (y) at the centre, plus uniform
    density noise in [-noise, noise] (seeded)."""
    x, y = grid(nx, ny)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    # Distance to the ellipse along the ray from the centre, scaled by the local radius.
    th = np.arctan2(y - cy, x - cx)
    r = np.hypot(x - cx, y - cy)
    r_e = ax * ay / np.sqrt((ay * np.cos(th)) ** 2 + (ax * np.sin(th)) ** 2)
    rho = tanh_profile(r - r_e, rho_l, rho_v, W)
    if noise:
        rng = np.random.default_rng(seed)
        rho = rho + rng.uniform(-noise, noise, size=rho.shape)
    return rho


def splash(nx, ny, rho_l, rho_v, W, film_h, D, U, velocity="fraction", gap=None):
    """Droplet of diameter D moving down at speed U above a liquid film of thickness
    film_h lying on the bottom wall (rows 0..film_h-1).  Returns rho, ux, uy.  The droplet
    velocity is weighted by its liquid fraction (velocity="fraction"), or is U on the nodes
    denser than the mean of the phase densities and zero elsewhere (velocity="sharp").
    The droplet's centre is D/2 + gap above the film, gap = 2W unless given."""
    x, y = grid(nx, ny)
    film = tanh_profile(y - (film_h - 0.5), rho_l, rho_v, W)
    cx = (nx - 1) / 2.0
    cy = film_h + D / 2.0 + (2.0 * W if gap is None else gap)
    drop = tanh_profile(np.hypot(x - cx, y - cy) - D / 2.0, rho_l, rho_v, W)
    rho = np.maximum(film, drop)
    if velocity == "fraction":
        frac = np.clip((drop - rho_v) / (rho_l - rho_v), 0.0, 1.0)
    elif velocity == "sharp":
        frac = (drop > 0.5 * (rho_l + rho_v)).astype(np.float64)
    else:
        raise ValueError("velocity must be 'fraction' or 'sharp'")
    ux = np.zeros_like(rho)
    uy = -U * frac
    return rho, ux, uy


def droplet_layout(nx, ny, n, rmin, rmax, seed, gap, max_tries=200000):
    """n non-overlapping droplets with radii uniform in [rmin, rmax] (rejection sampling,
    periodic distances, surface gap >= gap).  Returns centres (n, 2) and radii (n,)."""
    rng = np.random.default_rng(seed)
    cs, rs = [], []
    tries = 0
    while len(cs) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d droplets" % n)
        r = rng.uniform(rmin, rmax)
        c = (rng.uniform(0, nx), rng.uniform(0, ny))
        ok = True
        for (px, py), pr in zip(cs, rs):
            dx = abs(c[0] - px)
            dx = min(dx, nx - dx)
            dy = abs(c[1] - py)
            dy = min(dy, ny - dy)
            if math.hypot(dx, dy) < r + pr + gap:
                ok = False
                break
        if ok:
            cs.append(c)
            rs.append(r)
    return np.array(cs), np.array(rs)


def multi_droplets(nx, ny, rho_l, rho_v, W, n, rmin, rmax, seed, gap=None, max_tries=200000):
    """n non-overlapping droplets with radii uniform in [rmin, rmax] (rejection sampling,
    periodic distances, surface gap >= gap, default 4 W).  Returns rho, centres, radii."""
    gap = 4.0 * W if gap is None else gap
    cs, rs = droplet_layout(nx, ny, n, rmin, rmax, seed, gap, max_tries)
    rho = np.full((ny, nx), rho_v, dtype=np.float64)
    for (cx, cy), r in zip(cs, rs):
        # Only the bounding box of each droplet (plus its tail) is touched.
        R = int(r + 4 * W) + 2
        xs = (np.arange(int(cx) - R, int(cx) + R + 1)) % nx
        ys = (np.arange(int(cy) - R, int(cy) + R + 1)) % ny
        X, Y = np.meshgrid(xs, ys)
        dx = np.abs(X - cx)
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(Y - cy)
        dy = np.minimum(dy, ny - dy)
        prof = tanh_profile(np.hypot(dx, dy) - r, rho_l, rho_v, W)
        rho[Y, X] = np.maximum(rho[Y, X], prof)
    return rho, cs, rs


def sigma0(a):
    """Improved-forcing sigma by EOS parameter a: 0.114 at a <= 0.25 and 0.11 at a >= 0.5
    (the paper's two values, Sec. IV B), linear in log a between."""
    if a <= 0.25:
        return 0.114
    if a >= 0.5:
        return 0.11
    t = math.log(a / 0.25) / math.log(2.0)
    return 0.114 + t * (0.11 - 0.114)


def batch_draws(n=256, seed=4, lo=64, hi=512):
    """Parameters of the batched-equilibria workload: grid sides log-uniform in [lo, hi]
    (independently), a ~ U[0.125, 1], T/Tc ~ U[0.5, 0.9], sigma = sigma0(a) U[0.8, 1.2],
    viscosity ratio ~ U[1, 20]; even indices are flat films (thickness ny/2), odd ones
    droplets (radius min(nx, ny)/4)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        ny = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        a = rng.uniform(0.125, 1.0)
        tr = rng.uniform(0.5, 0.9)
        sig = sigma0(a) * rng.uniform(0.8, 1.2)
        ratio = rng.uniform(1.0, 20.0)
        out.append({"nx": nx, "ny": ny, "a": a, "T_over_Tc": tr, "sigma": sig,
                    "visc_ratio": ratio, "kind": "film" if i % 2 == 0 else "droplet"})
    return out


def warm_draws(n=256, seed=6, lo=64, hi=512, a=(0.125, 1.0), tr=(0.5, 0.9),
               sig=(0.8, 1.2), ratio=(1.0, 20.0)):
    """Parameter draws of the warm-start training set: per draw one flat film and one
    droplet of the same parameters.  Grid sides log-uniform in [lo, hi] (independently),
    a, T/Tc, sigma / sigma0(a) and the viscosity ratio uniform in the given ranges."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        ny = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        av = rng.uniform(*a)
        out.append({"nx": nx, "ny": ny, "a": av, "T_over_Tc": rng.uniform(*tr),
                    "sigma": sigma0(av) * rng.uniform(*sig), "visc_ratio": rng.uniform(*ratio)})
    return out


def mlp_init(seed, n_in=4, n_hid=64, n_out=5):
    """Initial weights of the warm-start network, packed W1, b1, W2, b2, W3, b3 (each W
    (out, in) row-major): every entry of a layer uniform in [-1/sqrt(fan_in),
    1/sqrt(fan_in)] (seeded).  float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in ((n_in, n_hid), (n_hid, n_hid), (n_hid, n_out)):
        k = 1.0 / math.sqrt(fi)
        parts.append(rng.uniform(-k, k, fo * fi))
        parts.append(rng.uniform(-k, k, fo))
    return np.concatenate(parts).astype(np.float32)
