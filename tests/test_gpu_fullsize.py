"""Parity at full workload sizes, in the launch configuration bench.py times.

The whole field is too large for the oracle to advance, but one step of one node depends
only on the populations within two nodes of it.  So: take the GPU state, let the GPU do one
step, and let the oracle compute the same step on small patches cut from that state
(periodic 5-column strips, or 5x5 squares), comparing the nodes whose dependency cone lies
inside the patch.  Sampled nodes include the domain edges, CTA strip boundaries and chunk
boundaries.
"""
import numpy as np
import pytest

import oracle
from oracle import thermo
from paper_1211_6932_gb300 import workloads as wl
from tests import pairs
from tests.textbook import T_W

pytestmark = pytest.mark.gpu


def close32(got, ref, tol=2e-6):
    rho = ref.sum(axis=0)
    scale = T_W.reshape((9,) + (1,) * (ref.ndim - 1)) * rho[None] + np.abs(ref)
    err = np.abs(got - ref) / scale
    return float(err.max())


def patch_check(p, f0, f1, centres, half=2):
    """Oracle step on (2 half + 1)^2 periodic patches of f0 around `centres`; compare the
    centre node with f1."""
    ny, nx = f0.shape[1:]
    n = 2 * half + 1
    pp = oracle.Params(**{**p.__dict__, "nx": n, "ny": n, "walls": False})
    worst = 0.0
    for (y, x) in centres:
        ys = np.arange(y - half, y + half + 1) % ny
        xs = np.arange(x - half, x + half + 1) % nx
        patch = f0[:, ys][:, :, xs]
        out = oracle.run(pp, patch, 1)
        worst = max(worst, close32(f1[:, y, x][:, None], out[:, half, half][:, None]))
    return worst


def column_check(p, f0, f1, columns):
    """Oracle step on full-height 5-column periodic strips (walls kept); compare the centre
    column."""
    ny, nx = f0.shape[1:]
    pp = oracle.Params(**{**p.__dict__, "nx": 5})
    worst = 0.0
    for x in columns:
        xs = np.arange(x - 2, x + 3) % nx
        out = oracle.run(pp, f0[:, :, xs], 1)
        worst = max(worst, close32(f1[:, :, x], out[:, :, 2]))
    return worst


def sample_nodes(nx, ny, strip, rows, rng, n_random=200):
    pts = set()
    for y in (0, 1, ny - 2, ny - 1, ny // 2):
        for x in (0, 1, nx - 2, nx - 1, nx // 2):
            pts.add((y, x))
    for k in range(1, min(nx // strip, 12) + 1):  # CTA strip boundaries
        for dx in (-1, 0):
            pts.add((int(rng.integers(ny)), (k * strip + dx) % nx))
    for k in range(1, min(ny // rows, 12) + 1):  # chunk boundaries
        for dy in (-1, 0):
            pts.add(((k * rows + dy) % ny, int(rng.integers(nx))))
    for _ in range(n_random):
        pts.add((int(rng.integers(ny)), int(rng.integers(nx))))
    return sorted(pts)


def test_bench_workload_4096_sampled_parity():
    """The 4096^2 field of bench.py (64 droplets, linear viscosity), default tiling."""
    import bench
    a, tr = bench.A, bench.TR
    T = tr * wl.t_crit(a)
    rl, rv, _ = thermo.maxwell(a, 4.0, 1.0, T)
    rho = bench.field(rl, rv)
    c = dict(nx=4096, ny=4096, a=a, T=T, sigma=bench.SIGMA, s=bench.RATES, visc="linear",
             nu_l=bench.NU_L, nu_v=bench.NU_V, walls=False, G=-1.0)
    with pairs.gpu_lattice(c, "fp32") as L:
        L.init_fields(rho)
        L.step(20)
        f0 = L.get_populations()
        L.step(1)
        f1 = L.get_populations()
        nt, vec, rows = L.tiling
    p = pairs.oracle_params(c)
    strip = nt * vec - 4
    pts = sample_nodes(4096, 4096, strip, rows, np.random.default_rng(11))
    assert patch_check(p, f0, f1, pts) <= 2e-6


def test_ellipse_1024_sampled_parity():
    """The 1024^2 oscillating ellipse (semi-axes 240 x 160, +-1e-4 noise, linear tau)."""
    a, tr = 0.25, 0.6
    T = tr * wl.t_crit(a)
    rl, rv, _ = thermo.maxwell(a, 4.0, 1.0, T)
    rho = wl.ellipse(1024, 1024, rl, rv, 240, 160, 4.0, noise=1e-4, seed=2)
    c = dict(nx=1024, ny=1024, a=a, T=T, sigma=0.114, s=oracle.rates_for(1.0),
             visc="linear", nu_l=0.05, nu_v=0.5, walls=False, G=-1.0)
    with pairs.gpu_lattice(c, "fp32") as L:
        L.init_fields(rho)
        L.step(50)
        f0 = L.get_populations()
        L.step(1)
        f1 = L.get_populations()
        nt, vec, rows = L.tiling
    p = pairs.oracle_params(c)
    pts = sample_nodes(1024, 1024, nt * vec - 4, rows, np.random.default_rng(12))
    assert patch_check(p, f0, f1, pts) <= 2e-6


def test_splash_2048x512_walls_column_parity():
    """The 2048 x 512 splash with bounce-back walls (film 32, D = 160, U = 0.05,
    T = 0.5 T_c, Re = 200, viscosity ratio 15, step viscosity): full-height columns,
    walls included, at strip boundaries, domain edges and random positions."""
    a, tr = 0.25, 0.5
    T = tr * wl.t_crit(a)
    rl, rv, _ = thermo.maxwell(a, 4.0, 1.0, T)
    rho, ux, uy = wl.splash(2048, 512, rl, rv, 4.0, 32, 160, 0.05)
    nu_l = 0.05 * 160 / 200
    s = (1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)
    c = dict(nx=2048, ny=512, a=a, T=T, sigma=0.114, s=s, visc="step", nu_l=nu_l,
             nu_v=15 * nu_l, walls=True, G=-1.0)
    with pairs.gpu_lattice(c, "fp32") as L:
        L.init_fields(rho, ux, uy)
        L.step(30)
        f0 = L.get_populations()
        L.step(1)
        f1 = L.get_populations()
        nt, vec, rows = L.tiling
    p = pairs.oracle_params(c)
    strip = nt * vec - 4
    rng = np.random.default_rng(13)
    cols = sorted({0, 1, 2047, 2046, 1024} | {k * strip + d for k in range(1, 6) for d in (-1, 0)}
                  | {int(v) for v in rng.integers(0, 2048, 10)})
    assert column_check(p, f0, f1, cols) <= 2e-6


def test_slab_beyond_2_31_elements():
    """Maximum-size indexing: a batch whose population slab holds more than 2^31 elements
    (a 17000^2 instance, 2.6e9 elements per slab, 21 GB for both), followed by a small
    droplet that therefore starts beyond element 2^31.  The small instance matches the
    oracle step for step; the large uniform vapour stays at rest, finite, with its mass
    conserved; no write leaves its buffer."""
    from paper_1211_6932_gb300 import Batch, Eos, Instance
    big = pairs.case(17000, 17000, tr=0.7, sigma=0.114)
    small = pairs.case(64, 48, tr=0.7, sigma=0.114)
    rl, rv = pairs.maxwell(small)
    insts = [Instance(nx=c["nx"], ny=c["ny"], eos=Eos(a=c["a"], T=c["T"]), G=c["G"],
                      sigma=c["sigma"], s=c["s"], rho_l=rl, rho_v=rv) for c in (big, small)]
    b = Batch(insts, precision="fp32")
    try:
        b.init_fields(0, np.full((17000, 17000), rv, dtype=np.float32))
        b.init_fields(1, wl.droplet(64, 48, rl, rv, 12.0, 4.0))
        f0 = b.get_populations(1)
        m0 = b.diagnostics()[0]["mass"]
        b.step(3)
        d = b.diagnostics()
        got = b.get_populations(1)
        b.check_guards()
    finally:
        b.close()
    ref = oracle.run(pairs.oracle_params(small), f0, 3)
    assert close32(got, ref, tol=6e-6) <= 6e-6
    assert d[0]["nonfinite"] == 0 and d[0]["max_u"] < 1e-7
    assert abs(d[0]["mass"] / m0 - 1) < 1e-6
