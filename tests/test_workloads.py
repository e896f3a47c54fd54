"""The seeded input recipes (workloads.py) against what they are stated to lay out: the
tanh profile of Eq. 31, droplets and films of the given size, the benchmark field's
droplet layout (64 non-overlapping droplets, radii in [40, 200], surface gaps of at least
4 W with periodic distances), the batched workload's parameter ranges, and the same
inputs for the same seed.  CPU only; phase densities are given numbers, not computed."""
import math

import numpy as np
import pytest

from paper_1211_6932_gb300 import workloads as wl

RL, RV = 0.4, 0.003  # phase densities of the layouts (any liquid > vapour pair)


def test_tanh_profile_has_its_stated_limits_and_midpoint():
    d = np.array([-1e3, -2.5, 0.0, 2.5, 1e3])
    p = wl.tanh_profile(d, RL, RV, 5.0)
    assert p[0] == pytest.approx(RL) and p[-1] == pytest.approx(RV)
    assert p[2] == pytest.approx(0.5 * (RL + RV))
    # antisymmetric about the midpoint; d = W/2 is tanh(1) of the half jump from it
    assert p[1] - p[2] == pytest.approx(p[2] - p[3])
    assert p[2] - p[3] == pytest.approx(0.5 * (RL - RV) * math.tanh(1.0))


def test_droplet_is_centred_periodic_and_of_the_given_radius():
    nx, ny, r0, W = 96, 80, 20.0, 4.0
    rho = wl.droplet(nx, ny, RL, RV, r0, W)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    inside = np.hypot(x - cx, y - cy) < r0 - 3 * W
    outside = np.hypot(x - cx, y - cy) > r0 + 3 * W
    assert np.all(rho[inside] > RL - 0.01 * (RL - RV))
    assert np.all(rho[outside] < RV + 0.01 * (RL - RV))
    # mirror symmetric about the centre (an even-sized grid centres between nodes)
    assert np.allclose(rho, rho[::-1, :]) and np.allclose(rho, rho[:, ::-1])
    # periodic distance: a droplet centred on the corner wraps onto all four corners
    c = wl.droplet(nx, ny, RL, RV, r0, W, cx=0.0, cy=0.0)
    assert c[0, 0] == pytest.approx(c[0, nx - 1], rel=0.05)
    assert c[0, 0] == pytest.approx(c[ny - 1, 0], rel=0.05)
    # the liquid area is that of a disc of radius r0 (the tanh tails cancel to first order)
    liquid = ((rho - RV) / (RL - RV)).sum()
    assert liquid == pytest.approx(math.pi * r0 ** 2, rel=0.02)


def test_flat_film_is_uniform_in_x_and_of_the_given_thickness():
    nx, ny, W, h = 16, 101, 5.0, 40.0
    rho = wl.flat_film(nx, ny, RL, RV, W, h)
    assert np.all(rho == rho[:, :1])
    col = rho[:, 0]
    yc = (ny - 1) // 2
    assert col[yc] == pytest.approx(RL, rel=1e-6)
    # the interfaces sit at yc +- h/2, where the profile passes the mean density
    assert col[yc + int(h / 2)] == pytest.approx(0.5 * (RL + RV))
    assert col[yc - int(h / 2)] == pytest.approx(0.5 * (RL + RV))
    assert ((col - RV) / (RL - RV)).sum() == pytest.approx(h, rel=1e-3)


def test_bench_field_layout_places_64_separated_droplets():
    """The benchmark field's layout at its full size: 4096^2, 64 droplets, radii in
    [40, 200], seed 5, surface gaps of at least 4 W (W = 4) with periodic distances."""
    W = 4.0
    cs, rs = wl.droplet_layout(4096, 4096, 64, 40.0, 200.0, 5, 4 * W)
    assert cs.shape == (64, 2) and rs.shape == (64,)
    assert np.all((rs >= 40.0) & (rs <= 200.0))
    assert np.all((cs >= 0) & (cs < 4096))
    for i in range(64):
        for j in range(i):
            d = np.abs(cs[i] - cs[j])
            d = np.minimum(d, 4096 - d)
            assert math.hypot(*d) >= rs[i] + rs[j] + 4 * W - 1e-9
    c2, r2 = wl.droplet_layout(4096, 4096, 64, 40.0, 200.0, 5, 4 * W)
    assert np.array_equal(cs, c2) and np.array_equal(rs, r2)
    c3, _ = wl.droplet_layout(4096, 4096, 64, 40.0, 200.0, 6, 4 * W)
    assert not np.array_equal(cs, c3)


def test_multi_droplets_field_holds_its_droplets():
    W = 4.0
    rho, cs, rs = wl.multi_droplets(512, 384, RL, RV, W, 6, 15.0, 40.0, seed=2)
    assert rho.shape == (384, 512)
    assert rho.min() >= RV - 1e-15 and rho.max() <= RL + 1e-15
    for (cx, cy), r in zip(cs, rs):
        assert rho[int(round(cy)) % 384, int(round(cx)) % 512] > RL - 0.01 * (RL - RV)
    liquid = ((rho - RV) / (RL - RV)).sum()
    assert liquid == pytest.approx(math.pi * float(np.sum(rs ** 2)), rel=0.03)


def test_batch_draws_stay_in_the_stated_ranges():
    draws = wl.batch_draws(256, seed=4)
    assert len(draws) == 256
    sides = np.array([[d["nx"], d["ny"]] for d in draws])
    assert sides.min() >= 64 and sides.max() <= 512
    # log-uniform in [64, 512]: the median side is near the geometric mean (181)
    assert 150 <= np.median(sides) <= 215
    for i, d in enumerate(draws):
        assert 0.125 <= d["a"] <= 1.0 and 0.5 <= d["T_over_Tc"] <= 0.9
        assert 0.8 <= d["sigma"] / wl.sigma0(d["a"]) <= 1.2
        assert 1.0 <= d["visc_ratio"] <= 20.0
        assert d["kind"] == ("film" if i % 2 == 0 else "droplet")
    assert draws == wl.batch_draws(256, seed=4)
    assert draws != wl.batch_draws(256, seed=5)


def test_sigma0_takes_the_two_printed_values_and_joins_them():
    assert wl.sigma0(0.125) == 0.114 and wl.sigma0(0.25) == 0.114
    assert wl.sigma0(0.5) == 0.11 and wl.sigma0(1.0) == 0.11
    mid = wl.sigma0(math.sqrt(0.25 * 0.5))  # halfway in log a
    assert mid == pytest.approx(0.112)
    xs = np.linspace(0.2, 0.6, 41)
    ys = [wl.sigma0(a) for a in xs]
    assert all(b <= a for a, b in zip(ys, ys[1:]))  # non-increasing in a
