"""CUDA step vs the FP64 oracle, element by element, through the C ABI.

Tolerances (written here, derived in the design notes):
  FP64 mode   per step max|df| / max|f| <= 1e-12 (spec bound); in practice ~1e-16.
  FP32 mode   per step, from the same state: |df_q| <= 2e-6 * (t_q rho + |f_q|) -- a few
              hundred ulps of float for ~150 operations per node on O(rho) quantities;
              over runs: max relative density error <= 1e-4 and coexistence densities
              within 1e-3 (spec bounds).
"""
import os

import numpy as np
import pytest

import oracle
from tests import pairs
from tests.textbook import T_W

pytestmark = pytest.mark.gpu

GRIDS = [(128, 128), (130, 67), (5, 3), (3, 40), (257, 129), (1, 7)]


def fp32_close(got, ref, rho, tol=2e-6):
    scale = T_W[:, None, None] * rho[None] + np.abs(ref)
    return float(np.max(np.abs(got - ref) / scale)) <= tol, float(np.max(np.abs(got - ref) / scale))


@pytest.mark.parametrize("nx,ny", GRIDS)
@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("nt,vec", [(64, 1), (128, 1)])
def test_fp64_per_step_parity(nx, ny, walls, nt, vec):
    c = pairs.case(nx, ny, tr=0.7, sigma=0.114, walls=walls,
                   s=(1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25))
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, vel=0.01)
    with pairs.gpu_lattice(c, "fp64", tile_threads=nt, tile_vec=vec, tile_rows=16) as L:
        for k in range(4):
            L.set_populations(f)
            L.step(1)
            got = L.get_populations()
            ref = oracle.run(p, f, 1)
            assert pairs.rel_err(got, ref) <= 1e-12, (k, pairs.rel_err(got, ref))
            f = ref


@pytest.mark.parametrize("visc", ["const", "step", "linear"])
@pytest.mark.parametrize("sigma", [0.0, 0.11])
def test_fp64_viscosity_modes_and_sigma(visc, sigma):
    # T/Tc = 0.85: the original scheme (sigma = 0) is stable only above ~0.8 (Sec. IV A)
    c = pairs.case(96, 80, a=0.5, tr=0.85, sigma=sigma, visc=visc, nu_l=0.05, nu_v=0.2)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, vel=0.005, seed=3)
    with pairs.gpu_lattice(c, "fp64") as L:
        L.set_populations(f)
        L.step(1)
        assert pairs.rel_err(L.get_populations(), oracle.run(p, f, 1)) <= 1e-12
        # and a 60-step trajectory, graph replay included, stays within 60 x the bound
        L.set_populations(f)
        L.step(60)
        assert pairs.rel_err(L.get_populations(), oracle.run(p, f, 60)) <= 60e-12


@pytest.mark.parametrize("nt,vec", [(64, 1), (128, 1), (256, 1), (32, 2), (64, 2), (96, 2),
                                    (128, 2)])
@pytest.mark.parametrize("walls", [False, True])
def test_fp32_per_step_parity(nt, vec, walls):
    c = pairs.case(131, 70, tr=0.6, sigma=0.114, walls=walls, visc="linear", nu_l=0.05,
                   nu_v=0.5)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, vel=0.01, seed=1)
    with pairs.gpu_lattice(c, "fp32", tile_threads=nt, tile_vec=vec, tile_rows=24) as L:
        for k in range(3):
            L.set_populations(f)
            f_in = L.get_populations()  # the float-rounded state the GPU starts from
            L.step(1)
            got = L.get_populations()
            ref = oracle.run(p, f_in, 1)
            ok, err = fp32_close(got, ref, oracle.fields(p, f_in)["rho"])
            assert ok, (k, err)
            f = ref


@pytest.mark.parametrize("nx,ny", [(1, 7), (5, 3), (3, 40), (4, 9), (254, 5), (253, 33)])
@pytest.mark.parametrize("walls", [False, True])
def test_fp32_pair_kernel_degenerate_and_ragged_widths(nx, ny, walls):
    """The default FP32 pair kernel on widths where the ghost copies overlap the owned
    columns (nx < 4), odd widths (column-by-column ghosts and tails), even widths one
    strip wide (paired ghosts) and a width one column past a 252-column strip."""
    if walls and ny < 5:
        pytest.skip("wall runs need a few fluid rows")
    c = pairs.case(nx, ny, tr=0.7, sigma=0.114, walls=walls)
    p = pairs.oracle_params(c)
    rl, rv = pairs.maxwell(c)
    rng = np.random.default_rng(nx * 100 + ny)
    rho = rv + (rl - rv) * rng.uniform(0.0, 1.0, (ny, nx))
    f = oracle.equilibrium(rho, 0.01 * rng.uniform(-1, 1, rho.shape),
                           0.01 * rng.uniform(-1, 1, rho.shape))
    with pairs.gpu_lattice(c, "fp32") as L:
        L.set_populations(f)
        for k in range(2):
            f_in = L.get_populations()
            L.step(1)
            got = L.get_populations()
            ref = oracle.run(p, f_in, 1)
            ok, err = fp32_close(got, ref, oracle.fields(p, f_in)["rho"])
            assert ok, (k, err)
        L.check_guards()


def test_fp32_psi_fp64_option_matches():
    c = pairs.case(64, 64, tr=0.6, sigma=0.114)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, vel=0.01)
    with pairs.gpu_lattice(c, "fp32", psi_fp64=True) as L:
        L.set_populations(f)
        f_in = L.get_populations()
        L.step(1)
        ok, err = fp32_close(L.get_populations(), oracle.run(p, f_in, 1),
                             oracle.fields(p, f_in)["rho"])
        assert ok, err


def test_fp64_droplet_128_full_run():
    """The 128^2 stationary droplet in full (a = 0.25, T = 0.7 T_c, sigma = 0.114, r0 = 30,
    W = 4, tau = 1) for 5000 steps in FP64 against the oracle: the per-step bound of
    1e-12 leaves the whole run within 1e-10 relative (measured far below)."""
    c = pairs.case(128, 128, a=0.25, tr=0.7, sigma=0.114, s=pairs.RATES_TAU1)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, r0=30, W=4.0)
    ref = oracle.run(p, f, 5000)
    with pairs.gpu_lattice(c, "fp64") as L:
        L.set_populations(f)
        L.step(5000)
        got = L.get_populations()
    assert pairs.rel_err(got, ref) <= 1e-10


def test_fp32_droplet_run_density_and_coexistence():
    """128^2 stationary droplet (a = 0.25, T = 0.7 T_c, sigma = 0.114, tau = 1): after
    3000 steps the FP32 density is within 1e-4 (max relative) of the FP64 oracle and the
    liquid/vapour densities within 1e-3."""
    c = pairs.case(128, 128, a=0.25, tr=0.7, sigma=0.114, s=pairs.RATES_TAU1)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, r0=30, W=4.0)
    steps = 3000
    ref = oracle.fields(p, oracle.run(p, f, steps))["rho"]
    with pairs.gpu_lattice(c, "fp32") as L:
        L.set_populations(f)
        L.step(steps)
        rho = L.moments()["rho"]
    assert float(np.max(np.abs(rho - ref) / ref)) <= 1e-4
    for (y, x) in ((64, 64), (0, 0)):
        assert abs(rho[y, x] - ref[y, x]) / ref[y, x] <= 1e-3


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_moments_match_oracle_fields(prec, tol):
    c = pairs.case(70, 45, tr=0.6, sigma=0.114, walls=True)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, vel=0.02)
    with pairs.gpu_lattice(c, prec) as L:
        L.set_populations(f)
        f_in = L.get_populations()
        m = L.moments()
    o = oracle.fields(p, f_in)
    assert np.max(np.abs(m["rho"] - o["rho"]) / o["rho"]) <= tol
    umax = max(np.max(np.abs(o["ux"])), np.max(np.abs(o["uy"])))
    assert np.max(np.abs(m["ux"] - o["ux"])) <= 50 * tol * umax + tol * 1e-3
    assert np.max(np.abs(m["uy"] - o["uy"])) <= 50 * tol * umax + tol * 1e-3


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_diagnostics_match_oracle(prec):
    c = pairs.case(100, 60, tr=0.7, sigma=0.114)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, vel=0.02)
    with pairs.gpu_lattice(c, prec) as L:
        L.set_populations(f)
        d0 = L.diagnostics()
        assert d0["dinf"] == -1.0 and d0["step"] == 0 and d0["nonfinite"] == 0
        L.step(10)
        f_in = L.get_populations()
        d1 = L.diagnostics()
    o = oracle.fields(p, f_in)
    o0 = oracle.fields(p, f)
    rtol = 1e-12 if prec == "fp64" else 1e-6
    assert abs(d1["mass"] - o["rho"].sum()) <= rtol * o["rho"].sum()
    mx = (o["rho"] * o["ux"]).sum()
    my = (o["rho"] * o["uy"]).sum()
    scale = o["rho"].sum() * 1e-2
    assert abs(d1["mom_x"] - mx) <= rtol * 10 * scale and abs(d1["mom_y"] - my) <= rtol * 10 * scale
    umax = np.sqrt(o["ux"] ** 2 + o["uy"] ** 2).max()
    assert abs(d1["max_u"] - umax) <= (1e-6 if prec == "fp32" else 1e-7) * max(umax, 1e-3)
    assert abs(d1["dinf"] - np.max(np.abs(o["rho"] - o0["rho"]))) <= 1e-6 * o["rho"].max()
    assert d1["step"] == 10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_psi_evaluation_accuracy(prec):
    """psi as the kernel computes it vs the oracle's FP64 psi at the same densities
    (the densities are float-representable, so only the evaluation differs)."""
    c = pairs.case(8, 8, a=0.25, tr=0.5)
    rho = np.concatenate([np.geomspace(1e-5, 0.05, 300), np.linspace(0.05, 0.6, 300)])
    rho = rho.astype(np.float32).astype(np.float64)
    ref = np.array([oracle.psi(r, c["a"], 4.0, 1.0, c["T"], -1.0) for r in rho])
    with pairs.gpu_lattice(c, prec) as L:
        got = L.eval_psi(rho)
    rel = np.abs(got - ref) / ref
    assert rel.max() <= (1e-15 if prec == "fp64" else 4e-7), rel.max()


def test_tiling_and_graph_do_not_change_results():
    """Rows per CTA and graph replay only move work around: for one kernel instantiation
    (threads per CTA) the FP32 results are bitwise equal.  Different instantiations are
    compiled separately and may contract multiply-adds differently, so across them the
    results agree to float rounding: a few 1e-7 per step, 1e-5 of the local scale after
    70 steps."""
    c = pairs.case(203, 77, tr=0.65, sigma=0.114, visc="step", nu_l=0.04, nu_v=0.3)
    f = pairs.droplet_state(c, vel=0.01)
    outs = {}
    cfgs = ((64, 2, 0), (64, 2, 5), (64, 2, 77), (64, 2, 1), (128, 2, 9), (128, 2, 16),
            (32, 2, 11), (96, 2, 24), (96, 2, 3), (128, 1, 0), (64, 1, 33), (256, 1, 7))
    for nt, vec, rows in cfgs:
        with pairs.gpu_lattice(c, "fp32", tile_threads=nt, tile_vec=vec, tile_rows=rows) as L:
            L.set_populations(f)
            L.step(70)  # one 64-step graph replay + 6 single launches
            outs.setdefault((nt, vec), []).append(L.get_populations())
    for key, lst in outs.items():
        for o in lst[1:]:
            assert np.array_equal(o, lst[0]), key
    ref = outs[(64, 2)][0]
    scale = T_W[:, None, None] * ref.sum(axis=0)[None] + np.abs(ref)
    for key, lst in outs.items():
        assert np.max(np.abs(lst[0] - ref) / scale) <= 1e-5, key
    with pairs.gpu_lattice(c, "fp32", tile_threads=64, tile_vec=2) as L:
        L.set_populations(f)
        for _ in range(70):
            L.step(1)
        assert np.array_equal(L.get_populations(), ref)


def test_save_load_resume_is_bitwise(tmp_path):
    c = pairs.case(64, 48, tr=0.7, sigma=0.114)
    f = pairs.droplet_state(c, vel=0.01)
    path = os.path.join(tmp_path, "state.lbm")
    with pairs.gpu_lattice(c, "fp32") as L:
        L.set_populations(f)
        L.step(30)
        L.save(path)
        L.step(40)
        straight = L.get_populations()
    with pairs.gpu_lattice(c, "fp32") as L2:
        L2.load(path)
        assert L2.step_count == 30
        L2.step(40)
        assert np.array_equal(L2.get_populations(), straight)
    with open(path, "r+b") as fh:  # a flipped byte is caught by the checksum
        fh.seek(200)
        b = fh.read(1)
        fh.seek(200)
        fh.write(bytes([b[0] ^ 0xFF]))
    from paper_1211_6932_gb300 import LbmError
    with pairs.gpu_lattice(c, "fp32") as L3:
        with pytest.raises(LbmError) as ei:
            L3.load(path)
        assert ei.value.code == -7


def test_save_load_across_full_width_and_strip_tilings(tmp_path):
    """A state saved after full-width sweeps (nx = 100 <= 2 x 128: ghost columns not kept)
    and loaded into a handle that sweeps the same lattice in 32-thread strips (which read
    the ghost columns) continues like the original: against the oracle, step by step."""
    c = pairs.case(100, 40, tr=0.65, sigma=0.114)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, vel=0.01, seed=5)
    path = os.path.join(tmp_path, "state.lbm")
    with pairs.gpu_lattice(c, "fp32") as L:  # default tiling: one full-width strip
        L.set_populations(f)
        L.step(30)
        L.save(path)
    with pairs.gpu_lattice(c, "fp32", tile_threads=32, tile_vec=2) as L2:
        L2.load(path)
        for k in range(2):
            f_in = L2.get_populations()
            L2.step(1)
            ok, err = fp32_close(L2.get_populations(), oracle.run(p, f_in, 1),
                                 oracle.fields(p, f_in)["rho"])
            assert ok, (k, err)


def test_nonfinite_state_is_reported():
    """A NaN placed in the input populations (on the host) is reported by lbm_sync."""
    from paper_1211_6932_gb300 import LbmError
    c = pairs.case(32, 32, tr=0.7, sigma=0.114)
    f = pairs.droplet_state(c)
    f[:, 5, 7] = np.nan
    with pairs.gpu_lattice(c, "fp32") as L:
        L.set_populations(f)
        L.step(2)
        with pytest.raises(LbmError) as ei:
            L.sync()
        assert ei.value.code == -4
        assert L.diagnostics()["nonfinite"] > 0


def test_init_fields_validates_and_matches_equilibrium():
    from paper_1211_6932_gb300 import LbmError
    c = pairs.case(40, 30, tr=0.7, sigma=0.114)
    rl, rv = pairs.maxwell(c)
    from paper_1211_6932_gb300 import workloads as wl
    rho = wl.droplet(40, 30, rl, rv, 9.0, 4.0)
    ux = np.full_like(rho, 0.01)
    uy = np.full_like(rho, -0.02)
    with pairs.gpu_lattice(c, "fp64") as L:
        L.init_fields(rho, ux, uy)
        assert np.max(np.abs(L.get_populations() - oracle.equilibrium(rho, ux, uy))) < 1e-15
        bad = rho.copy()
        bad[3, 3] = 1.5  # beyond 4/b
        with pytest.raises(LbmError) as ei:
            L.init_fields(bad)
        assert ei.value.code == -1


def test_fp32_deviation_reference_choice():
    """Deviation storage around the vapour density (default) is at least as accurate as
    plain float storage (rho_ref = 0) against the oracle after 500 steps."""
    c = pairs.case(96, 96, a=0.25, tr=0.55, sigma=0.114)
    p = pairs.oracle_params(c)
    f = pairs.droplet_state(c, r0=25)
    ref = oracle.fields(p, oracle.run(p, f, 500))
    errs = []
    for rr in (None, 0.0):
        with pairs.gpu_lattice(c, "fp32", rho_ref=rr) as L:
            L.set_populations(f)
            L.step(500)
            m = L.moments()
        errs.append(float(np.max(np.abs(m["rho"] - ref["rho"]) / ref["rho"])))
    assert errs[0] <= 1e-4 and errs[0] <= 1.5 * errs[1], errs


@pytest.mark.parametrize("nt", [32, 64, 96, 128])
@pytest.mark.parametrize("dx", [-1, 0, 1])
@pytest.mark.parametrize("walls", [False, True])
def test_fp32_full_width_and_strip_boundary(nt, dx, walls):
    """Widths at the switch between a full-width strip (nx <= 2 NT: one CTA across the row,
    x wrapped in shared memory, no ghost columns) and strips (nx = 2 NT + 1), for every
    pair-kernel width, periodic and with walls: two steps against the oracle, a 64-step
    graph replay and a single launch after it, then two more steps against the oracle."""
    nx = 2 * nt + dx
    c = pairs.case(nx, 11, tr=0.65, sigma=0.114, walls=walls, visc="linear", nu_l=0.05,
                   nu_v=0.4)
    p = pairs.oracle_params(c)
    rl, rv = pairs.maxwell(c)
    rng = np.random.default_rng(nx * 7 + int(walls))
    rho = rv + (rl - rv) * rng.uniform(0.0, 1.0, (11, nx))
    f = oracle.equilibrium(rho, 0.01 * rng.uniform(-1, 1, rho.shape),
                           0.01 * rng.uniform(-1, 1, rho.shape))
    with pairs.gpu_lattice(c, "fp32", tile_threads=nt, tile_vec=2, tile_rows=4) as L:
        L.set_populations(f)
        for phase in range(2):
            for k in range(2):
                f_in = L.get_populations()
                L.step(1)
                ok, err = fp32_close(L.get_populations(), oracle.run(p, f_in, 1),
                                     oracle.fields(p, f_in)["rho"])
                assert ok, (phase, k, err)
            if phase == 0:
                L.step(65)  # one graph replay of 64 steps and one single launch
                assert L.diagnostics()["nonfinite"] == 0
        L.check_guards()
