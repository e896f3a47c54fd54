"""Batches of ragged instances (one launch per step over every instance)."""
import numpy as np
import pytest

import oracle
from paper_1211_6932_gb300 import workloads as wl
from tests import pairs

pytestmark = pytest.mark.gpu

CASES = [
    pairs.case(70, 45, a=0.25, tr=0.7, sigma=0.114),
    pairs.case(130, 67, a=0.5, tr=0.8, sigma=0.11, walls=True, visc="step", nu_l=0.05,
               nu_v=0.3),
    pairs.case(5, 3, a=1.0, tr=0.9, sigma=0.11),
    pairs.case(257, 31, a=0.125, tr=0.6, sigma=0.114, visc="linear", nu_l=0.04, nu_v=0.4),
    pairs.case(64, 200, a=0.75, tr=0.85, sigma=0.1),
]


def instance(c, layout="auto"):
    from paper_1211_6932_gb300 import Eos, Instance
    rl, rv = pairs.maxwell(c)
    return Instance(nx=c["nx"], ny=c["ny"], eos=Eos(a=c["a"], T=c["T"]), G=c["G"],
                    sigma=c["sigma"], s=c["s"], nu_l=c["nu_l"], nu_v=c["nu_v"],
                    visc_mode=c["visc"], bc="walls" if c["walls"] else "periodic",
                    rho_c=0.5218 / 4.0, rho_l=rl, rho_v=rv, layout=layout)


MIRROR = [0, 2, 1, 4, 3, 5, 8, 7, 6]  # D2Q9 velocity with its components exchanged


def exchanged(f):
    """Populations (9, ny, nx) of a lattice with x and y exchanged: (9, nx, ny)."""
    return np.stack([f[MIRROR[a]].T for a in range(9)])


def start_fields(c, seed):
    rl, rv = pairs.maxwell(c)
    rho = wl.droplet(c["nx"], c["ny"], rl, rv, 0.3 * min(c["nx"], c["ny"]), 4.0)
    rng = np.random.default_rng(seed)
    return rho, 0.01 * rng.uniform(-1, 1, rho.shape), 0.01 * rng.uniform(-1, 1, rho.shape)


def test_fp64_batch_matches_oracle_per_instance():
    from paper_1211_6932_gb300 import Batch
    b = Batch([instance(c) for c in CASES], precision="fp64", tile_rows=16)
    starts = []
    for i, c in enumerate(CASES):
        rho, ux, uy = start_fields(c, i)
        b.init_fields(i, rho, ux, uy)
        starts.append(oracle.equilibrium(rho, ux, uy))
    b.step(5)
    for i, c in enumerate(CASES):
        ref = oracle.run(pairs.oracle_params(c), starts[i], 5)
        assert pairs.rel_err(b.get_populations(i), ref) <= 5e-12, i
    b.close()


def test_fp32_batch_equals_single_lattices_bitwise():
    """Same kernel instantiation, so the batch and one-lattice runs are bitwise equal.  The
    64 x 200 instance is stored transposed (64 strip rows of 200 columns instead of 200 of
    64, at the same cost per strip row): it equals the
    200 x 64 lattice started from the transposed fields, with x and y exchanged in its
    populations, moments and momentum."""
    from paper_1211_6932_gb300 import Batch
    b = Batch([instance(c) for c in CASES], precision="fp32")
    assert [b.is_transposed(i) for i in range(len(CASES))] == [False] * 4 + [True]
    fields = [start_fields(c, 10 + i) for i, c in enumerate(CASES)]
    for i, fl in enumerate(fields):
        b.init_fields(i, *fl)
    b.step(70)
    diags = b.diagnostics()
    for i, c in enumerate(CASES):
        t = b.is_transposed(i)
        rho, ux, uy = fields[i]
        with pairs.gpu_lattice(dict(c, nx=c["ny"], ny=c["nx"]) if t else c, "fp32") as L:
            L.init_fields(*((rho.T, uy.T, ux.T) if t else (rho, ux, uy)))
            L.step(70)
            f = L.get_populations()
            assert np.array_equal(b.get_populations(i), exchanged(f) if t else f), i
            d = L.diagnostics()
            assert diags[i]["mass"] == d["mass"] and diags[i]["max_u"] == d["max_u"], i
            assert diags[i]["mom_x"] == d["mom_y" if t else "mom_x"], i
            assert diags[i]["mom_y"] == d["mom_x" if t else "mom_y"], i
            assert diags[i]["step"] == 70
            for dt in (np.float64, np.float32):
                m, ml = b.moments(i, dtype=dt), L.moments(dtype=dt)
                if t:
                    ml = {"rho": ml["rho"].T, "ux": ml["uy"].T, "uy": ml["ux"].T}
                for k in ("rho", "ux", "uy"):
                    assert m[k].dtype == dt and np.array_equal(m[k], ml[k]), (i, k, dt)
    b.close()


def test_explicit_layouts():
    """Instance.layout: "rows" keeps the given orientation, "transposed" exchanges the axes
    (same physics: within FP32 rounding of the as-given run after a few steps, and the
    host sees the given orientation); an instance with walls cannot be transposed."""
    from paper_1211_6932_gb300 import Batch, LbmError
    c = CASES[0]
    b = Batch([instance(c, lay) for lay in ("rows", "transposed", "auto")], precision="fp32")
    assert [b.is_transposed(i) for i in range(3)] == [False, True, False]
    fl = start_fields(c, 50)
    for i in range(3):
        b.init_fields(i, *fl)
    b.step(5)
    f0, f1, f2 = (b.get_populations(i) for i in range(3))
    assert f1.shape == (9, c["ny"], c["nx"])
    assert np.array_equal(f0, f2)
    assert pairs.rel_err(f1, f0) <= 2e-5
    m0, m1 = b.moments(0), b.moments(1)
    for k in ("rho", "ux", "uy"):
        assert np.max(np.abs(m1[k] - m0[k])) <= 2e-5 * np.max(np.abs(m0["rho"])), k
    b.close()
    with pytest.raises(LbmError) as e:
        Batch([instance(CASES[1], "transposed")], precision="fp32")
    assert e.value.code == -1 and "walls" in str(e.value)


def test_per_instance_widths_equal_uniform_tiling_bitwise():
    """Per-instance kernel widths (one launch per width and kind of strip, graph branches)
    give the populations and diagnostics of the uniform tiling bit for bit, through graph
    replays (64 steps) and single launches."""
    from paper_1211_6932_gb300 import Batch
    from paper_1211_6932_gb300.lattice import TILE_PER_INSTANCE
    cs = CASES + [pairs.case(400, 40, a=0.25, tr=0.75, sigma=0.114),
                  pairs.case(220, 36, a=0.5, tr=0.8, sigma=0.11, walls=True)]
    fields = [start_fields(c, 30 + i) for i, c in enumerate(cs)]
    out = []
    for threads in (0, TILE_PER_INSTANCE):
        b = Batch([instance(c) for c in cs], precision="fp32", tile_threads=threads)
        for i, fl in enumerate(fields):
            b.init_fields(i, *fl)
        b.step(70)
        # uniform 128 threads: strips (400, 257) and full-width strips (the rest, nx <= 256);
        # per instance: widths 32 (nx 5, full), 64 (70, full), 96 (130 full, 257 strips)
        # and 128 (220 and the transposed 64 x 200 full, 400 strips)
        assert b.launches_per_step == (2 if threads == 0 else 6)
        # both creation tilings store 64 x 200 transposed (200-column rows) and nothing else
        assert [b.is_transposed(i) for i in range(len(cs))] == [False] * 4 + [True, False, False]
        pops = [b.get_populations(i) for i in range(len(cs))]
        diags = b.diagnostics()
        b.step(3)
        out.append((pops, diags, [b.get_populations(i) for i in range(len(cs))]))
        assert b.tiling[0] == (threads or 128)
        b.close()
    (p0, d0, q0), (p1, d1, q1) = out
    for i in range(len(cs)):
        assert np.array_equal(p0[i], p1[i]), i
        assert np.array_equal(q0[i], q1[i]), i
        for k in ("mass", "mom_x", "mom_y", "max_u", "nonfinite"):
            assert d0[i][k] == d1[i][k], (i, k)


@pytest.mark.parametrize("threads", [0, -1])
def test_run_to_equilibrium_freezes_converged_instances(threads):
    """Flat films converge; a converged instance is no longer stepped (its state and step
    count stay fixed) while the others continue (uniform and per-instance widths: the
    launch groups are rebuilt at each retirement)."""
    from paper_1211_6932_gb300 import Batch
    cs = [pairs.case(3, 64, a=0.5, tr=0.85, sigma=0.11),
          pairs.case(4, 96, a=0.25, tr=0.8, sigma=0.114),
          pairs.case(130, 67, a=0.5, tr=0.8, sigma=0.11)]
    b = Batch([instance(c) for c in cs], precision="fp32", tile_threads=threads)
    for i, c in enumerate(cs):
        rl, rv = pairs.maxwell(c)
        if c["nx"] <= 4:
            rho = wl.flat_film(c["nx"], c["ny"], rl, rv, 4.0, c["ny"] / 2)
        else:
            rho = wl.droplet(c["nx"], c["ny"], rl, rv, 20.0, 4.0)
        b.init_fields(i, rho)
    left, steps = b.run_to_equilibrium(tol=2e-6, check_every=100, max_steps=20000)
    assert left == 0, steps
    assert (steps > 0).all() and (steps % 100 == 0).all()
    frozen = [b.get_populations(i) for i in range(3)]
    b.step(50)  # nothing is active any more
    assert b.launches_per_step == 0
    for i in range(3):
        assert np.array_equal(b.get_populations(i), frozen[i])
    d = b.diagnostics()
    assert [di["step"] for di in d] == list(steps)
    b.close()


def test_batch_rejects_bad_instance():
    from paper_1211_6932_gb300 import Batch, LbmError
    bad = instance(CASES[0])
    bad.s = (1.0,) * 8 + (2.5,)
    with pytest.raises(LbmError) as ei:
        Batch([instance(CASES[1]), bad])
    assert ei.value.code == -1


def test_batch_of_256_workload_draws_runs():
    """The batched-equilibria recipe (256 instances, sides 64..512) builds and steps; every
    instance stays finite and conserves mass over 200 steps."""
    from paper_1211_6932_gb300 import batched
    insts, fields, _ = batched.instances(256, seed=4)
    b = batched.new_batch(insts, fields)
    d0 = b.diagnostics()
    b.step(200)
    d1 = b.diagnostics()
    for i in range(256):
        assert d1[i]["nonfinite"] == 0, i
        assert abs(d1[i]["mass"] - d0[i]["mass"]) <= 1e-5 * d0[i]["mass"], i
    b.close()


def test_unstable_draws_are_retired_and_unstable_in_fp64_too():
    """A 10^4-step screen of the 256-instance recipe retires the instances that turn
    non-finite (lbm_batch_retire_nonfinite): they lie in the low-temperature corner
    (T/Tc < 0.6), turn non-finite in the FP64 mode as well (so the cause is the method at
    those parameters, not FP32), and the batch of the others stays finite."""
    from paper_1211_6932_gb300 import batched
    insts, fields, draws = batched.instances(256, seed=4)
    bad = batched.screen(insts, fields, steps=10000)
    assert 0 < len(bad) <= 16
    assert all(draws[i]["T_over_Tc"] < 0.6 for i in bad), [draws[i] for i in bad]
    b = batched.new_batch([insts[i] for i in bad], [fields[i] for i in bad], "fp64")
    b.step(10000)
    assert all(d["nonfinite"] > 0 for d in b.diagnostics())
    b.close()
    keep = [i for i in range(256) if i not in bad][::8]
    b = batched.new_batch([insts[i] for i in keep], [fields[i] for i in keep])
    b.step(10000)
    assert all(d["nonfinite"] == 0 for d in b.diagnostics())
    assert b.retire_nonfinite() == []
    b.close()


def test_retire_stops_stepping_an_instance():
    """lbm_batch_retire freezes one instance (its state and step count stay) while the
    others go on; init_fields makes it active again."""
    from paper_1211_6932_gb300 import Batch
    b = Batch([instance(c) for c in CASES[:3]], precision="fp32")
    fields = [start_fields(c, 20 + i) for i, c in enumerate(CASES[:3])]
    for i, fl in enumerate(fields):
        b.init_fields(i, *fl)
    b.step(5)
    b.retire(1)
    assert not b.is_active(1) and b.is_active(0) and b.active == 2
    f1 = b.get_populations(1)
    b.step(7)
    d = b.diagnostics()
    assert [x["step"] for x in d] == [12, 5, 12]
    assert np.array_equal(b.get_populations(1), f1)
    b.init_fields(1, *fields[1])
    assert b.is_active(1) and b.active == 3
    b.close()


def test_fp64_reaches_the_stated_equilibrium_tolerance():
    """The stated criterion |d rho|_inf < 1e-9 per 100 steps is reached in the FP64 mode by
    the 8 smallest stable instances of the recipe; the FP32 path's floor is higher (its
    reading is 1e-6), and its equilibria agree with the FP64 ones: bulk phase densities
    within 1e-4."""
    from paper_1211_6932_gb300 import batched
    insts, fields, draws = batched.instances(256, seed=4)
    order = sorted(range(256), key=lambda i: insts[i].nx * insts[i].ny)
    sub = [i for i in order if draws[i]["T_over_Tc"] >= 0.6][:8]
    si, sf = [insts[i] for i in sub], [fields[i] for i in sub]
    e64 = batched.run_to_equilibrium(si, sf, tol=1e-9, max_steps=100000, precision="fp64",
                                     keep_fields=True)
    assert not e64.unstable and not e64.unconverged, e64.steps
    e32 = batched.run_to_equilibrium(si, sf, tol=1e-6, max_steps=100000, keep_fields=True)
    assert not e32.unstable and not e32.unconverged, e32.steps
    for k, i in enumerate(sub):
        rl, rv = insts[i].rho_l, insts[i].rho_v
        l64, v64 = batched.phase_densities(e64.rho[k], rl, rv)
        l32, v32 = batched.phase_densities(e32.rho[k], rl, rv)
        assert abs(l32 / l64 - 1) <= 1e-4 and abs(v32 / v64 - 1) <= 1e-4, (i, l32, l64, v32, v64)


def test_autotune_keeps_state_and_uses_cache(tmp_path):
    """The autotuner times tilings on a saved copy: populations and step count are
    unchanged, the choice is valid, and a second call is served from the cache."""
    import os
    c = pairs.case(300, 200, tr=0.7, sigma=0.114)
    f = pairs.droplet_state(c, vel=0.01)
    cache = os.path.join(tmp_path, "tiles.txt")
    with pairs.gpu_lattice(c, "fp32") as L:
        L.set_populations(f)
        L.step(3)
        before = L.get_populations()
        t, v, r, ms = L.autotune(steps=6, cache=cache)
        assert (t, v) in ((64, 1), (128, 1), (256, 1), (32, 2), (64, 2), (96, 2), (128, 2),
                          (-1, 2))
        assert r in (1, 2, 4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 64)
        assert ms > 0 and L.tiling == (t, v, r)
        assert L.step_count == 3
        assert np.array_equal(L.get_populations(), before)
        L.step(2)  # stepping after tuning works with the chosen tiling
    with pairs.gpu_lattice(c, "fp32") as L2:
        L2.set_populations(f)
        t2, v2, r2, ms2 = L2.autotune(steps=6, cache=cache)
        assert (t2, v2, r2) == (t, v, r) and abs(ms2 - ms) < 1e-5
    assert len(open(cache).read().strip().splitlines()) == 1


def test_autotune_chooses_between_persistent_and_per_step_stepping(tmp_path):
    """A tiling that steps persistently is timed that way and with one launch per step; the
    faster is kept and cached (a sixth field, 1 if persistent stepping is allowed), a cache
    hit restores it, an entry recording one launch per step as faster turns persistent
    stepping off for its tiling, and an explicit tiling returns to the default rule."""
    import os
    c = pairs.case(600, 250, tr=0.7, sigma=0.114)
    f = pairs.droplet_state(c, vel=0.01)
    cache = os.path.join(tmp_path, "tiles.txt")
    old = os.environ.get("LBM_PERSISTENT")
    os.environ["LBM_PERSISTENT"] = "2"  # persistent wherever the dependency rule allows
    try:
        with pairs.gpu_lattice(c, "fp32") as L:
            L.set_populations(f)
            t, v, r, ms = L.autotune(steps=6, cache=cache)
            key, *vals = open(cache).read().split()
            assert len(vals) == 5 and vals[4] in ("0", "1")
            if vals[4] == "0":
                assert not L.persistent
            assert L.tiling == (t, v, r)
        out = []
        for allow in ("1", "0"):
            with open(cache, "a") as fh:
                fh.write("%s 128 2 16 0.1 %s\n" % (key, allow))
            with pairs.gpu_lattice(c, "fp32") as L2:
                L2.set_populations(f)
                assert L2.autotune(steps=6, cache=cache)[:3] == (128, 2, 16)
                assert L2.persistent == (allow == "1")
                L2.step(70)
                out.append(L2.get_populations())
                L2.set_tiling(128, 2, 16)
                assert L2.persistent
        assert np.array_equal(out[0], out[1])
    finally:
        if old is None:
            del os.environ["LBM_PERSISTENT"]
        else:
            os.environ["LBM_PERSISTENT"] = old
