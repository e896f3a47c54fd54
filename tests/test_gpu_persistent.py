"""Persistent stepping (sweep2_persist_kernel: one launch per run of up to 64 steps and
launch group, CTAs taking (step, chunk row, strip) items from a queue and waiting only on
the chunk rows of the previous step they depend on) gives the populations of one launch
per step and group bit for bit: periodic and wall boundaries, strips and full-width
strips, odd widths, ragged last chunks (down to one row), two-row chunks, graph replays
and shorter runs, batches of one launch group and of strips and full-width strips in one
launch, and the 256-instance batch (per-instance widths keep one launch per step and
group)."""
import os

import numpy as np
import pytest

from tests import pairs

pytestmark = pytest.mark.gpu


def _run(make, persistent, steps=(70, 5)):
    old = os.environ.get("LBM_PERSISTENT")
    # 2: persistent whenever the dependency rule allows, also with fewer items per step
    # than the default rule asks for (these small lattices are the hard cases)
    os.environ["LBM_PERSISTENT"] = "2" if persistent else "0"
    try:
        obj = make()
    finally:
        if old is None:
            del os.environ["LBM_PERSISTENT"]
        else:
            os.environ["LBM_PERSISTENT"] = old
    try:
        mode = obj.persistent
        out = []
        for n in steps:
            obj.step(n)
            out.append(obj.get_populations() if hasattr(obj, "nx") else
                       [obj.get_populations(i) for i in range(len(obj))])
        return mode, out
    finally:
        obj.close()


LATTICES = [
    (pairs.case(600, 250, tr=0.7, sigma=0.114), {}),                      # strips, periodic
    (pairs.case(300, 97, tr=0.6, sigma=0.114, walls=True, visc="step", nu_l=0.05, nu_v=0.3),
     {}),                                                                  # walls, ragged chunk
    (pairs.case(257, 37, tr=0.7, sigma=0.114), {"tile_rows": 12}),        # odd nx, 1-row last chunk
    (pairs.case(200, 64, tr=0.8, sigma=0.11), {"tile_rows": 2}),          # full width, 2-row chunks
    (pairs.case(301, 50, tr=0.7, sigma=0.114), {"tile_threads": 64}),     # 64-thread strips
]


@pytest.mark.parametrize("k", range(len(LATTICES)))
def test_persistent_lattice_equals_per_step_launches(k):
    c, kw = LATTICES[k]
    f0 = pairs.droplet_state(c, vel=0.01)

    def make():
        L = pairs.gpu_lattice(c, "fp32", **kw)
        L.set_populations(f0)
        return L
    mp, a = _run(make, True)
    mq, b = _run(make, False)
    assert mp and not mq
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_default_rule_steps_large_lattices_persistently():
    """Without LBM_PERSISTENT the 4096^2 field steps persistently (its default 32-row chunks
    give 2176 items per step, about three waves) and a 1024^2 lattice does not (fewer
    items than two waves of resident CTAs)."""
    c = pairs.case(4096, 4096, tr=0.7, sigma=0.114)
    with pairs.gpu_lattice(c, "fp32") as L:
        assert L.persistent and L.tiling[2] == 32
    with pairs.gpu_lattice(dict(c, nx=1024, ny=1024), "fp32") as L:
        assert not L.persistent


def test_persistent_batch_equals_per_step_launches():
    """Batches whose instances share one kernel width step persistently: one launch group
    (every instance swept in one full-width 128-thread strip per row), and strips and
    full-width strips together (one launch, each item taking its instance's sweep); with
    per-instance widths they keep one launch per step and group.  All give the per-step
    populations bit for bit."""
    from paper_1211_6932_gb300 import Batch
    from paper_1211_6932_gb300.lattice import TILE_PER_INSTANCE
    from tests.test_gpu_batch import CASES, instance, start_fields
    single = CASES[:1] + CASES[2:3] + [pairs.case(200, 90, tr=0.75, sigma=0.114),
                                      pairs.case(130, 67, tr=0.8, sigma=0.11, walls=True)]
    mixed = CASES + [pairs.case(400, 40, tr=0.75, sigma=0.114)]
    for cs, threads, persistent in ((single, 0, True), (mixed, 0, True),
                                    (mixed, TILE_PER_INSTANCE, False)):
        fields = [start_fields(c, 60 + i) for i, c in enumerate(cs)]

        def make():
            b = Batch([instance(c) for c in cs], precision="fp32", tile_threads=threads)
            for i, fl in enumerate(fields):
                b.init_fields(i, *fl)
            if b.persistent:
                assert b.launches_per_step == 1
            return b
        mp, a = _run(make, True)
        mq, b = _run(make, False)
        assert mp == persistent and not mq
        for x, y in zip(a, b):
            for i in range(len(cs)):
                assert np.array_equal(x[i], y[i]), i


def test_batch_of_256_persistent_equals_per_step_launches():
    """The 256-instance batch of ragged instances (sides 64 to 512; the instances that turn
    non-finite within 10^4 steps screened out, as timed; strips and full-width strips in one
    persistent launch at the default tiling) stepped 640 steps persistently and with one
    launch per step and group ends in the same populations bit for bit."""
    from paper_1211_6932_gb300 import Batch, batched
    insts, fields, _ = batched.instances(256, seed=4)
    bad = batched.screen(insts, fields, steps=10000)
    insts = [x for i, x in enumerate(insts) if i not in bad]
    fields = [x for i, x in enumerate(fields) if i not in bad]

    def make(persistent):
        old = os.environ.get("LBM_PERSISTENT")
        os.environ["LBM_PERSISTENT"] = "1" if persistent else "0"
        try:
            b = Batch(insts, precision="fp32")
        finally:
            if old is None:
                del os.environ["LBM_PERSISTENT"]
            else:
                os.environ["LBM_PERSISTENT"] = old
        assert b.persistent == persistent
        assert b.launches_per_step == (1 if persistent else 2)
        for i, rho in enumerate(fields):
            b.init_fields(i, rho)
        b.step(640)
        return b
    bp = make(True)
    try:
        bq = make(False)
        try:
            for i in range(len(insts)):
                assert np.array_equal(bp.get_populations(i), bq.get_populations(i)), i
        finally:
            bq.close()
    finally:
        bp.close()


def test_long_persistent_run_on_the_field_equals_per_step_launches():
    """Stress test of the cross-step pipeline: the 4096^2 field of 64 droplets (the bench's
    recipe) stepped 10^4 times persistently (its default, 2176 items per step on 760 CTAs)
    and with one launch per step ends in the same populations bit for bit."""
    from paper_1211_6932_gb300 import Eos, Lattice, maxwell
    from paper_1211_6932_gb300 import workloads as wl
    a = 0.25
    eos = Eos(a=a, T=0.6 * wl.t_crit(a))
    rl, rv = maxwell(eos)
    rho, _, _ = wl.multi_droplets(4096, 4096, rl, rv, 4.0, 64, 40.0, 200.0, seed=5)

    def run(persistent):
        old = os.environ.get("LBM_PERSISTENT")
        os.environ["LBM_PERSISTENT"] = "1" if persistent else "0"
        try:
            L = Lattice(4096, 4096, eos, sigma=0.114, nu_l=0.05, nu_v=0.5, visc_mode="linear",
                        precision="fp32")
        finally:
            if old is None:
                del os.environ["LBM_PERSISTENT"]
            else:
                os.environ["LBM_PERSISTENT"] = old
        with L:
            assert L.persistent == persistent
            L.init_fields(rho)
            L.step(10000)
            return L.moments(dtype=np.float32)["rho"], L.get_populations()
    rp, fp = run(True)
    rq, fq = run(False)
    assert np.isfinite(rp).all()
    assert np.array_equal(rp, rq) and np.array_equal(fp, fq)
