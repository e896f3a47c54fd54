"""Failure detection on the GPU without a fault: a bounded wait that runs out is reported
as LBM_ETIMEOUT through the handle's status word, and the context stays usable; guard
bands around the device buffers catch writes outside them; an out-of-memory injected at
any allocation is reported and leaves nothing allocated."""
import numpy as np
import pytest

from tests import pairs

pytestmark = pytest.mark.gpu


def test_bounded_wait_timeout_is_reported_and_context_survives():
    from paper_1211_6932_gb300 import LbmError
    c = pairs.case(96, 80, tr=0.7, sigma=0.114)
    f = pairs.droplet_state(c, vel=0.01)
    with pairs.gpu_lattice(c, "fp32") as L, pairs.gpu_lattice(c, "fp32") as ref:
        L.set_populations(f)
        L.step(5)
        with pytest.raises(LbmError) as ei:
            L.selftest_timeout(1000)
        assert ei.value.code == -5
        with pytest.raises(LbmError) as ei:  # stays reported until the state is replaced
            L.sync()
        assert ei.value.code == -5
        L.set_populations(f)
        ref.set_populations(f)
        L.step(20)
        ref.step(20)
        L.sync()
        assert np.array_equal(L.get_populations(), ref.get_populations())


@pytest.mark.parametrize("walls", [False, True])
def test_persistent_dependency_wait_runs_out_cleanly(walls):
    """The persistent kernel's dependency wait on a counter that nothing increments gives
    up after its bound: LBM_ETIMEOUT, reported until the state is replaced, the current
    state untouched, and the lattice then steps (persistently) as a fresh one does."""
    from paper_1211_6932_gb300 import LbmError
    c = pairs.case(300, 70, tr=0.7, sigma=0.114, walls=walls)
    f = pairs.droplet_state(c, vel=0.01)
    with pairs.gpu_lattice(c, "fp32") as L, pairs.gpu_lattice(c, "fp32") as ref:
        L.set_populations(f)
        with pytest.raises(LbmError) as ei:
            L.selftest_dep_timeout(2000)
        assert ei.value.code == -5
        with pytest.raises(LbmError) as ei:
            L.sync()
        assert ei.value.code == -5
        # the populations are copied before the status is reported
        from paper_1211_6932_gb300.lattice import _d
        g = np.empty((9,) + L.shape)
        assert L._L.lbm_get_populations(L.handle, _d(g)) == -5
        ref.set_populations(f)
        assert np.array_equal(g, ref.get_populations())
        L.set_populations(f)
        ref.set_populations(f)
        L.step(70)
        ref.step(70)
        L.sync()
        assert np.array_equal(L.get_populations(), ref.get_populations())
        for polls in (0, 1 << 21):
            with pytest.raises(LbmError) as ei:
                L.selftest_dep_timeout(polls)
            assert ei.value.code == -1


def test_selftest_rejects_bad_poll_counts():
    from paper_1211_6932_gb300 import LbmError
    c = pairs.case(32, 32, tr=0.7, sigma=0.114)
    with pairs.gpu_lattice(c, "fp32") as L:
        for polls in (0, -3, 1 << 21):
            with pytest.raises(LbmError) as ei:
                L.selftest_timeout(polls)
            assert ei.value.code == -1
        L.sync()  # nothing was launched


GUARD_CASES = [
    (pairs.case(96, 80, tr=0.7, sigma=0.114), "fp32"),
    (pairs.case(97, 41, tr=0.7, sigma=0.114, walls=True, visc="step", nu_l=0.05, nu_v=0.3),
     "fp32"),
    (pairs.case(5, 3, a=1.0, tr=0.9, sigma=0.11), "fp32"),
    (pairs.case(70, 45, a=0.5, tr=0.8, sigma=0.11), "fp64"),
]


@pytest.mark.parametrize("c,prec", GUARD_CASES)
def test_guard_bands_stay_intact(c, prec, tmp_path):
    """Every write of the step, moments, diagnostics, population and checkpoint paths
    stays inside its buffer: the guard bands around the slabs, fields, previous density
    and staging buffer are intact afterwards (odd and even widths, walls, both
    precisions, graph replays and single launches)."""
    rl, rv = pairs.maxwell(c)
    from paper_1211_6932_gb300 import workloads as wl
    rho = wl.droplet(c["nx"], c["ny"], rl, rv, 0.3 * min(c["nx"], c["ny"]), 4.0)
    with pairs.gpu_lattice(c, prec) as L:
        L.init_fields(rho)
        L.step(70)
        L.diagnostics()
        L.moments()
        L.step(3)
        L.diagnostics()
        f = L.get_populations()
        L.set_populations(f)
        L.save(str(tmp_path / "s.lbm"))
        L.load(str(tmp_path / "s.lbm"))
        L.step(1)
        L.check_guards()


def test_guard_bands_of_a_batch_stay_intact():
    from paper_1211_6932_gb300 import Batch, Eos, Instance
    from paper_1211_6932_gb300.lattice import TILE_PER_INSTANCE
    from paper_1211_6932_gb300 import workloads as wl
    cs = [GUARD_CASES[0][0], GUARD_CASES[1][0], GUARD_CASES[2][0],
          pairs.case(400, 40, a=0.25, tr=0.75, sigma=0.114)]
    insts = []
    for c in cs:
        rl, rv = pairs.maxwell(c)
        insts.append(Instance(nx=c["nx"], ny=c["ny"], eos=Eos(a=c["a"], T=c["T"]), G=c["G"],
                              sigma=c["sigma"], s=c["s"], nu_l=c["nu_l"], nu_v=c["nu_v"],
                              visc_mode=c["visc"],
                              bc="walls" if c["walls"] else "periodic", rho_c=0.5218 / 4.0,
                              rho_l=rl, rho_v=rv))
    for threads in (0, TILE_PER_INSTANCE):
        b = Batch(insts, precision="fp32", tile_threads=threads)
        try:
            for i, c in enumerate(cs):
                rl, rv = pairs.maxwell(c)
                b.init_fields(i, wl.droplet(c["nx"], c["ny"], rl, rv,
                                            0.3 * min(c["nx"], c["ny"]), 4.0))
            b.step(67)
            b.diagnostics()
            for i in range(len(cs)):
                b.moments(i)
            b.check_guards()
        finally:
            b.close()


def test_guard_corruption_is_reported():
    """A byte written just past a guarded buffer (planted from the host) is reported as
    LBM_ECORRUPT naming the buffer."""
    from paper_1211_6932_gb300 import LbmError
    c = pairs.case(64, 48, tr=0.7, sigma=0.114)
    for which, name in ((0, "population slab 0"), (1, "population slab 1"),
                        (2, "previous density")):
        with pairs.gpu_lattice(c, "fp32") as L:
            L.check_guards()
            L.debug_corrupt_guard(which)
            with pytest.raises(LbmError) as ei:
                L.check_guards()
            assert ei.value.code == -8 and name in str(ei.value), str(ei.value)
    with pairs.gpu_lattice(c, "fp32") as L:
        with pytest.raises(LbmError) as ei:
            L.debug_corrupt_guard(7)
        assert ei.value.code == -1


def test_allocation_failures_are_reported_and_release_everything():
    """Out-of-memory injected at every device allocation of a lattice's life (create,
    equilibrium start, stepping, moments, diagnostics, autotuning) is reported as
    LBM_ENOMEM by the call that allocates, and once the handle is closed every device
    allocation it made is released."""
    from paper_1211_6932_gb300 import LbmError
    from paper_1211_6932_gb300.lattice import debug_fail_alloc, debug_live_allocs
    from paper_1211_6932_gb300 import workloads as wl
    c = pairs.case(64, 48, tr=0.7, sigma=0.114)
    rl, rv = pairs.maxwell(c)
    rho = wl.droplet(64, 48, rl, rv, 12.0, 4.0)

    def life():
        with pairs.gpu_lattice(c, "fp32") as L:
            L.init_fields(rho)
            L.step(66)
            L.moments()
            L.diagnostics()
            L.autotune(steps=2)
            L.get_populations()

    life()  # module loading and first-use work outside the count
    base = debug_live_allocs()
    failures = 0
    try:
        for k in range(200):
            debug_fail_alloc(k)
            try:
                life()
            except LbmError as e:
                assert e.code == -2, (k, e)
                failures += 1
            armed = debug_fail_alloc(-1)
            assert debug_live_allocs() == base, k
            if armed >= 0:  # the k-th allocation was never reached: every one was tried
                break
        else:
            raise AssertionError("more than 200 allocations in one lattice's life")
    finally:
        debug_fail_alloc(-1)
    assert failures == k and failures >= 8, failures
