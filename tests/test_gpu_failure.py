"""Failure detection on the GPU without a fault: a bounded wait that runs out is reported
as LBM_ETIMEOUT through the handle's status word, and the context stays usable."""
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


def test_selftest_rejects_bad_poll_counts():
    from paper_1211_6932_gb300 import LbmError
    c = pairs.case(32, 32, tr=0.7, sigma=0.114)
    with pairs.gpu_lattice(c, "fp32") as L:
        for polls in (0, -3, 1 << 21):
            with pytest.raises(LbmError) as ei:
                L.selftest_timeout(polls)
            assert ei.value.code == -1
        L.sync()  # nothing was launched
