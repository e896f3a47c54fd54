"""The JSON-lines run log of Lattice.run: one record per interval with the step count,
the diagnostics of the Eq. 6 fields and the interval's MLUPS."""
import io
import json

import pytest

from tests import pairs

pytestmark = pytest.mark.gpu


def test_run_writes_one_json_record_per_interval():
    from paper_1211_6932_gb300 import workloads as wl
    c = pairs.case(96, 64, tr=0.7, sigma=0.114)
    rl, rv = pairs.maxwell(c)
    buf = io.StringIO()
    with pairs.gpu_lattice(c, "fp32") as L:
        L.init_fields(wl.droplet(96, 64, rl, rv, 18.0, 4.0))
        m0 = L.diagnostics()["mass"]
        recs = L.run(250, log_every=100, log=buf)
        d = L.diagnostics()
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert lines == recs
    assert [r["step"] for r in recs] == [100, 200, 250]
    for r in recs:
        assert r["nonfinite"] == 0 and r["mlups"] > 0
        assert abs(r["mass"] / m0 - 1) < 1e-6
        assert 0 < r["max_u"] < 0.1 and r["dinf"] > 0
    assert d["step"] == 250
