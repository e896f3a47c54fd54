"""The allocation-free diagnostics entry point against lbm_diagnostics.

lbm_diagnostics_noalloc serves callers that may not allocate device memory: a plug-in
whose host application owns the whole device-memory budget, or a time-critical loop that
cannot afford cudaMalloc/cudaFree (they may synchronise the device).  It runs the same
reduction with its partial sums in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run every other
test; it also passes alone in a fresh process (the array's address is looked up by the
first call).
"""
import numpy as np
import pytest

from tests import pairs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_noalloc_diagnostics_match_lbm_diagnostics(prec, rtol):
    import torch
    c = pairs.case(150, 90, tr=0.65, sigma=0.114, walls=True)
    f = pairs.droplet_state(c, vel=0.02)
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    with pairs.gpu_lattice(c, prec) as L:
        L.set_populations(f)
        for call in range(2):  # two calls in a row, with steps in between
            L.step(7)
            ref = L.diagnostics()
            L.diagnostics_noalloc(out)
            L.sync()
            got = out.cpu().numpy()
            for k, key in enumerate(("mass", "mom_x", "mom_y", "max_u")):
                scale = max(abs(ref["mass"]) * 1e-6, abs(ref[key])) if k else abs(ref[key])
                assert abs(got[k] - ref[key]) <= rtol * scale, (call, key, got[k], ref[key])
            assert got[4] == 0.0 and got[5] == ref["nonfinite"] == 0
            assert np.isfinite(got).all()


def test_noalloc_rejects_lattices_beyond_the_fixed_array():
    """A lattice whose tiling needs more work items than LBM_NOALLOC_MAX_ITEMS (FP64,
    64-thread strips of 60 columns, one-row chunks: 10 strips x 2000 rows = 20000 items)
    is refused with LBM_EINVAL and nothing is queued: the output keeps its contents."""
    import torch

    from paper_1211_6932_gb300 import Eos, Lattice, LbmError, maxwell
    from paper_1211_6932_gb300 import workloads as wl
    eos = Eos(a=0.25, T=0.7 * wl.t_crit(0.25))
    rl, rv = maxwell(eos)
    out = torch.full((6,), 7.0, dtype=torch.float64, device="cuda")
    with Lattice(600, 2000, eos, sigma=0.114, precision="fp64", tile_threads=64,
                 tile_rows=1) as L:
        L.init_fields(wl.droplet(600, 2000, rl, rv, 100.0, 4.0))
        with pytest.raises(LbmError) as ex:
            L.diagnostics_noalloc(out)
        assert ex.value.code == -1 and "work items" in str(ex.value)  # LBM_EINVAL
        L.sync()
        assert torch.all(out == 7.0).item()
        # the same lattice with taller chunks fits, and matches lbm_diagnostics
        L.set_tiling(64, 1, 64)
        ref = L.diagnostics()
        L.diagnostics_noalloc(out)
        L.sync()
        got = out.cpu().numpy()
        assert abs(got[0] - ref["mass"]) <= 1e-12 * ref["mass"]
