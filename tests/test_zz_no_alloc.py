"""The allocation-free diagnostics entry point against lbm_diagnostics.

lbm_diagnostics_noalloc serves callers that may not allocate device memory (work being
captured into a CUDA graph, fixed memory budgets).  It runs the same reduction with its
partial sums in a fixed array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also passes alone
in a fresh process (the array's address is looked up by the first call).
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
