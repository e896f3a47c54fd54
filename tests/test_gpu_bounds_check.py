"""The bounds-check build (kernels compiled with LBM_BOUNDS_CHECK, standing in for a
memory sanitizer): every global and shared-memory access of the step kernels is checked
against its buffer, and a failed check is reported as LBM_ECORRUPT.  The library is built
in that variant and a child process (LBM_LIBRARY=check) runs both precisions and every
kernel family over degenerate, odd, even and ragged widths, walls, graph replays and
single launches, the moments and diagnostics passes (including the allocation-free
diagnostics, whose partial sums sit in the library's fixed array), and a batch (with a
transposed instance) under uniform and per-instance widths: every check must pass."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import numpy as np
    import torch
    from paper_1211_6932_gb300 import _lib, Batch, Eos, Instance, Lattice, maxwell
    from paper_1211_6932_gb300 import workloads as wl
    from paper_1211_6932_gb300.lattice import TILE_PER_INSTANCE
    assert _lib.lib().lbm_bounds_checked() == 1
    eos = Eos(a=0.25, T=0.7 * wl.t_crit(0.25))
    rl, rv = maxwell(eos)
    s = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25)
    sizes = [(1, 7, False), (5, 3, False), (3, 40, True), (64, 48, False), (131, 70, True),
             (254, 33, False), (253, 20, True), (400, 17, False)]
    tilings = {"fp32": [(0, 0, 0), (32, 2, 1), (96, 2, 5), (128, 2, 0), (64, 1, 3),
                        (256, 1, 0), (TILE_PER_INSTANCE, 2, 0)],
               "fp64": [(0, 0, 0), (64, 1, 2), (128, 1, 7)]}
    n = 0
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    for prec, tl in tilings.items():
        for nx, ny, walls in sizes:
            rho = wl.droplet(nx, ny, rl, rv, 0.3 * min(nx, ny), 4.0)
            for t, v, r in tl:
                with Lattice(nx, ny, eos, sigma=0.114, s=s, nu_l=0.05, nu_v=0.3,
                             visc_mode="step", bc="walls" if walls else "periodic",
                             precision=prec, tile_threads=t, tile_vec=v, tile_rows=r) as L:
                    L.init_fields(rho)
                    L.step(67)
                    L.moments()
                    L.diagnostics()
                    L.diagnostics_noalloc(out)
                    L.step(2)
                    L.sync()
                    L.check_guards()
                    n += 1
    # the batch adds a 40 x 300 instance, stored transposed (two strips of its 300-column
    # rows), and reads every instance back through each host path
    bsizes = sizes + [(40, 300, False)]
    insts = [Instance(nx=nx, ny=ny, eos=eos, sigma=0.114, s=s,
                      bc="walls" if w else "periodic", rho_l=rl, rho_v=rv)
             for nx, ny, w in bsizes]
    for t in (0, TILE_PER_INSTANCE):
        b = Batch(insts, precision="fp32", tile_threads=t)
        assert b.is_transposed(len(sizes)) and not any(map(b.is_transposed, range(len(sizes))))
        for i, (nx, ny, w) in enumerate(bsizes):
            b.init_fields(i, wl.droplet(nx, ny, rl, rv, 0.3 * min(nx, ny), 4.0))
        b.step(67)
        b.diagnostics()
        for i in range(len(bsizes)):
            b.moments(i)
            b.moments(i, dtype=np.float32)
            b.get_populations(i)
        b.check_guards()
        b.close()
        n += 1
    print("ok", n)
''')


@pytest.mark.parametrize("persistent", ["0", "2"])
def test_bounds_check_build_runs_clean(persistent):
    """Once with one launch per step, once with persistent stepping wherever the
    dependency rule allows (LBM_PERSISTENT=2: every FP32 pair tiling of one kernel width)."""
    from paper_1211_6932_gb300 import build
    build.build(check=True)
    env = dict(os.environ, LBM_LIBRARY="check", LBM_PERSISTENT=persistent)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.split()[-2] == "ok", r.stdout[-500:]
