"""CPU-side checks of the C ABI: the library builds, loads and exports every symbol the
headers declare; host-only entry points work; without a GPU nothing falls back to the CPU."""
import ctypes
import glob
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(lbm_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1211_6932_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 30
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_declares_every_header_function():
    from paper_1211_6932_gb300 import _lib
    assert declared_functions() == set(_lib.SIGNATURES)


def test_options_default(lib):
    from paper_1211_6932_gb300 import _lib as C
    o = C.lbm_options()
    lib.lbm_options_default(ctypes.byref(o))
    assert o.precision == C.LBM_FP32_DEV and o.visc_mode == -1 and o.rho_ref < 0
    assert o.tile_threads == 0 and o.tile_rows == 0 and not o.stream


def test_host_maxwell_matches_oracle_quadrature(lib):
    """The library's closed-form Maxwell solver agrees with the oracle's quadrature one."""
    from oracle import thermo
    from paper_1211_6932_gb300 import Eos, maxwell
    for a in (0.125, 0.25, 0.5, 1.0):
        for tr in (0.5, 0.6, 0.75, 0.9):
            T = tr * 0.3773 * a / 4.0
            rl, rv = maxwell(Eos(a=a, T=T))
            ol, ov, _ = thermo.maxwell(a, 4.0, 1.0, T)
            assert math.isclose(rl, ol, rel_tol=1e-10) and math.isclose(rv, ov, rel_tol=1e-9)


def test_host_maxwell_rejects_supercritical(lib):
    from paper_1211_6932_gb300 import Eos, LbmError, maxwell
    with pytest.raises(LbmError):
        maxwell(Eos(a=0.25, T=0.03))


def test_no_cpu_fallback_without_gpu(lib):
    """On a machine without a usable CUDA device lbm_create fails with LBM_ECUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1211_6932_gb300 import Eos, LbmError, Lattice
    with pytest.raises(LbmError) as ei:
        Lattice(8, 8, Eos(a=0.25, T=0.01))
    assert ei.value.code == -3


def test_create_validates_arguments(lib):
    """Argument checks run before any device work (error code EINVAL, not ECUDA)."""
    from paper_1211_6932_gb300 import Eos, LbmError, Lattice
    for kw in ({"s": (1.0,) * 8 + (2.5,)}, {"visc_mode": "step"}):
        with pytest.raises(LbmError) as ei:
            Lattice(8, 8, Eos(a=0.25, T=0.01), **kw)
        assert ei.value.code == -1
    with pytest.raises(LbmError) as ei:
        Lattice(0, 8, Eos(a=0.25, T=0.01))
    assert ei.value.code == -1
