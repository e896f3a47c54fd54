"""The boundary from plain C: tests/c/droplet.c includes only include/lbm.h, links the
shared library with gcc, runs a droplet for 500 steps and reports through printf (on a
machine without a GPU the same program gets LBM_ECUDA from lbm_create: no fallback)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    from paper_1211_6932_gb300 import _lib
    lib_dir = os.path.dirname(_lib.LIB_PATH)
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    exe = str(tmp_path / "droplet")
    subprocess.run(["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "droplet.c"), "-o", exe,
                    "-L", lib_dir, "-llbm_gb300", "-Wl,-rpath," + lib_dir, "-lm"],
                   check=True)
    return exe


def test_c_program_without_a_gpu_gets_ecuda(tmp_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([_build(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 3 and "no CUDA device" in r.stderr, (r.returncode, r.stderr)


@pytest.mark.gpu
def test_c_program_runs_a_droplet(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    vals = dict(zip(r.stdout.split()[0::2], r.stdout.split()[1::2]))
    assert float(vals["mass_drift"]) < 1e-6
    assert 0.0 < float(vals["max_u"]) < 0.05
    assert float(vals["rho_centre"]) > 0.3 and float(vals["rho_corner"]) < 0.02
    assert int(vals["steps"]) == 500
