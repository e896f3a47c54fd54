"""Mutation check of the oracle's pins: each plausible mistake below (a dropped term, a
wrong sign, a wrong weight or index, a transposed operand), written into a copy of the C
oracle, must make the committed pins (tests/test_oracle_pins.py) fail.  Each altered copy
is compiled into a temporary directory and loaded by a child pytest through
LBM_ORACLE_LIB; the oracle's own source is never touched.  A control copy without any
change must pass the same pins, so that a failure means the mistake was caught, not that
the harness broke.  The two slowest pins (the Table II droplet run and Laplace's law) are
left out of these runs to keep them short; every mistake is caught without them."""
import os
import subprocess
import sys

import pytest

import oracle
from oracle import build as obuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAST = "not table_ii_numerical_droplet and not laplace_law"

# (what the mistake is, the passage it breaks, text in lbm_oracle.c, its replacement)
MUTATIONS = [
    ("velocity without the F/2 term", "Eq. 6",
     "ux[n] = (jx + 0.5 * Fx) / rho[n];", "ux[n] = jx / rho[n];"),
    ("improved forcing term of the energy moment with the wrong sign", "Eq. 25",
     "S[1] = 6.0 * vF + 12.0", "S[1] = 6.0 * vF - 12.0"),
    ("improved forcing term of the energy-square moment dropped", "Eq. 25",
     "S[2] = -6.0 * vF - 12.0 * p->sigma * F2_over_psi2 / (tau_z - 0.5);",
     "S[2] = -6.0 * vF;"),
    ("forcing of p_xx with the wrong sign between its terms", "Eq. 9",
     "S[7] = 2.0 * (vx * Fx - vy * Fy);", "S[7] = 2.0 * (vx * Fx + vy * Fy);"),
    ("forcing applied without the (I - Lambda/2) factor", "Eq. 4",
     "+ (1.0 - 0.5 * lam[i]) * S[i];", "+ S[i];"),
    ("Carnahan-Starling numerator without its cubic term", "Eq. 30",
     "double num = 1.0 + x + x * x - x * x * x;", "double num = 1.0 + x + x * x;"),
    ("pseudopotential without the factor 2", "Eq. 24",
     "double arg = 2.0 * (oracle_p_eos", "double arg = 1.0 * (oracle_p_eos"),
    ("diagonal interaction weight 1/36 instead of 1/12", "Eq. 7",
     "if (e2 == 2) return 1.0 / 12.0;", "if (e2 == 2) return 1.0 / 36.0;"),
    ("interaction force with the wrong sign", "Eq. 7",
     "fpx[n] = -p->G * sx;", "fpx[n] = p->G * sx;"),
    ("M^-1 built from M without the transpose", "Eq. 5",
     "Minv[b][i] = M[i][b] / n2;", "Minv[i][b] = M[i][b] / n2;"),
    ("equilibrium of q_x with the wrong sign", "Eq. 3",
     "meq[4] = -rho * vx;", "meq[4] = rho * vx;"),
    ("linear viscosity mode interpolating the rate instead of the relaxation time",
     "Sec. IV C",
     "return 1.0 / (tau_v + frac * (tau_l - tau_v));",
     "return 1.0 / tau_v + frac * (1.0 / tau_l - 1.0 / tau_v);"),
    ("step viscosity mode with the phases exchanged", "Sec. IV C",
     "double nu = (rho >= p->rho_c) ? p->nu_l : p->nu_v;",
     "double nu = (rho >= p->rho_c) ? p->nu_v : p->nu_l;"),
    ("bounce-back at a wall keeping the incoming direction", "Sec. IV C",
     "fnew[OPP[a] * N + n] = fstar[a * N + n];", "fnew[a * N + n] = fstar[a * N + n];"),
    ("streaming against the lattice velocity in x", "Eq. 5",
     "int xd = wrap(x + EX[a], nx);", "int xd = wrap(x - EX[a], nx);"),
    ("two diagonal velocities exchanged in the velocity table", "Eq. 3",
     "static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};",
     "static const int EX[Q] = {0, 1, 0, -1, 0, -1, 1, -1, 1};"),
]


def _pins(lib_path):
    env = dict(os.environ, LBM_ORACLE_LIB=lib_path)
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
           "-x", "-q", "-p", "no:cacheprovider", "-k", FAST]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True)


def _compile(tmp_path, name, text):
    src = os.path.join(tmp_path, name + ".c")
    with open(src, "w") as fh:
        fh.write(text)
    return obuild.compile_to(src, os.path.join(tmp_path, name + ".so"))


@pytest.fixture(scope="module")
def source():
    with open(obuild.SRC) as fh:
        return fh.read()


def test_unaltered_copy_passes_the_pins(source, tmp_path):
    r = _pins(_compile(str(tmp_path), "control", source))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("what,passage,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mistake(source, tmp_path, what, passage, old, new):
    assert source.count(old) == 1, "the text to alter must occur exactly once"
    r = _pins(_compile(str(tmp_path), "mutant", source.replace(old, new)))
    assert r.returncode == 1, (what, passage, r.stdout[-2000:])


def test_the_check_loads_the_named_build(tmp_path):
    """LBM_ORACLE_LIB names the shared object the oracle package loads."""
    code = "import oracle; print(oracle.lib()._name)"
    path = oracle.build.build()
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, LBM_ORACLE_LIB=path))
    assert r.returncode == 0 and r.stdout.strip() == path
