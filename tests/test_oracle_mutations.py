"""Mutation check of the oracle's pins: each plausible mistake below (a dropped term, a
wrong sign, a wrong weight or index, a transposed operand), written into a copy of the
oracle, must make the committed pins fail.  The C step (lbm_oracle.c) is altered in a
copy compiled into a temporary directory and loaded by a child pytest through
LBM_ORACLE_LIB; a Python module of the oracle (the pressure tensor of Eq. 18, the
thermodynamics, the warm-start network and measurements) is altered in a copy whose
definitions a child process puts in place of the module's before it runs its pins.  The oracle's own sources are never touched.
Control copies without any change must pass the same pins, so that a failure means the
mistake was caught, not that the harness broke.  The two slowest pins (the Table II
droplet run and Laplace's law) are left out of these runs to keep them short; every
mistake is caught without them."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

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
    ("pseudopotential without the clamp of a negative argument", "Eq. 24 (reading)",
     "if (arg < 0.0) arg = 0.0;", ""),
    ("force reported without its psi(x) factor", "Eq. 7",
     "if (Fx_out) Fx_out[n] = psi[n] * fpx[n];", "if (Fx_out) Fx_out[n] = fpx[n];"),
    ("bounce-back at the bottom wall only", "Sec. IV C",
     "if (p->walls && (yd < 0 || yd >= ny)) {", "if (p->walls && (yd < 0)) {"),
    ("psi above the top wall read from the bottom row", "Sec. IV C",
     "if (y >= p->ny) y = p->ny - 1;", "if (y >= p->ny) y = 0;"),
    ("equilibrium populations through M instead of M^-1", "Eq. 3",
     "for (int i = 0; i < Q; ++i) acc += Minv[a][i] * meq[i];",
     "for (int i = 0; i < Q; ++i) acc += M[i][a] * meq[i] / 9.0;"),
    ("collision relaxing away from the equilibrium", "Eq. 4",
     "ms[i] = m[i] - lam[i] * (m[i] - meq[i])", "ms[i] = m[i] - lam[i] * (meq[i] - m[i])"),
    ("two diagonal velocities exchanged in the velocity table", "Eq. 3",
     "static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};",
     "static const int EX[Q] = {0, 1, 0, -1, 0, -1, 1, -1, 1};"),
]


PIN_FILES = [os.path.join(ROOT, "tests", f) for f in ("test_oracle_pins.py",
                                                     "test_pressure_oracle.py")]
PYTEST_ARGS = PIN_FILES + ["-x", "-q", "-p", "no:cacheprovider", "-k", FAST]


# The children run side by side, each with a share of the cores for the oracle's OpenMP.
WORKERS = max(1, min(8, os.cpu_count() or 1))


def _env(**extra):
    threads = max(1, (os.cpu_count() or 1) // WORKERS)
    return dict(os.environ, OMP_NUM_THREADS=str(threads), **extra)


def _pins(lib_path):
    cmd = [sys.executable, "-m", "pytest"] + PYTEST_ARGS
    return subprocess.run(cmd, cwd=ROOT, env=_env(LBM_ORACLE_LIB=lib_path),
                          capture_output=True, text=True)


# Child process for a Python module of the oracle: execute the altered copy as that module
# (same package, so its relative imports resolve), put its definitions in place of the
# module's, then run the pins in the same interpreter.
RUNNER = """
import importlib, sys, types
import pytest
name, path = sys.argv[1], sys.argv[2]
real = importlib.import_module(name)
alt = types.ModuleType(name)
alt.__package__ = name.rpartition(".")[0]
alt.__file__ = path
with open(path) as fh:
    exec(compile(fh.read(), path, "exec"), alt.__dict__)
for k, v in list(alt.__dict__.items()):
    if not k.startswith("__"):
        setattr(real, k, v)
sys.exit(pytest.main(sys.argv[3:]))
"""


def _tests(*names):
    return [os.path.join(ROOT, "tests", n) for n in names]


# Each module's pins (its own first, so that a caught mistake ends the run early).  The
# warm-start measurements' file also compares the library's host code with the oracle;
# only the oracle's own pins (test_oracle_*) are run for them.
MODULE_PINS = {
    "oracle.pressure": (_tests("test_pressure_oracle.py", "test_oracle_pins.py"), FAST),
    "oracle.thermo": (_tests("test_oracle_pins.py", "test_pressure_oracle.py"), FAST),
    "oracle.mlp": (_tests("test_mlp_oracle.py"), None),
    "oracle.warm": (_tests("test_warm_host.py"), "test_oracle_"),
}


def _pins_with_module(name, path):
    files, k = MODULE_PINS[name]
    args = files + ["-x", "-q", "-p", "no:cacheprovider"] + (["-k", k] if k else [])
    cmd = [sys.executable, "-c", RUNNER, name, path] + args
    return subprocess.run(cmd, cwd=ROOT, env=_env(), capture_output=True, text=True)


def _compile(tmp_path, name, text):
    src = os.path.join(tmp_path, name + ".c")
    with open(src, "w") as fh:
        fh.write(text)
    return obuild.compile_to(src, os.path.join(tmp_path, name + ".so"))


# (what the mistake is, the passage it breaks, module, text in its source, replacement)
PY_MUTATIONS = [
    ("pressure tensor with the diagonal weight 1/6", "Eqs. 7, 18", "oracle.pressure",
     "_W = {1: 1.0 / 3.0, 2: 1.0 / 12.0}", "_W = {1: 1.0 / 3.0, 2: 1.0 / 6.0}"),
    ("pressure tensor without the factor 1/2 of G", "Eq. 18", "oracle.pressure",
     "half = 0.5 * G * psi", "half = G * psi"),
    ("ideal-gas part rho/2 instead of rho c_s^2", "Eq. 18", "oracle.pressure",
     "iso = rho / 3.0 + 2.0 * sigma", "iso = rho / 2.0 + 2.0 * sigma"),
    ("sigma term with G instead of G^2", "Eq. 26", "oracle.pressure",
     "2.0 * sigma * G * G * (gx * gx + gy * gy)", "2.0 * sigma * G * (gx * gx + gy * gy)"),
    ("shear component from e_x e_x", "Eq. 18", "oracle.pressure",
     "sxy += wp * ex * ey", "sxy += wp * ex * ex"),
    ("pressure tensor at walls reading the wrapped row", "Eq. 18 (reading)",
     "oracle.pressure", "idx = np.clip(np.arange(ny) + ey, 0, ny - 1)",
     "idx = (np.arange(ny) + ey) % ny"),
    ("surface tension over both interfaces instead of one", "Eq. 18", "oracle.pressure",
     "return 0.5 * float(np.sum(", "return float(np.sum("),
    ("CS compressibility factor without its cubic term", "Eq. 30", "oracle.thermo",
     "return (1.0 + x + x * x - x ** 3) / (1.0 - x) ** 3", "return (1.0 + x + x * x) / (1.0 - x) ** 3"),
    ("derivative of the CS numerator with a wrong coefficient", "Eq. 30", "oracle.thermo",
     "N1 = 1.0 + 2.0 * x - 3.0 * x * x", "N1 = 1.0 + 2.0 * x - 2.0 * x * x"),
    ("Maxwell rule weighted by 1/rho instead of 1/rho^2", "Eq. 22", "oracle.thermo",
     "lambda r: 1.0 / (r * r)", "lambda r: 1.0 / r"),
    ("epsilon of Eq. 29 with the wrong sign", "Eq. 29", "oracle.thermo",
     "return -2.0 * (alpha + 24.0 * G * sigma) / beta", "return 2.0 * (alpha + 24.0 * G * sigma) / beta"),
    ("mechanical-stability weight psi^(1 - eps) instead of psi^(1 + eps)", "Eq. 21",
     "oracle.thermo", "** (1.0 + eps)", "** (1.0 - eps)"),
    ("lattice sound speed squared 1/2", "Eq. 24", "oracle.thermo",
     "CS2 = 1.0 / 3.0", "CS2 = 1.0 / 2.0"),
    ("pseudopotential without the clamp of a negative argument", "Eq. 24 (reading)",
     "oracle.thermo", "return math.sqrt(max(arg, 0.0))", "return math.sqrt(arg)"),
    ("critical temperature without the factor 2", "Sec. IV A", "oracle.thermo",
     "Tc = 2.0 * a / ((b / 4.0)", "Tc = a / ((b / 4.0)"),
    ("GELU derivative without its z phi(z) term", "GELU", "oracle.mlp",
     "return _phi_cdf(z) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)",
     "return _phi_cdf(z)"),
    ("normal CDF with the wrong sign of its argument", "GELU", "oracle.mlp",
     "return 0.5 * _erfc(-z / math.sqrt(2.0))", "return 0.5 * _erfc(z / math.sqrt(2.0))"),
    ("loss gradient without the factor 2", "squared error", "oracle.mlp",
     "dy = 2.0 * (y - tn) / (n * N_OUT)", "dy = (y - tn) / (n * N_OUT)"),
    ("gradient of the square hidden layer transposed", "chain rule", "oracle.mlp",
     'g["W2"] = dz2.T @ c["h1"]', 'g["W2"] = (dz2.T @ c["h1"]).T'),
    ("Adam without the bias correction of v", "Adam", "oracle.mlp",
     "vhat = v / (1.0 - beta2 ** k)", "vhat = v"),
    ("Adam first moment without the (1 - beta1) weight", "Adam", "oracle.mlp",
     "m = beta1 * m + (1.0 - beta1) * g", "m = beta1 * m + g"),
    ("bf16 rounding half up instead of to even", "bf16", "oracle.mlp",
     "r = (b + np.uint64(0x7FFF) + lsb)", "r = (b + np.uint64(0x8000))"),
    ("inputs multiplied by their scale instead of divided", "standardisation", "oracle.mlp",
     '/ scaling["in_scale"]', '* scaling["in_scale"]'),
    ("integral width with the factor 2 instead of 4", "Eq. 31", "oracle.warm",
     "width = 4.0 * float(np.sum(g * (1.0 - g))) / 2.0",
     "width = 2.0 * float(np.sum(g * (1.0 - g))) / 2.0"),
    ("equimolar radius from the inner density alone", "Eq. 31", "oracle.warm",
     "(math.pi * (ri - ro))", "(math.pi * ri)"),
    ("Laplace coefficient divided by the radius", "Eq. 30", "oracle.warm",
     "lap = (thermo.p_eos(ri, a, b, R, T) - thermo.p_eos(ro, a, b, R, T)) * Rg",
     "lap = (thermo.p_eos(ri, a, b, R, T) - thermo.p_eos(ro, a, b, R, T)) / Rg"),
    ("vapour law returning the slope without dividing by rho_v", "1/R law", "oracle.warm",
     "return float(rv), float(s / rv)", "return float(rv), float(s)"),
    ("liquid response taken at the vapour's compressibility", "Eq. 30", "oracle.warm",
     'dp / thermo.dp_drho(p["rho_l"], a, b, R, T)', "dp / thermo.dp_drho(ro, a, b, R, T)"),
    ("droplet field with the tanh profile inverted", "Eq. 31", "oracle.warm",
     "- 0.5 * (ri - rho_v) * np.tanh(2.0 * s / width)",
     "+ 0.5 * (ri - rho_v) * np.tanh(2.0 * s / width)"),
    ("Gibbs surface from the whole liquid excess instead of half", "Eq. 31", "oracle.warm",
     "yg = c + L / 2.0", "yg = c + L"),
]


def _module_source(name):
    path = os.path.join(ROOT, *name.split(".")) + ".py"
    with open(path) as fh:
        return fh.read()


def _write(tmp_path, name, text):
    path = os.path.join(tmp_path, name.replace(".", "_") + ".py")
    with open(path, "w") as fh:
        fh.write(text)
    return path


@pytest.fixture(scope="module")
def source():
    with open(obuild.SRC) as fh:
        return fh.read()


@pytest.fixture(scope="module")
def runs(source, tmp_path_factory):
    """Every copy's pin run, side by side: {(kind, what): CompletedProcess}."""
    d = str(tmp_path_factory.mktemp("mutants"))
    jobs = {("c", "control"): (lambda: _pins(_compile(d, "c_control", source)))}
    for i, (what, _, old, new) in enumerate(MUTATIONS):
        if source.count(old) == 1:
            text = source.replace(old, new)
            jobs[("c", what)] = (lambda t=text, k="c_%d" % i: _pins(_compile(d, k, t)))
    for name in sorted(MODULE_PINS):
        path = _write(d, name + "_control", _module_source(name))
        jobs[("py", name)] = (lambda n=name, p=path: _pins_with_module(n, p))
    for i, (what, _, name, old, new) in enumerate(PY_MUTATIONS):
        text = _module_source(name)
        if text.count(old) == 1:
            path = _write(d, "%s_%d" % (name, i), text.replace(old, new))
            jobs[("py", what)] = (lambda n=name, p=path: _pins_with_module(n, p))
    with ThreadPoolExecutor(WORKERS) as ex:
        futures = {k: ex.submit(f) for k, f in jobs.items()}
        return {k: f.result() for k, f in futures.items()}


def test_unaltered_copy_passes_the_pins(runs):
    r = runs[("c", "control")]
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("what,passage,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mistake(runs, source, what, passage, old, new):
    assert source.count(old) == 1, "the text to alter must occur exactly once"
    r = runs[("c", what)]
    assert r.returncode == 1, (what, passage, r.stdout[-2000:])


@pytest.mark.parametrize("name", sorted(MODULE_PINS))
def test_unaltered_module_copy_passes_the_pins(runs, name):
    r = runs[("py", name)]
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("what,passage,name,old,new", PY_MUTATIONS,
                         ids=[m[0] for m in PY_MUTATIONS])
def test_pins_catch_the_mistake_in_a_module(runs, what, passage, name, old, new):
    assert _module_source(name).count(old) == 1, "the text to alter must occur exactly once"
    r = runs[("py", what)]
    assert r.returncode == 1, (what, passage, r.stdout[-2000:])


def test_the_check_loads_the_named_build():
    """LBM_ORACLE_LIB names the shared object the oracle package loads."""
    code = "import oracle; print(oracle.lib()._name)"
    path = oracle.build.build()
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, LBM_ORACLE_LIB=path))
    assert r.returncode == 0 and r.stdout.strip() == path
