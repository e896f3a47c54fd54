"""Python front end of the C ABI (include/lbm.h).  Marshalling only: every step of the
method runs in the CUDA library."""
import ctypes
import dataclasses

import numpy as np

from . import _lib as C

_PREC = {"fp64": C.LBM_FP64, "fp32": C.LBM_FP32_DEV, "fp32_dev": C.LBM_FP32_DEV}
_VISC = {None: -1, "const": C.LBM_VISC_CONST, "step": C.LBM_VISC_STEP,
         "linear": C.LBM_VISC_LINEAR}
TILE_PER_INSTANCE = C.LBM_TILE_PER_INSTANCE  # tile_threads: a kernel width per instance


def debug_fail_alloc(n):
    """lbm_debug_fail_alloc: the next n device allocations of lattice and batch handles
    succeed and the one after fails with LBM_ENOMEM (n < 0 disarms); returns the previous
    setting."""
    return C.lib().lbm_debug_fail_alloc(int(n))


def debug_live_allocs():
    """lbm_debug_live_allocs: device allocations of lattice and batch handles not yet
    released (process-wide)."""
    return int(C.lib().lbm_debug_live_allocs())
_BC = {"periodic": C.LBM_BC_PERIODIC, "walls": C.LBM_BC_WALLS_Y, "walls_y": C.LBM_BC_WALLS_Y}
_LAYOUT = {"auto": C.LBM_LAYOUT_AUTO, "rows": C.LBM_LAYOUT_ROWS,
           "transposed": C.LBM_LAYOUT_TRANSPOSED}


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lbm error %d: %s" % (code, msg))
        self.code = code


@dataclasses.dataclass
class Eos:
    """Carnahan-Starling parameters (Eq. 30)."""
    a: float
    T: float
    b: float = 4.0
    R: float = 1.0

    def c(self):
        return C.lbm_eos(self.a, self.b, self.R, self.T)


def _d(a):
    return a.ctypes.data_as(C.dptr) if a is not None else None


def _f(a):
    return a.ctypes.data_as(C.fptr) if a is not None else None


def _f32(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _f64(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _device_of(stream, device):
    if device is not None:
        return int(device)
    dev = getattr(stream, "device", None)
    if dev is not None and getattr(dev, "index", None) is not None:
        return int(dev.index)
    return -1


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def maxwell(eos: Eos):
    """Maxwell equal-area coexistence densities (Eq. 22) from the library's host solver."""
    L = C.lib()
    rl, rv = ctypes.c_double(), ctypes.c_double()
    rc = L.lbm_maxwell(eos.c(), ctypes.byref(rl), ctypes.byref(rv))
    if rc != 0:
        raise LbmError(rc, "no Maxwell solution (T must be below T_c)")
    return rl.value, rv.value


def mechanical_stability(eos: Eos, sigma, G=-1.0):
    """Flat-interface coexistence densities of Eq. 21 (library host solver)."""
    rl, rv = ctypes.c_double(), ctypes.c_double()
    rc = C.lib().lbm_mechanical_stability(eos.c(), float(G), float(sigma), ctypes.byref(rl),
                                          ctypes.byref(rv))
    if rc != 0:
        raise LbmError(rc, "no solution of the mechanical-stability condition")
    return rl.value, rv.value


def sigma_consistent(eos: Eos, G=-1.0):
    """The sigma that makes Eq. 21 give the Maxwell vapour density (library host solver)."""
    s = ctypes.c_double()
    rc = C.lib().lbm_sigma_consistent(eos.c(), float(G), ctypes.byref(s))
    if rc != 0:
        raise LbmError(rc, "no consistent sigma bracketed")
    return s.value


def _diag_dict(d):
    return {"mass": d.mass, "mom_x": d.mom_x, "mom_y": d.mom_y, "max_u": d.max_u,
            "dinf": d.dinf, "step": d.step, "nonfinite": d.nonfinite}


class Lattice:
    """One nx x ny lattice (lbm_create ... lbm_destroy)."""

    def __init__(self, nx, ny, eos: Eos, G=-1.0, sigma=0.0, s=None, nu_l=0.0, nu_v=0.0,
                 precision="fp32", visc_mode=None, bc="periodic", psi_fp64=False,
                 rho_ref=None, rho_c=None, rho_l=None, rho_v=None, stream=None, tile_threads=0,
                 tile_rows=0, device=None, tile_vec=0):
        self._L = C.lib()
        self.nx, self.ny = int(nx), int(ny)
        self.precision = precision
        s = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0) if s is None else s
        sv = (ctypes.c_double * 9)(*[float(v) for v in s])
        o = C.lbm_options()
        self._L.lbm_options_default(ctypes.byref(o))
        o.precision = _PREC[precision]
        o.visc_mode = _VISC[visc_mode]
        o.bc = _BC[bc]
        o.psi_fp64 = int(bool(psi_fp64))
        if rho_ref is not None:
            o.rho_ref = float(rho_ref)
        if rho_c is not None:
            o.rho_c = float(rho_c)
        if rho_l is not None:
            o.rho_l = float(rho_l)
        if rho_v is not None:
            o.rho_v = float(rho_v)
        sp = _stream_ptr(stream)
        o.stream = sp.value if sp is not None else None
        o.device = _device_of(stream, device)
        o.tile_threads = int(tile_threads)
        o.tile_vec = int(tile_vec)
        o.tile_rows = int(tile_rows)
        h = ctypes.c_void_p()
        rc = self._L.lbm_create(ctypes.byref(h), self.nx, self.ny, eos.c(), float(G),
                                float(sigma), sv, float(nu_l), float(nu_v), ctypes.byref(o))
        if rc != 0:
            raise LbmError(rc, self._L.lbm_last_error(None).decode())
        self._h = h
        self.stream_keepalive = stream
        self._in_flight = []  # host arrays of asynchronous transfers, until the next sync

    # -- helpers -----------------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise LbmError(rc, self._L.lbm_last_error(self._h).decode())
        return rc

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        return (self.ny, self.nx)

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state ---------------------------------------------------------------------------
    def init_fields(self, rho, ux=None, uy=None):
        """Equilibrium start from host (ny, nx) fields; float32 arrays take the float
        transfer (lbm_init_fields_f32), anything else is sent as float64."""
        if getattr(rho, "dtype", None) == np.float32:
            r, u, v = _f32(rho, self.shape), _f32(ux, self.shape), _f32(uy, self.shape)
            self._check(self._L.lbm_init_fields_f32(self._h, _f(r), _f(u), _f(v)))
            return
        r = _f64(rho, self.shape)
        u = _f64(ux, self.shape)
        v = _f64(uy, self.shape)
        self._check(self._L.lbm_init_fields(self._h, _d(r), _d(u), _d(v)))

    def init_fields_device(self, rho, ux=None, uy=None):
        """rho/ux/uy: contiguous float64 CUDA tensors of shape (ny, nx)."""
        ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._check(self._L.lbm_init_fields_device(self._h, ptr(rho), ptr(ux), ptr(uy)))

    def set_populations(self, f):
        f = _f64(f, (9,) + self.shape)
        self._check(self._L.lbm_set_populations(self._h, _d(f)))

    def get_populations(self):
        f = np.empty((9,) + self.shape)
        self._check(self._L.lbm_get_populations(self._h, _d(f)))
        return f

    def step(self, n=1):
        self._check(self._L.lbm_step(self._h, int(n)))

    @property
    def persistent(self):
        """Whether steps run as persistent launches (lbm_persistent)."""
        rc = self._L.lbm_persistent(self._h)
        if rc < 0:
            self._check(rc)
        return bool(rc)

    def sync(self):
        """lbm_sync: wait for the queued steps and asynchronous transfers."""
        try:
            self._check(self._L.lbm_sync(self._h))
        finally:
            self._in_flight.clear()

    def _async_array(self, a, writable):
        """A host array for an asynchronous transfer: (ny, nx), C-contiguous, of the
        storage type (float32 for FP32, float64 for FP64), used in place (no copy, so that
        the caller's, possibly page-locked, buffer is the one transferred)."""
        if a is None:
            return None
        dt = np.float64 if self.precision == "fp64" else np.float32
        if not isinstance(a, np.ndarray) or a.dtype != dt or a.shape != self.shape or \
                not a.flags["C_CONTIGUOUS"] or (writable and not a.flags["WRITEABLE"]):
            raise ValueError("asynchronous transfers take C-contiguous %s arrays of shape %s"
                             % (np.dtype(dt).name, self.shape))
        return a

    def init_fields_async(self, rho, ux=None, uy=None):
        """lbm_init_fields_async: returns at once; the arrays (see _async_array; page-locked,
        e.g. torch's pin_memory().numpy(), for the copy to overlap) stay referenced, and
        must stay unchanged, until the next sync(), which reports invalid fields."""
        arrs = [self._async_array(a, False) for a in (rho, ux, uy)]
        ptr = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        self._in_flight.extend(a for a in arrs if a is not None)
        self._check(self._L.lbm_init_fields_async(self._h, *[ptr(a) for a in arrs]))

    def moments_async(self, rho, ux=None, uy=None):
        """lbm_moments_async into the given arrays (see _async_array) of the state after the
        steps queued so far; they hold the fields after the next sync()."""
        arrs = [self._async_array(a, True) for a in (rho, ux, uy)]
        ptr = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        self._in_flight.extend(a for a in arrs if a is not None)
        self._check(self._L.lbm_moments_async(self._h, *[ptr(a) for a in arrs]))

    def pressure_tensor(self, include_sigma=False):
        """(pxx, pyy, pxy) of Eq. 18 as (ny, nx) arrays (lbm_pressure_tensor)."""
        out = [np.empty(self.shape) for _ in range(3)]
        self._check(self._L.lbm_pressure_tensor(self._h, *[_d(a) for a in out],
                                                1 if include_sigma else 0))
        return tuple(out)

    def check_guards(self):
        """lbm_check_guards: raises LbmError (LBM_ECORRUPT) if a guard band around one of
        the handle's device buffers was overwritten."""
        self._check(self._L.lbm_check_guards(self._h))

    def debug_corrupt_guard(self, which=0):
        """lbm_debug_corrupt_guard: overwrite one guard byte of buffer `which` (tests)."""
        self._check(self._L.lbm_debug_corrupt_guard(self._h, int(which)))

    def run(self, steps, log_every=100, log=None):
        """Advance `steps` steps; every `log_every` steps (and at the end) append one JSON
        line to `log` (a writable text file, or None to skip writing) with the step count,
        the diagnostics of Eq. 6 fields (mass, momentum, max |v|, |d rho|_inf over the
        interval) and the MLUPS of the interval (wall clock, stream synchronised).
        Returns the list of records."""
        import json
        import time
        recs = []
        done = 0
        self.diagnostics()  # reference density for the first |d rho|_inf
        while done < steps:
            n = min(int(log_every), steps - done)
            self.sync()
            t0 = time.perf_counter()
            self.step(n)
            self.sync()
            dt = time.perf_counter() - t0
            done += n
            d = self.diagnostics()
            rec = {"step": d["step"], "mass": d["mass"], "mom_x": d["mom_x"],
                   "mom_y": d["mom_y"], "max_u": d["max_u"], "dinf": d["dinf"],
                   "nonfinite": d["nonfinite"],
                   "mlups": self.shape[0] * self.shape[1] * n / dt / 1e6}
            recs.append(rec)
            if log is not None:
                log.write(json.dumps(rec) + "\n")
                log.flush()
        return recs

    def selftest_timeout(self, polls=1000):
        """Run the bounded-wait failure check (lbm_selftest_timeout); raises LbmError with
        code LBM_ETIMEOUT when the timeout is detected and reported."""
        self._check(self._L.lbm_selftest_timeout(self._h, int(polls)))

    def selftest_dep_timeout(self, polls=1000):
        """The same check for the persistent kernel's dependency wait
        (lbm_selftest_dep_timeout); raises LbmError with code LBM_ETIMEOUT."""
        self._check(self._L.lbm_selftest_dep_timeout(self._h, int(polls)))

    def moments(self, out=None, dtype=np.float64):
        """rho, ux, uy of Eq. 6 as host arrays of dtype (float64, or float32 for the float
        transfer, lbm_moments_f32).  With out= (a C-contiguous float64 or float32 (ny, nx)
        array, e.g. a pinned buffer) only the density is copied, into out."""
        if out is not None:
            if (out.dtype not in (np.float64, np.float32) or out.shape != self.shape
                    or not out.flags.c_contiguous):
                raise ValueError("out must be a C-contiguous float64 or float32 array of "
                                 "shape %s" % (self.shape,))
            if out.dtype == np.float32:
                self._check(self._L.lbm_moments_f32(self._h, _f(out), None, None))
            else:
                self._check(self._L.lbm_moments(self._h, _d(out), None, None))
            return out
        res = {k: np.empty(self.shape, dtype=dtype) for k in ("rho", "ux", "uy")}
        if np.dtype(dtype) == np.float32:
            self._check(self._L.lbm_moments_f32(self._h, _f(res["rho"]), _f(res["ux"]),
                                                _f(res["uy"])))
        else:
            self._check(self._L.lbm_moments(self._h, _d(res["rho"]), _d(res["ux"]),
                                            _d(res["uy"])))
        return res

    def moments_device(self, rho=None, ux=None, uy=None):
        ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._check(self._L.lbm_moments_device(self._h, ptr(rho), ptr(ux), ptr(uy)))

    def diagnostics(self):
        d = C.lbm_diag()
        self._check(self._L.lbm_diagnostics(self._h, ctypes.byref(d)))
        return _diag_dict(d)

    def diagnostics_noalloc(self, out_dev):
        """Allocation-free diagnostics into caller-owned device memory (6 doubles: mass,
        mom_x, mom_y, max_u, 0, nonfinite); queued on the lattice's stream.  out_dev is a
        device pointer (int) or an object with data_ptr() (e.g. a CUDA tensor)."""
        ptr = out_dev.data_ptr() if hasattr(out_dev, "data_ptr") else int(out_dev)
        self._check(self._L.lbm_diagnostics_noalloc(self._h, ctypes.c_void_p(ptr)))

    def init_droplets(self, drops, params, curvature=False, balanced=False):
        """Droplet field from (n, 3) rows (cx, cy, radius) and a warm.WarmParams
        (lbm_init_droplets; curvature / balanced set LBM_WARM_CURVATURE /
        LBM_WARM_BALANCED)."""
        d = np.ascontiguousarray(drops, dtype=np.float64)
        if d.ndim != 2 or d.shape[1] != 3:
            raise ValueError("drops must be an (n, 3) array of (cx, cy, radius)")
        arr = (C.lbm_droplet * len(d))(*[C.lbm_droplet(*row) for row in d])
        flags = (C.LBM_WARM_CURVATURE if curvature else 0) | (C.LBM_WARM_BALANCED if balanced
                                                              else 0)
        self._check(self._L.lbm_init_droplets(self._h, arr, len(d), ctypes.byref(params.c()),
                                              flags))

    def phase_stats(self, rho_vap_max, rho_liq_min):
        """(mean vapour density, vapour nodes, mean liquid density, liquid nodes)."""
        out = np.empty(4)
        self._check(self._L.lbm_phase_stats(self._h, float(rho_vap_max), float(rho_liq_min),
                                            _d(out)))
        return out[0], int(out[1]), out[2], int(out[3])

    @property
    def step_count(self):
        return self._L.lbm_step_count(self._h)

    def eval_psi(self, rho):
        r = np.ascontiguousarray(rho, dtype=np.float64).ravel()
        out = np.empty_like(r)
        self._check(self._L.lbm_eval_psi(self._h, _d(r), _d(out), r.size))
        return out.reshape(np.shape(rho))

    def save(self, path):
        self._check(self._L.lbm_save(self._h, str(path).encode()))

    def load(self, path):
        self._check(self._L.lbm_load(self._h, str(path).encode()))

    @property
    def tiling(self):
        """(threads per CTA, columns per thread, rows per CTA sweep) of the step kernel."""
        t, v, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._L.lbm_get_tiling(self._h, ctypes.byref(t), ctypes.byref(v),
                                           ctypes.byref(r)))
        return t.value, v.value, r.value

    def set_tiling(self, threads=0, vec=0, rows=0):
        self._check(self._L.lbm_set_tiling(self._h, int(threads), int(vec), int(rows)))

    @property
    def stream(self):
        return self._L.lbm_stream(self._h)

    def autotune(self, steps=20, cache=None):
        """Time the available tilings on a saved copy of the state and keep the fastest;
        returns (threads, vec, rows, ms_per_step)."""
        t, v, r, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self._L.lbm_autotune(self._h, int(steps),
                                         None if cache is None else str(cache).encode(),
                                         ctypes.byref(t), ctypes.byref(v), ctypes.byref(r),
                                         ctypes.byref(ms)))
        return t.value, v.value, r.value, ms.value


@dataclasses.dataclass
class Instance:
    """One member of a Batch (fields as lbm_instance)."""
    nx: int
    ny: int
    eos: Eos
    G: float = -1.0
    sigma: float = 0.0
    s: tuple = (1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0)
    nu_l: float = 0.0
    nu_v: float = 0.0
    visc_mode: str = "const"
    bc: str = "periodic"
    rho_c: float = 0.0
    rho_l: float = 0.0
    rho_v: float = 0.0
    rho_ref: float = -1.0
    layout: str = "auto"  # "auto", "rows" (as given) or "transposed" (lbm_instance.layout)

    def c(self):
        ci = C.lbm_instance()
        ci.nx, ci.ny = int(self.nx), int(self.ny)
        ci.eos = self.eos.c()
        ci.G, ci.sigma = float(self.G), float(self.sigma)
        for i in range(9):
            ci.s[i] = float(self.s[i])
        ci.nu_l, ci.nu_v = float(self.nu_l), float(self.nu_v)
        ci.visc_mode = _VISC[self.visc_mode]
        ci.bc = _BC[self.bc]
        ci.rho_c, ci.rho_l, ci.rho_v = float(self.rho_c), float(self.rho_l), float(self.rho_v)
        ci.rho_ref = float(self.rho_ref)
        ci.layout = _LAYOUT[self.layout]
        return ci


class Batch:
    """Many independent lattices advanced together, one launch per step and kernel width
    (lbm_batch_*)."""

    def __init__(self, instances, precision="fp32", stream=None, tile_threads=0, tile_rows=0,
                 device=None, tile_vec=0):
        self._L = C.lib()
        self.instances = list(instances)
        arr = (C.lbm_instance * len(self.instances))(*[i.c() for i in self.instances])
        h = ctypes.c_void_p()
        sp = _stream_ptr(stream)
        rc = self._L.lbm_batch_create(ctypes.byref(h), len(self.instances), arr,
                                      _PREC[precision], sp, _device_of(stream, device),
                                      int(tile_threads), int(tile_vec), int(tile_rows))
        if rc != 0:
            raise LbmError(rc, self._L.lbm_batch_last_error(None).decode())
        self._h = h
        self.stream_keepalive = stream

    def _check(self, rc):
        if rc < 0:
            raise LbmError(rc, self._L.lbm_batch_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.instances)

    def init_fields(self, i, rho, ux=None, uy=None):
        """As Lattice.init_fields for instance i (float32 arrays: the float transfer)."""
        inst = self.instances[i]
        shp = (inst.ny, inst.nx)
        if getattr(rho, "dtype", None) == np.float32:
            r, u, v = _f32(rho, shp), _f32(ux, shp), _f32(uy, shp)
            self._check(self._L.lbm_batch_init_fields_f32(self._h, int(i), _f(r), _f(u),
                                                          _f(v)))
            return
        r, u, v = _f64(rho, shp), _f64(ux, shp), _f64(uy, shp)
        self._check(self._L.lbm_batch_init_fields(self._h, int(i), _d(r), _d(u), _d(v)))

    def step(self, n=1):
        self._check(self._L.lbm_batch_step(self._h, int(n)))

    def moments(self, i, dtype=np.float64):
        """rho, ux, uy of instance i as host arrays of dtype (float64 or float32)."""
        inst = self.instances[i]
        out = {k: np.empty((inst.ny, inst.nx), dtype=dtype) for k in ("rho", "ux", "uy")}
        if np.dtype(dtype) == np.float32:
            self._check(self._L.lbm_batch_moments_f32(self._h, int(i), _f(out["rho"]),
                                                      _f(out["ux"]), _f(out["uy"])))
        else:
            self._check(self._L.lbm_batch_moments(self._h, int(i), _d(out["rho"]),
                                                  _d(out["ux"]), _d(out["uy"])))
        return out

    def density(self, i):
        """rho of instance i alone (lbm_batch_moments with no velocity outputs)."""
        inst = self.instances[i]
        rho = np.empty((inst.ny, inst.nx))
        self._check(self._L.lbm_batch_moments(self._h, int(i), _d(rho), None, None))
        return rho

    def get_populations(self, i):
        inst = self.instances[i]
        f = np.empty((9, inst.ny, inst.nx))
        self._check(self._L.lbm_batch_get_populations(self._h, int(i), _d(f)))
        return f

    def diagnostics(self):
        arr = (C.lbm_diag * len(self.instances))()
        self._check(self._L.lbm_batch_diagnostics(self._h, arr))
        return [_diag_dict(d) for d in arr]

    def run_to_equilibrium(self, tol, check_every=100, max_steps=100000):
        steps = (ctypes.c_longlong * len(self.instances))()
        left = self._check(self._L.lbm_batch_run_to_equilibrium(
            self._h, float(tol), int(check_every), int(max_steps), steps))
        return left, np.array(steps[:], dtype=np.int64)

    @property
    def active(self):
        return self._check(self._L.lbm_batch_active(self._h))

    @property
    def persistent(self):
        """Whether steps run as persistent launches (lbm_batch_persistent)."""
        return bool(self._check(self._L.lbm_batch_persistent(self._h)))

    def is_transposed(self, i):
        """Whether instance i is stored with its axes exchanged
        (lbm_batch_instance_transposed; Instance.layout)."""
        return bool(self._check(self._L.lbm_batch_instance_transposed(self._h, int(i))))

    def is_active(self, i):
        """Whether instance i is still being stepped (lbm_batch_instance_active)."""
        return bool(self._check(self._L.lbm_batch_instance_active(self._h, int(i))))

    def retire(self, i):
        """Stop stepping instance i (lbm_batch_retire)."""
        self._check(self._L.lbm_batch_retire(self._h, int(i)))

    def retire_nonfinite(self):
        """Retire every active instance with a non-finite or non-positive density
        (lbm_batch_retire_nonfinite); returns the indices retired."""
        flags = (ctypes.c_int * len(self.instances))()
        self._check(self._L.lbm_batch_retire_nonfinite(self._h, flags))
        return [i for i in range(len(self.instances)) if flags[i]]

    def autotune(self, steps=20, cache=None):
        """As Lattice.autotune, for all active instances together."""
        t, v, r, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self._L.lbm_batch_autotune(self._h, int(steps),
                                               None if cache is None else str(cache).encode(),
                                               ctypes.byref(t), ctypes.byref(v),
                                               ctypes.byref(r), ctypes.byref(ms)))
        return t.value, v.value, r.value, ms.value

    @property
    def tiling(self):
        """(threads per CTA or TILE_PER_INSTANCE, columns per thread, rows per sweep)."""
        t, v, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._L.lbm_batch_get_tiling(self._h, ctypes.byref(t), ctypes.byref(v),
                                                 ctypes.byref(r)))
        return t.value, v.value, r.value

    def check_guards(self):
        """lbm_batch_check_guards (see Lattice.check_guards)."""
        self._check(self._L.lbm_batch_check_guards(self._h))

    @property
    def launches_per_step(self):
        """Step-kernel launches per step: one per launch group (kernel width and kind of
        strip), or 1 when the batch steps persistently (one launch per run of up to 64
        steps for all groups)."""
        return self._check(self._L.lbm_batch_launches_per_step(self._h))
