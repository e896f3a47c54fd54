"""ctypes declarations of the C ABI in include/*.h (argument marshalling only)."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm_gb300.so")
# the bounds-check build (kernels compiled with -DLBM_BOUNDS_CHECK), selected by
# LBM_LIBRARY=check in the environment
CHECK_LIB_PATH = os.path.join(HERE, "liblbm_gb300_check.so")

c_int, c_double, c_void_p, c_size_t, c_longlong = (ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_void_p, ctypes.c_size_t,
                                                   ctypes.c_longlong)
dptr = ctypes.POINTER(ctypes.c_double)
llptr = ctypes.POINTER(ctypes.c_longlong)

(LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE, LBM_EIO,
 LBM_ECORRUPT) = (0, -1, -2, -3, -4, -5, -6, -7, -8)
LBM_FP64, LBM_FP32_DEV = 0, 1
LBM_VISC_CONST, LBM_VISC_STEP, LBM_VISC_LINEAR = 0, 1, 2
LBM_BC_PERIODIC, LBM_BC_WALLS_Y = 0, 1
LBM_LAYOUT_AUTO, LBM_LAYOUT_ROWS, LBM_LAYOUT_TRANSPOSED = 0, 1, 2
LBM_TILE_PER_INSTANCE = -1


class lbm_eos(ctypes.Structure):
    _fields_ = [("a", c_double), ("b", c_double), ("R", c_double), ("T", c_double)]


class lbm_options(ctypes.Structure):
    _fields_ = [("precision", c_int), ("visc_mode", c_int), ("bc", c_int), ("psi_fp64", c_int),
                ("rho_ref", c_double), ("rho_c", c_double), ("rho_l", c_double),
                ("rho_v", c_double), ("stream", c_void_p), ("device", c_int),
                ("tile_threads", c_int), ("tile_vec", c_int), ("tile_rows", c_int)]


class lbm_diag(ctypes.Structure):
    _fields_ = [("mass", c_double), ("mom_x", c_double), ("mom_y", c_double),
                ("max_u", c_double), ("dinf", c_double), ("step", c_longlong),
                ("nonfinite", c_longlong)]


class lbm_instance(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("eos", lbm_eos), ("G", c_double),
                ("sigma", c_double), ("s", c_double * 9), ("nu_l", c_double),
                ("nu_v", c_double), ("visc_mode", c_int), ("bc", c_int), ("rho_c", c_double),
                ("rho_l", c_double), ("rho_v", c_double), ("rho_ref", c_double),
                ("layout", c_int)]


class lbm_adam(ctypes.Structure):
    _fields_ = [("lr", c_double), ("beta1", c_double), ("beta2", c_double), ("eps", c_double)]


class lbm_warm_params(ctypes.Structure):
    _fields_ = [("rho_l", c_double), ("rho_v", c_double), ("width", c_double),
                ("shift", c_double), ("curvature", c_double)]


class lbm_droplet(ctypes.Structure):
    _fields_ = [("cx", c_double), ("cy", c_double), ("radius", c_double)]


LBM_WARM_CURVATURE = 1
LBM_WARM_BALANCED = 2
fptr = ctypes.POINTER(ctypes.c_float)
LBM_MLP_NPARAMS = 4805

# name -> (restype, argtypes); every symbol include/*.h declares.
SIGNATURES = {
    "lbm_options_default": (None, [ctypes.POINTER(lbm_options)]),
    "lbm_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, lbm_eos, c_double, c_double,
                           dptr, c_double, c_double, ctypes.POINTER(lbm_options)]),
    "lbm_destroy": (None, [c_void_p]),
    "lbm_last_error": (ctypes.c_char_p, [c_void_p]),
    "lbm_init_fields": (c_int, [c_void_p, dptr, dptr, dptr]),
    "lbm_init_fields_device": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_set_populations": (c_int, [c_void_p, dptr]),
    "lbm_get_populations": (c_int, [c_void_p, dptr]),
    "lbm_step": (c_int, [c_void_p, c_int]),
    "lbm_sync": (c_int, [c_void_p]),
    "lbm_selftest_timeout": (c_int, [c_void_p, c_longlong]),
    "lbm_pressure_tensor": (c_int, [c_void_p, dptr, dptr, dptr, c_int]),
    "lbm_moments": (c_int, [c_void_p, dptr, dptr, dptr]),
    "lbm_moments_device": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_diagnostics": (c_int, [c_void_p, ctypes.POINTER(lbm_diag)]),
    "lbm_diagnostics_noalloc": (c_int, [c_void_p, c_void_p]),
    "lbm_step_count": (c_longlong, [c_void_p]),
    "lbm_eval_psi": (c_int, [c_void_p, dptr, dptr, c_size_t]),
    "lbm_save": (c_int, [c_void_p, ctypes.c_char_p]),
    "lbm_load": (c_int, [c_void_p, ctypes.c_char_p]),
    "lbm_get_tiling": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                               ctypes.POINTER(c_int)]),
    "lbm_set_tiling": (c_int, [c_void_p, c_int, c_int, c_int]),
    "lbm_stream": (c_void_p, [c_void_p]),
    "lbm_autotune": (c_int, [c_void_p, c_int, ctypes.c_char_p, ctypes.POINTER(c_int),
                             ctypes.POINTER(c_int), ctypes.POINTER(c_int), dptr]),
    "lbm_maxwell": (c_int, [lbm_eos, dptr, dptr]),
    "lbm_eos_psi2": (c_int, [lbm_eos, c_double, c_double, dptr]),
    "lbm_mechanical_stability": (c_int, [lbm_eos, c_double, c_double, dptr, dptr]),
    "lbm_sigma_consistent": (c_int, [lbm_eos, c_double, dptr]),
    "lbm_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(lbm_instance),
                                 c_int, c_void_p, c_int, c_int, c_int, c_int]),
    "lbm_batch_destroy": (None, [c_void_p]),
    "lbm_batch_last_error": (ctypes.c_char_p, [c_void_p]),
    "lbm_batch_init_fields": (c_int, [c_void_p, c_int, dptr, dptr, dptr]),
    "lbm_batch_step": (c_int, [c_void_p, c_int]),
    "lbm_batch_moments": (c_int, [c_void_p, c_int, dptr, dptr, dptr]),
    "lbm_batch_get_populations": (c_int, [c_void_p, c_int, dptr]),
    "lbm_batch_diagnostics": (c_int, [c_void_p, ctypes.POINTER(lbm_diag)]),
    "lbm_batch_run_to_equilibrium": (c_int, [c_void_p, c_double, c_int, c_longlong, llptr]),
    "lbm_batch_active": (c_int, [c_void_p]),
    "lbm_batch_instance_active": (c_int, [c_void_p, c_int]),
    "lbm_batch_instance_transposed": (c_int, [c_void_p, c_int]),
    "lbm_init_fields_async": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_persistent": (c_int, [c_void_p]),
    "lbm_debug_persist_plan": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int, c_int,
                                       c_void_p, c_void_p, c_void_p]),
    "lbm_selftest_dep_timeout": (c_int, [c_void_p, c_int]),
    "lbm_batch_persistent": (c_int, [c_void_p]),
    "lbm_moments_async": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lbm_batch_retire": (c_int, [c_void_p, c_int]),
    "lbm_batch_retire_nonfinite": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_autotune": (c_int, [c_void_p, c_int, ctypes.c_char_p, ctypes.POINTER(c_int),
                                   ctypes.POINTER(c_int), ctypes.POINTER(c_int), dptr]),
    "lbm_batch_get_tiling": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                     ctypes.POINTER(c_int)]),
    "lbm_batch_launches_per_step": (c_int, [c_void_p]),
    "lbm_init_fields_f32": (c_int, [c_void_p, fptr, fptr, fptr]),
    "lbm_moments_f32": (c_int, [c_void_p, fptr, fptr, fptr]),
    "lbm_batch_init_fields_f32": (c_int, [c_void_p, c_int, fptr, fptr, fptr]),
    "lbm_batch_moments_f32": (c_int, [c_void_p, c_int, fptr, fptr, fptr]),
    "lbm_check_guards": (c_int, [c_void_p]),
    "lbm_bounds_checked": (c_int, []),
    "lbm_batch_check_guards": (c_int, [c_void_p]),
    "lbm_debug_fail_alloc": (c_int, [c_int]),
    "lbm_debug_live_allocs": (ctypes.c_longlong, []),
    "lbm_debug_corrupt_guard": (c_int, [c_void_p, c_int]),
    # include/lbm_mlp.h
    "lbm_mlp_create": (c_int, [ctypes.POINTER(c_void_p), fptr, c_int, c_void_p, c_int]),
    "lbm_mlp_destroy": (None, [c_void_p]),
    "lbm_mlp_last_error": (ctypes.c_char_p, [c_void_p]),
    "lbm_mlp_set_scaling": (c_int, [c_void_p, dptr, dptr, dptr, dptr]),
    "lbm_mlp_fit_scaling": (c_int, [c_void_p, dptr, dptr, c_int]),
    "lbm_mlp_set_data": (c_int, [c_void_p, dptr, dptr, c_int]),
    "lbm_mlp_train": (c_int, [c_void_p, c_int, ctypes.POINTER(lbm_adam), fptr]),
    "lbm_mlp_gradient": (c_int, [c_void_p, fptr, fptr]),
    "lbm_mlp_predict": (c_int, [c_void_p, dptr, c_int, dptr]),
    "lbm_mlp_get_params": (c_int, [c_void_p, c_int, fptr]),
    "lbm_mlp_set_params": (c_int, [c_void_p, c_int, fptr]),
    "lbm_mlp_update_count": (c_longlong, [c_void_p]),
    # include/lbm_warm.h
    "lbm_measure_film": (c_int, [dptr, c_int, c_int, ctypes.POINTER(lbm_warm_params)]),
    "lbm_measure_droplet": (c_int, [dptr, c_int, c_int, lbm_eos, dptr, dptr, dptr, dptr]),
    "lbm_warm_encode": (c_int, [lbm_eos, ctypes.POINTER(lbm_warm_params), dptr]),
    "lbm_warm_decode": (c_int, [lbm_eos, dptr, ctypes.POINTER(lbm_warm_params)]),
    "lbm_vapour_law": (c_int, [c_double, c_double, c_double, c_double, dptr, dptr]),
    "lbm_curved_densities": (c_int, [lbm_eos, ctypes.POINTER(lbm_warm_params), c_double, dptr,
                                     dptr]),
    "lbm_init_droplets": (c_int, [c_void_p, ctypes.POINTER(lbm_droplet), c_int,
                                  ctypes.POINTER(lbm_warm_params), c_int]),
    "lbm_phase_stats": (c_int, [c_void_p, c_double, c_double, dptr]),
}

_LIB = None


def load(path: str = None):
    """Load the library (no build, no fallback: a missing library is an error).  The
    default is the normal build, or the bounds-check build when LBM_LIBRARY=check."""
    global _LIB
    if path is None:
        path = CHECK_LIB_PATH if os.environ.get("LBM_LIBRARY") == "check" else LIB_PATH
    if _LIB is None:
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing; run __graft_entry__.build() or "
                               "python -m paper_1211_6932_gb300.build" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def lib():
    return load()
