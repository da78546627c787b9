"""ctypes declarations of include/hyb.h: the structures and entry points with the
same names as the C ABI.  Argument marshalling only -- every step of the
hybrid fluid-kinetic time step runs in the CUDA library libhyb.so.

The library is built in-tree (``paper_2510_11174_gb300/build.py``); importing
this module raises if it is missing, there is no fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhyb.so")

HYB_OK, HYB_EINVAL, HYB_ENOMEM, HYB_ECUDA, HYB_EOVERFLOW, HYB_ENAN, HYB_ETIMEOUT, HYB_ESTATE = range(8)
STATUS_NAMES = {0: "HYB_OK", 1: "HYB_EINVAL", 2: "HYB_ENOMEM", 3: "HYB_ECUDA", 4: "HYB_EOVERFLOW",
                5: "HYB_ENAN", 6: "HYB_ETIMEOUT", 7: "HYB_ESTATE"}
HYB_BC_PERIODIC, HYB_BC_MUR = 0, 1
HYB_LASER_NONE, HYB_LASER_GAUSS = 0, 1
HYB_LUT_IONIZE = 0
HYB_KIND_MASSIVE, HYB_KIND_PHOTON = 0, 1
HYB_QED_H, HYB_QED_T, HYB_QED_EM_SAMPLE, HYB_QED_PAIR_SAMPLE = 0, 1, 2, 3
HYB_MAX_SPECIES = 8


class hyb_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("dt", C.c_double), ("cfl_frac", C.c_double),
                ("bc", C.c_int * 3), ("lambda_um", C.c_double),
                ("laser_kind", C.c_int),
                ("a0", C.c_double), ("tau_fwhm", C.c_double), ("w0_spot", C.c_double),
                ("t_peak", C.c_double), ("y_c", C.c_double), ("z_c", C.c_double),
                ("x_src", C.c_int), ("pol", C.c_int),
                ("seed", C.c_uint32), ("tile", C.c_int),
                ("stream", C.c_void_p), ("arena_dev", C.c_void_p), ("arena_bytes", C.c_size_t), ("shape_order", C.c_int)]


class hyb_species_desc(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("n", C.c_longlong),
                ("tile_capacity", C.c_longlong), ("ptr_on_device", C.c_int),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("ux", C.c_void_p), ("uy", C.c_void_p), ("uz", C.c_void_p), ("w", C.c_void_p),
                ("zq", C.c_void_p), ("ids", C.c_void_p),
                ("zmax", C.c_int), ("ip_eV", C.c_double * 8), ("l_qn", C.c_int * 8),
                ("ionize_into", C.c_int),
                ("kind", C.c_int), ("qed", C.c_int), ("photon_species", C.c_int),
                ("photon_eps_min", C.c_double), ("pair_electron", C.c_int), ("pair_positron", C.c_int),
                ("pusher", C.c_int)]


class hyb_diag(C.Structure):
    _fields_ = [("step", C.c_longlong), ("time", C.c_double),
                ("w_e", C.c_double), ("w_b", C.c_double),
                ("w_kin", C.c_double * HYB_MAX_SPECIES),
                ("count", C.c_longlong * HYB_MAX_SPECIES),
                ("n_species", C.c_int), ("status", C.c_int),
                ("launches_per_step", C.c_longlong),
                ("w_ionize", C.c_double), ("n_ionize", C.c_longlong),
                ("w_photon_untracked", C.c_double), ("w_pair_deficit", C.c_double),
                ("n_emit", C.c_longlong), ("n_pair", C.c_longlong),
                ("n_fluids", C.c_int), ("w_fluid", C.c_double * 4), ("n_fluid", C.c_double * 4),
                ("n_clamped", C.c_longlong), ("launches_classify", C.c_longlong),
                ("tile_capacity", C.c_longlong * HYB_MAX_SPECIES), ("classified_cells", C.c_longlong),
                ("fluid_cells", C.c_longlong)]


HYB_NPHASE = 10
PHASES = ["push", "j_reduce", "source", "rebin", "field", "fluid", "classify", "regime", "conv_l1", "conv_l2"]
HYB_MAX_FLUIDS = 4


class hyb_fluid_desc(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("ptr_on_device", C.c_int),
                ("n", C.c_void_p), ("ux", C.c_void_p), ("uy", C.c_void_p), ("uz", C.c_void_p),
                ("n_floor", C.c_double), ("temperature_keV", C.c_double), ("gamma_ad", C.c_double),
                ("n_ref", C.c_double)]


class hyb_phase_times_t(C.Structure):
    _fields_ = [("ms", C.c_float * HYB_NPHASE)]


class hyb_regime_desc(C.Structure):
    _fields_ = [("a_thr", C.c_double), ("n_thr", C.c_double), ("c_thr", C.c_double), ("chi_thr", C.c_double),
                ("dilate", C.c_int), ("k_sigma", C.c_double), ("ppc", C.c_int),
                ("to_species", C.c_int * 4), ("policy", C.c_int), ("quiet", C.c_int), ("reach", C.c_int)]


HYB_REGIME_DEFAULT, HYB_REGIME_UNION, HYB_REGIME_ALL_KINETIC = 0, 1, 2


class hyb_model_desc(C.Structure):
    _fields_ = [("dropout", C.c_double), ("mc_passes", C.c_int), ("seed", C.c_uint32),
                ("mean", C.c_float * 6), ("std", C.c_float * 6),
                ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("energy_weight", C.c_double), ("stream", C.c_void_p)]


class hyb_train_stats(C.Structure):
    _fields_ = [("loss", C.c_double), ("bce", C.c_double), ("accuracy", C.c_double), ("step", C.c_longlong)]


class hyb_surrogate_desc(C.Structure):
    _fields_ = [("seed", C.c_uint32), ("dropout", C.c_double), ("mc_passes", C.c_int),
                ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("huber_delta", C.c_double), ("energy_weight", C.c_double),
                ("mean", C.c_float * 10), ("std", C.c_float * 10), ("dstd", C.c_float * 10), ("stream", C.c_void_p)]


class hyb_switchnet_desc(C.Structure):
    _fields_ = [("seed", C.c_uint32), ("dropout", C.c_double), ("mc_passes", C.c_int),
                ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("energy_weight", C.c_double), ("mean", C.c_float * 10), ("std", C.c_float * 10),
                ("stream", C.c_void_p)]


class hyb_surrogate_stats(C.Structure):
    _fields_ = [("loss", C.c_double), ("huber", C.c_double), ("energy", C.c_double), ("step", C.c_longlong)]


_P = C.c_void_p
_ctx = C.c_void_p

# name -> (restype, argtypes)
PROTOTYPES = {
    "hyb_init_grid": (C.c_int, [C.POINTER(hyb_grid_desc), C.POINTER(C.c_void_p)]),
    "hyb_destroy": (None, [_ctx]),
    "hyb_load_species": (C.c_int, [_ctx, C.POINTER(hyb_species_desc), C.POINTER(C.c_int)]),
    "hyb_set_fields": (C.c_int, [_ctx, _P, _P, C.c_int]),
    "hyb_step": (C.c_int, [_ctx, C.c_int]),
    "hyb_diagnostics": (C.c_int, [_ctx, C.POINTER(hyb_diag)]),
    "hyb_get_fields": (C.c_int, [_ctx, _P, _P, _P]),
    "hyb_get_species": (C.c_int, [_ctx, C.c_int, C.c_longlong] + [_P] * 9 + [C.POINTER(C.c_longlong)]),
    "hyb_clear_status": (C.c_int, [_ctx]),
    "hyb_set_auto_grow": (C.c_int, [_ctx, C.c_int]),
    "hyb_get_state": (C.c_int, [_ctx, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "hyb_set_state": (C.c_int, [_ctx, _P, C.c_size_t]),
    "hyb_selftest_wait_timeout": (C.c_int, [_ctx, C.c_longlong]),
    "hyb_last_error": (C.c_char_p, []),
    "hyb_set_profiling": (C.c_int, [_ctx, C.c_int]),
    "hyb_phase_times": (C.c_int, [_ctx, C.POINTER(hyb_phase_times_t)]),
    "hyb_eval_rate_table": (C.c_int, [_ctx, C.c_int, C.c_int, C.c_int, _P, C.c_int, _P]),
    "hyb_eval_qed": (C.c_int, [_ctx, C.c_int, _P, _P, C.c_int, _P]),
    "hyb_load_fluid": (C.c_int, [_ctx, C.c_void_p, C.POINTER(C.c_int)]),
    "hyb_set_regime": (C.c_int, [_ctx, C.POINTER(hyb_regime_desc)]),
    "hyb_classify": (C.c_int, [_ctx, _P, _P, _P, _P]),
    "hyb_get_regime": (C.c_int, [_ctx, _P, _P]),
    "hyb_node_fields": (C.c_int, [_ctx, _P]),
    "hyb_node_state": (C.c_int, [_ctx, _P]),
    "hyb_surrogate_create": (C.c_int, [C.POINTER(hyb_surrogate_desc), C.POINTER(C.c_void_p)]),
    "hyb_surrogate_destroy": (None, [_P]),
    "hyb_surrogate_set_layer": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_surrogate_get_layer": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_surrogate_forward": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P]),
    "hyb_surrogate_mc": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "hyb_surrogate_train_step": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_int,
                                           C.POINTER(hyb_surrogate_stats)]),
    "hyb_surrogate_get_grad": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_switchnet_create": (C.c_int, [C.POINTER(hyb_switchnet_desc), C.POINTER(C.c_void_p)]),
    "hyb_switchnet_destroy": (None, [_P]),
    "hyb_switchnet_set_layer": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_switchnet_get_layer": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_switchnet_get_grad": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_switchnet_forward": (C.c_int, [_P, _P, C.c_longlong, C.c_int, _P]),
    "hyb_switchnet_mc": (C.c_int, [_P, _P, C.c_longlong, _P, _P]),
    "hyb_switchnet_train_step": (C.c_int, [_P, _P, _P, C.c_longlong, C.POINTER(hyb_train_stats)]),
    "hyb_model_create": (C.c_int, [C.POINTER(hyb_model_desc), C.POINTER(C.c_void_p)]),
    "hyb_model_destroy": (None, [_P]),
    "hyb_model_set_layer": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_model_get_layer": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_model_forward": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P]),
    "hyb_train_step": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(hyb_train_stats)]),
    "hyb_model_get_grad": (C.c_int, [_P, C.c_int, _P, _P]),
    "hyb_get_fluid": (C.c_int, [_ctx, C.c_int, _P, _P, _P, _P]),
    "hyb_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _P, C.POINTER(C.c_void_p)]),
    "hyb_batch_step": (C.c_int, [_P, C.c_int]),
    "hyb_batch_destroy": (None, [_P]),
    "hyb_field_energy_noalloc":(C.c_int, [_P, _P, C.c_longlong, C.c_double, C.c_double, C.c_double, _P, _P]),
}

_lib = None


def load():
    """Load libhyb.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhyb.so is not built (run paper_2510_11174_gb300/build.py); "
                               "there is no CPU fallback")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class HybError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


def check(code):
    if code != HYB_OK:
        raise HybError(code, load().hyb_last_error().decode())
    return code
