"""ctypes declarations of the C ABI in include/lhv.h (argument marshalling only)."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblhv.so")

LHV_OK, LHV_EINVAL, LHV_ENOMEM, LHV_ECUDA, LHV_ETIMEOUT, LHV_ENONFINITE, LHV_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
LHV_FP32, LHV_FP64, LHV_TF32X3 = 0, 1, 2
LHV_TERMS_NEAR, LHV_TERMS_FAR, LHV_TERMS_ALL = 1, 2, 3
LHV_FORM_PHI_CHI, LHV_FORM_PSI, LHV_FORM_RCR = 0, 1, 2
LHV_MAX_LEVELS = 22
LHV_NUM_STAGES = 12
STAGES = ["tree", "p2m", "m2m", "m2l", "l2l", "l2p", "p2p", "rk4", "ops", "copy", "m2l_products", "select"]
EXPORT = {"keys": 1, "perm": 2, "box_keys": 3, "box_range": 4, "colleagues": 5,
          "multipole": 6, "local": 7, "cube": 8}


class Config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("leaf_max", ctypes.c_int), ("core_a", ctypes.c_double),
                ("eps", ctypes.c_double), ("precision", ctypes.c_int), ("terms", ctypes.c_int),
                ("max_level", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("leaf_level", ctypes.c_int), ("nbox", ctypes.c_int * LHV_MAX_LEVELS), ("n", ctypes.c_int64),
                ("p2p_pairs", ctypes.c_int64), ("m2l_pairs", ctypes.c_int64),
                ("stage_ms", ctypes.c_double * LHV_NUM_STAGES),
                ("stage_launches", ctypes.c_int64 * LHV_NUM_STAGES), ("kernel_launches", ctypes.c_int64),
                ("level_p", ctypes.c_int * LHV_MAX_LEVELS), ("selector_leaf_max", ctypes.c_int),
                ("selector_selections", ctypes.c_int64), ("selector_checks", ctypes.c_int64),
                ("selector_fallbacks", ctypes.c_int64), ("selector_err_v", ctypes.c_double),
                ("selector_err_s", ctypes.c_double), ("tuned_p2p_targets_per_thread", ctypes.c_int),
                ("tuned_p2p_sources_per_stage", ctypes.c_int),
                ("tuned_m2l_pairs_per_chunk", ctypes.c_int), ("tuned_m2l_tensor_cores", ctypes.c_int),
                ("tune_ms", ctypes.c_double * 12), ("graph_captures", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("graph_fallbacks", ctypes.c_int64),
                ("graph_kernels", ctypes.c_int64)]


# exported function -> (restype, argtypes); every name here is declared in include/lhv.h
_vp, _i64, _dbl, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
SIGNATURES = {
    "lhv_create": (_int, [ctypes.POINTER(Config), _vp, ctypes.POINTER(_vp)]),
    "lhv_destroy": (None, [_vp]),
    "lhv_status_string": (ctypes.c_char_p, [_int]),
    "lhv_last_error": (ctypes.c_char_p, [_vp]),
    "lhv_build_tree": (_int, [_vp, _i64, _vp]),
    "lhv_evaluate_velocity_stretching": (_int, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "lhv_step": (_int, [_vp, _i64, _vp, _vp, _dbl]),
    "lhv_step_host": (_int, [_vp, _i64, _vp, _vp, _dbl]),
    "lhv_evaluate_velocity_stretching_f64": (_int, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "lhv_step_f64": (_int, [_vp, _i64, _vp, _vp, _dbl]),
    "lhv_get_stats": (_int, [_vp, ctypes.POINTER(Stats)]),
    "lhv_set_level_p": (_int, [_vp, ctypes.POINTER(_int), _int]),
    "lhv_autotune": (_int, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "lhv_autotune_batched": (_int, [_vp, _int, ctypes.POINTER(_i64), _vp, _vp, _vp, _vp]),
    "lhv_set_launch_shape": (_int, [_vp, _int, _int, _int, _int]),
    "lhv_set_selector": (_int, [_vp, _vp, _vp, _dbl, _int, _int]),
    "lhv_selector_features": (_int, [_vp, _i64, _vp, _vp, _dbl, _vp, _int, ctypes.POINTER(_int)]),
    "lhv_mlp_forward": (_int, [_int, _vp, _vp, _vp, _vp, _vp]),
    "lhv_mlp_loss_grad": (_int, [_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lhv_mlp_adam": (_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _int, ctypes.c_float, _vp]),
    "lhv_direct_sampled": (_int, [_vp, _i64, _vp, _vp, _int, _vp, _vp, _vp]),
    "lhv_direct_sampled_f64": (_int, [_vp, _i64, _vp, _vp, _int, _vp, _vp, _vp]),
    "lhv_set_timing": (_int, [_vp, _int]),
    "lhv_reset_stats": (_int, [_vp]),
    "lhv_export": (_int, [_vp, _int, _int, _vp, _i64, ctypes.POINTER(_i64)]),
    "lhv_tc_selftest": (_int, [_vp, _vp, _vp, _int, _int]),
    "lhv_evaluate_batched": (_int, [_vp, _int, ctypes.POINTER(_i64), _vp, _vp, _vp, _vp]),
    "lhv_step_batched": (_int, [_vp, _int, ctypes.POINTER(_i64), _vp, _vp, _dbl]),
    "lhv_morton_sort_noalloc": (_int, [_i64, _vp, _vp, _vp, _vp, _vp]),
    "lhv_evaluate_potential_gradient": (_int, [_vp, _i64, _vp, _vp, _vp]),
    "lhv_evaluate_potential_gradient_f64": (_int, [_vp, _i64, _vp, _vp, _vp]),
    "lhv_set_form": (_int, [_vp, _int]),
    "lhv_set_graph": (_int, [_vp, _int]),
    "lhv_evaluate_filaments": (_int, [_vp, _int, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int32), _vp, _vp, _vp]),
    "lhv_evaluate_filaments_f64": (_int, [_vp, _int, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int32), _vp, _vp,
                                          _vp]),
    "lhv_peak_probe": (_int, [_int, _int, _int, _vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]),
}

NOALLOC_MAX_N = 1 << 20  # LHV_NOALLOC_MAX_N
PEAK = {"ffma": 1, "ffma2": 2, "mufu": 3, "tf32_mma": 4, "bf16_mma": 5}  # LHV_PEAK_*
MLP_IN, MLP_OUT, MLP_NP, MLP_NW, MLP_NB = 12, 21, 17, 10304, 213  # LHV_MLP_*

_lib = None


def load(path=LIB_PATH):
    """Load liblhv.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1201_5430_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LHVError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status
