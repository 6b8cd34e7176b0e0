"""ctypes declarations of the C-ABI in include/mmncg.h (argument marshalling
only: every step of the computation runs in the CUDA library)."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmmncg.so")

MM_OK = 0
MM_NOT_CONVERGED = 1
MM_STALLED = 2
MM_ERR_ARG = -1
MM_ERR_MESH = -2
MM_ERR_OOM = -3
MM_ERR_CUDA = -4
MM_ERR_NONFINITE = -5
MM_ERR_DEVICE_TIMEOUT = -6
MM_ERR_STATE = -7

MM_OP_DIV = 0
MM_OP_DIVT = 1
MM_OP_LOCAL = 2

STATUS_NAMES = {0: "ok", 1: "not_converged", 2: "stalled", -1: "err_arg", -2: "err_mesh",
                -3: "err_oom", -4: "err_cuda", -5: "err_nonfinite", -6: "err_device_timeout",
                -7: "err_state"}


class mm_material(C.Structure):
    _fields_ = [("Ms", C.c_double), ("A", C.c_double), ("K1", C.c_double), ("axis", C.c_double * 3)]


class mm_options(C.Structure):
    _fields_ = [("device", C.c_int), ("blocks_per_sm", C.c_int), ("stream", C.c_void_p)]


class mm_params(C.Structure):
    _fields_ = [("tau_F", C.c_double), ("jmax", C.c_int), ("max_iter", C.c_int),
                ("theta_max", C.c_double), ("c1", C.c_double), ("max_backtrack", C.c_int),
                ("keep_last_term", C.c_int), ("poisson_tol", C.c_double),
                ("poisson_max_iter", C.c_int), ("precision", C.c_int), ("inner_tol", C.c_double),
                ("max_refine", C.c_int), ("amg", C.c_int), ("beta_rule", C.c_int),
                ("poisson_sched", C.c_int), ("poisson_tol_max", C.c_double)]


class mm_stats(C.Structure):
    _fields_ = [("evals", C.c_int64), ("nli", C.c_int64), ("li", C.c_int64), ("mi", C.c_int64),
                ("ls_extra", C.c_int64), ("mr", C.c_int64), ("status", C.c_int32), ("pad", C.c_int32),
                ("F", C.c_double), ("terms", C.c_double * 4), ("F_internal", C.c_double),
                ("M", C.c_double * 3), ("li2", C.c_int64), ("li2_first", C.c_int64),
                ("restarts", C.c_int64), ("steepest", C.c_int64)]


EXPORTS = {
    # name: (restype, argtypes)
    "mm_default_params": (None, [C.POINTER(mm_params)]),
    "mm_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(mm_options)]),
    "mm_destroy": (None, [C.c_void_p]),
    "mm_last_error": (C.c_char_p, [C.c_void_p]),
    "mm_upload_mesh": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_void_p, C.c_int32, C.POINTER(mm_material)]),
    "mm_sizes": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int64)] * 4),
    "mm_amg_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                              C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int32]),
    "mm_k32_host_apply": (C.c_int, [C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mm_amg_host_apply": (C.c_int, [C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                    C.c_int32]),
    "mm_set_magnetization": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mm_get_magnetization": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mm_set_magnetization_dev": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mm_get_magnetization_dev": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mm_set_field": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mm_set_tiles": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "mm_k32_layout_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64)]),
    "mm_minimize": (C.c_int, [C.c_void_p, C.POINTER(mm_params), C.POINTER(mm_stats)]),
    "mm_minimize_async": (C.c_int, [C.c_void_p, C.POINTER(mm_params)]),
    "mm_get_stats": (C.c_int, [C.c_void_p, C.POINTER(mm_stats)]),
    "mm_energy": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(mm_params), C.POINTER(C.c_double),
                            C.POINTER(C.c_double)]),
    "mm_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(mm_params), C.c_void_p, C.c_int]),
    "mm_get_potential": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mm_precond_solve": (C.c_int, [C.c_void_p, C.POINTER(mm_params), C.c_void_p,
                                   C.POINTER(C.c_int64)]),
    "mm_hessian_apply": (C.c_int, [C.c_void_p, C.POINTER(mm_params), C.c_void_p, C.c_void_p]),
    "mm_potential_matvec": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mm_demag_curve": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(mm_params),
                                 C.POINTER(mm_stats)]),
    "mm_autotune_jmax": (C.c_int, [C.c_void_p, C.POINTER(mm_params), C.c_int64, C.c_void_p, C.c_void_p,
                                   C.c_int32, C.POINTER(C.c_int32), C.c_void_p]),
    "mm_last_kernel_ms": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mm_batch_plan": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.c_int, C.c_double,
                                C.POINTER(C.c_int32)]),
    "mm_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]),
    "mm_batch_destroy": (None, [C.c_void_p]),
    "mm_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "mm_batch_config": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "mm_batch_set_tiles": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "mm_batch_get_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                      C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mm_batch_minimize": (C.c_int, [C.c_void_p, C.POINTER(mm_params), C.POINTER(mm_stats)]),
    "mm_batch_demag_curve": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(mm_params),
                                       C.POINTER(mm_stats)]),
    "mm_batch_autotune": (C.c_int, [C.c_void_p, C.POINTER(mm_params), C.POINTER(C.c_int),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mm_batch_last_ms": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mm_mlp_param_count": (C.c_int64, []),
    "mm_mlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_uint64]),
    "mm_mlp_destroy": (None, [C.c_void_p]),
    "mm_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "mm_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "mm_mlp_set_input_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mm_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mm_mlp_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                  C.POINTER(C.c_float)]),
    "mm_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                    C.POINTER(C.c_float)]),
    "mm_mlp_set_tensor_path": (C.c_int, [C.c_void_p, C.c_int]),
    "mm_mlp_fit_input_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "mm_mlp_get_input_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mm_mlp_fit_target_scales": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                           C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mm_warmstart_targets": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                       C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mm_warmstart_features": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "mm_warmstart_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_double,
                                     C.c_double, C.c_double]),
    "mm_energy_gradient_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(mm_params),
                                             C.c_void_p, C.c_int, C.c_void_p]),
    "mm_operator_apply": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "mm_coercive_field": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int32)]),
    "mm_stream": (C.c_void_p, [C.c_void_p]),
}

_lib = None


def load():
    """Load libmmncg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "or python paper_1801_03690_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
