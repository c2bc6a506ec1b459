"""ctypes binding of libcool (include/cool.h), same entry-point names.

Argument marshalling only: every computation runs in the CUDA library.
Torch is used for device memory and the current stream.  If libcool.so is
missing or fails to load, every call raises: there is no CPU fallback.
"""
import ctypes as C
import dataclasses
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcool.so")

COOL_OK, COOL_EINVAL, COOL_ENULL, COOL_EALIGN, COOL_ECUDA, COOL_ENOMEM, COOL_ESTATE, \
    COOL_EUNSUPPORTED, COOL_EIO = range(9)
COOL_F32, COOL_BF16, COOL_F16, COOL_F64 = range(4)
COOL_EXPLICIT_LIMITED, COOL_IMPLICIT_STIFF = 0, 1
COOL_PATH_L2WINDOW, COOL_PATH_TMA_SMEM, COOL_PATH_TEXTURE_POINT, COOL_PATH_TEXTURE_HWLERP, \
    COOL_PATH_SURROGATE, COOL_PATH_QTOTAL = range(6)

# Every entry point declared in include/cool.h (checked by the CPU tests).
EXPORTS = (
    "cool_strerror", "cool_last_cuda_error", "cool_table_spec_default", "cool_params_default",
    "cool_build_table", "cool_table_free", "cool_table_l2_persist", "cool_table_get_spec", "cool_table_export",
    "cool_table_nodes", "cool_table_save", "cool_table_load", "cool_step", "cool_debug_lookup",
    "cool_build_channels_noalloc", "cool_table_packed_bytes", "cool_table_export_packed", "cool_step_bwd",
    "cool_step_fwd_jac", "cool_step_bwd_jac",
    "cool_debug_gemm_bf16", "cool_debug_wait_timeout", "cool_fit_spec_default", "cool_surrogate_fit",
    "cool_surrogate_free",
    "cool_surrogate_info", "cool_surrogate_get_params", "cool_surrogate_set_params", "cool_surrogate_grads",
    "cool_surrogate_eval", "cool_surrogate_mask", "cool_surrogate_set_mask", "cool_surrogate_infer",
    "cool_step_direct", "cool_step_host", "cool_radiation_te", "cool_step_disk", "cool_tma_error",
    "cool_release_scratch",
)


class cool_table_spec(C.Structure):
    _fields_ = [("n_H", C.c_int), ("n_B", C.c_int), ("n_ne", C.c_int), ("n_Te", C.c_int),
                ("n_Tc", C.c_int),
                ("H_min", C.c_double), ("H_max", C.c_double), ("B_min", C.c_double),
                ("B_max", C.c_double), ("ne_min", C.c_double), ("ne_max", C.c_double),
                ("T_min", C.c_double), ("T_max", C.c_double),
                ("dtype", C.c_int), ("row_scaled", C.c_int), ("k2_switch_T", C.c_double),
                ("lnLambda", C.c_double), ("theta_i_uses_mp", C.c_int),
                ("compton_literal", C.c_int)]


class cool_params(C.Structure):
    _fields_ = [("rho_scale", C.c_double), ("M_bh_msun", C.c_double), ("gamma_e", C.c_double),
                ("gamma_i", C.c_double), ("dt", C.c_double), ("n_sub", C.c_int), ("mode", C.c_int),
                ("limiter_frac", C.c_double), ("eq_band", C.c_double),
                ("coulomb_clamp", C.c_double), ("implicit_iters", C.c_int), ("path", C.c_int),
                ("fp64_critical", C.c_int)]


class cool_fit_spec(C.Structure):
    _fields_ = [("channel", C.c_int), ("n_samples", C.c_longlong), ("batch", C.c_int), ("epochs", C.c_int),
                ("lr", C.c_double), ("lr_final", C.c_double), ("seed", C.c_ulonglong),
                ("fallback_tol", C.c_double)]


class cool_surrogate_stats(C.Structure):
    _fields_ = [("final_loss", C.c_double), ("steps", C.c_longlong), ("mask_cells", C.c_longlong),
                ("fallback_cells", C.c_longlong), ("param_bytes_bf16", C.c_longlong), ("mean", C.c_double),
                ("std", C.c_double), ("x_switch", C.c_double)]


class cool_counters(C.Structure):
    _fields_ = [(n, C.c_ulonglong) for n in ("n_clamped", "n_nonfinite", "n_stiff",
                                              "n_fp64_coulomb", "n_implicit_fail", "n_fallback", "n_floor",
                                              "n_exact_redo")]


class cool_disk(C.Structure):
    _fields_ = [("spin", C.c_double), ("h_floor", C.c_double), ("h_from_state", C.c_int)]


class CoolError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib_or_none_strerror(status)
        extra = ""
        if status == COOL_ECUDA and _LIB is not None:
            extra = f" (cudaError {_LIB.cool_last_cuda_error()})"
        super().__init__(f"{where}: {msg}{extra}")
        self.status = status


_LIB = None


def _lib_or_none_strerror(status):
    if _LIB is None:
        return f"status {status}"
    return _LIB.cool_strerror(status).decode()


def lib():
    """Load libcool.so (raises if it is missing: no fallback path exists)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcool.so not built at {LIB_PATH}; run "
                               "`python -m paper_2505_08855_b300.build`")
        L = C.CDLL(LIB_PATH)
        P, I, LL, D = C.c_void_p, C.c_int, C.c_longlong, C.c_double
        sig = {
            "cool_strerror": (C.c_char_p, [I]),
            "cool_last_cuda_error": (I, []),
            "cool_table_spec_default": (I, [P]),
            "cool_params_default": (I, [P]),
            "cool_build_table": (I, [P, P, P]),
            "cool_table_free": (I, [P]),
            "cool_table_l2_persist": (I, [P, I]),
            "cool_table_get_spec": (I, [P, P]),
            "cool_table_export": (I, [P, I, P, LL]),
            "cool_table_nodes": (I, [P, I, P, I]),
            "cool_table_save": (I, [P, C.c_char_p]),
            "cool_table_load": (I, [C.c_char_p, P, P]),
            "cool_step": (I, [P, P, LL, I, P, P, P, P, P, P, P, P, P, P, P]),
            "cool_debug_lookup": (I, [P, I, LL, P, P, P, P]),
            "cool_build_channels_noalloc": (I, [P, P, P, P, P]),
            "cool_table_packed_bytes": (I, [P, P]),
            "cool_step_bwd": (I, [P, P, LL] + [P] * 15 + [P]),
            "cool_step_fwd_jac": (I, [P, P, LL] + [P] * 8 + [P]),
            "cool_step_bwd_jac": (I, [LL] + [P] * 8 + [P]),
            "cool_debug_gemm_bf16": (I, [P, P, P, I, I, I, P, P]),
            "cool_debug_wait_timeout": (I, [I, P, P]),
            "cool_fit_spec_default": (I, [P]),
            "cool_surrogate_fit": (I, [P, P, P, P]),
            "cool_surrogate_free": (I, [P]),
            "cool_surrogate_info": (I, [P, P]),
            "cool_surrogate_get_params": (I, [P, P, I]),
            "cool_surrogate_set_params": (I, [P, P, I]),
            "cool_surrogate_grads": (I, [P, LL, P, P, P, P, P]),
            "cool_surrogate_eval": (I, [P, LL, P, P, P]),
            "cool_surrogate_mask": (I, [P, P, LL]),
            "cool_surrogate_set_mask": (I, [P, P, LL]),
            "cool_step_direct": (I, [P, P, LL, P, P, P, P, P, P, P, P, P, P, P]),
            "cool_step_host": (I, [P, P, LL, P, P, P, P, P, P, P, LL, P, P]),
            "cool_radiation_te": (I, [P, D, D, LL, P, P, P, P, P, P]),
            "cool_step_disk": (I, [P, P, P, LL, P, P, P, P, P, P, P, P, P, P, P, P]),
            "cool_surrogate_infer": (I, [P, P, P, LL, P, P, P, P, P, P, P, P, P, P, P]),
            "cool_table_export_packed": (I, [P, P, LL]),
            "cool_tma_error": (I, [P, I]),
            "cool_release_scratch": (I, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(status, where):
    if status != COOL_OK:
        raise CoolError(status, where)


def ref(x):
    return C.cast(C.pointer(x), C.c_void_p)
