"""ctypes declarations of the C ABI in include/hdd.h (one Python name per C entry point)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(HERE, "libhdd.so")

STATUS = ["HDD_OK", "HDD_ERR_INVALID_ARG", "HDD_ERR_STATE", "HDD_ERR_OOM", "HDD_ERR_CUDA",
          "HDD_ERR_SINGULAR_COARSE", "HDD_ERR_SINGULAR_LOCAL", "HDD_ERR_NO_CONVERGENCE",
          "HDD_ERR_BREAKDOWN", "HDD_ERR_NONFINITE", "HDD_ERR_TIMEOUT"]

# every entry point declared in include/hdd.h
SYMBOLS = ["hdd_create", "hdd_destroy", "hdd_status_str", "hdd_last_error", "hdd_assemble",
           "hdd_build_rhs", "hdd_apply_A", "hdd_setup_dd", "hdd_get_subdomain",
           "hdd_num_subdomains", "hdd_get_offsets", "hdd_setup_deflation", "hdd_setup_exact",
           "hdd_solve", "hdd_ras_apply", "hdd_local_op", "hdd_profile", "hdd_profile_count",
           "hdd_profile_get", "hdd_launch_count", "hdd_apply_PA_noalloc", "hdd_setup_batch", "hdd_autotune",
           "hdd_warmstart_load", "hdd_warmstart_save",
           "hdd_num_rhs", "hdd_cnn_num_params", "hdd_cnn_set_params", "hdd_cnn_get_params",
           "hdd_cnn_forward", "hdd_cnn_infer", "hdd_cnn_loss_grad", "hdd_cnn_train_step", "hdd_get_outer_vector",
           "hdd_stencil_rows", "hdd_set_option", "hdd_setup_coarse_grid", "hdd_coarse_grid_op",
           "hdd_coarse_grid_size"]


def status_name(code: int) -> str:
    return STATUS[code] if 0 <= code < len(STATUS) else f"HDD_STATUS_{code}"


class HDDError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        self.code = code
        super().__init__(f"{where}: {status_name(code)}" + (f" ({msg})" if msg else ""))


class AssembleParams(C.Structure):
    _fields_ = [("k", C.c_double), ("N", C.c_int), ("diag", C.c_int), ("bc", C.c_int)]


class DDParams(C.Structure):
    _fields_ = [("Sx", C.c_int), ("Sy", C.c_int), ("overlap", C.c_int),
                ("ifx", C.POINTER(C.c_int)), ("ify", C.POINTER(C.c_int))]


class SolveParams(C.Structure):
    _fields_ = [("outer_tol", C.c_double), ("outer_restart", C.c_int), ("outer_maxit", C.c_int),
                ("inner_tol", C.c_double), ("inner_restart", C.c_int), ("inner_maxit", C.c_int),
                ("inner_prec", C.c_int), ("warm_start", C.c_int), ("outer_reorth32", C.c_int),
                ("two_level", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("outer_its", C.c_int), ("status", C.c_int), ("rel_res_true", C.c_double),
                ("inner_its_total", C.c_longlong), ("inner_its_avg", C.c_double),
                ("inner_its_max", C.c_int), ("inner_maxit_hits", C.c_longlong),
                ("t_solve_ms", C.c_double), ("n_history", C.c_int),
                ("res_history", C.POINTER(C.c_double)), ("outer_reorth_fp64", C.c_longlong)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_longlong), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double), ("bound", C.c_int)]


_lib = None


def lib(build_if_missing: bool = True):
    """Load libhdd.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {lib_path} is not built")
        from . import build as _b
        _b.build()
    L = C.CDLL(lib_path)
    P, I, D, V = C.c_void_p, C.c_int, C.c_double, C.c_void_p
    L.hdd_create.argtypes = [C.POINTER(P), I]
    L.hdd_create.restype = I
    L.hdd_destroy.argtypes = [P]
    L.hdd_destroy.restype = None
    L.hdd_status_str.argtypes = [I]
    L.hdd_status_str.restype = C.c_char_p
    L.hdd_last_error.argtypes = [P]
    L.hdd_last_error.restype = C.c_char_p
    L.hdd_assemble.argtypes = [P, C.POINTER(AssembleParams)]
    L.hdd_assemble.restype = I
    L.hdd_build_rhs.argtypes = [P, I, C.POINTER(D), I, C.POINTER(D), V, V]
    L.hdd_build_rhs.restype = I
    L.hdd_apply_A.argtypes = [P, V, V, I, V]
    L.hdd_apply_A.restype = I
    L.hdd_setup_dd.argtypes = [P, C.POINTER(DDParams)]
    L.hdd_setup_dd.restype = I
    L.hdd_get_subdomain.argtypes = [P, I, C.POINTER(I)]
    L.hdd_get_subdomain.restype = I
    L.hdd_num_subdomains.argtypes = [P]
    L.hdd_num_subdomains.restype = I
    L.hdd_get_offsets.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    L.hdd_get_offsets.restype = I
    L.hdd_setup_deflation.argtypes = [P, V]
    L.hdd_setup_deflation.restype = I
    L.hdd_setup_exact.argtypes = [P, V]
    L.hdd_setup_exact.restype = I
    L.hdd_solve.argtypes = [P, V, V, C.POINTER(SolveParams), C.POINTER(SolveStats), V]
    L.hdd_solve.restype = I
    L.hdd_ras_apply.argtypes = [P, V, V, C.POINTER(SolveParams), C.POINTER(I), V]
    L.hdd_ras_apply.restype = I
    L.hdd_local_op.argtypes = [P, I, I, V, V, V]
    L.hdd_local_op.restype = I
    L.hdd_profile.argtypes = [P, I]
    L.hdd_profile.restype = I
    L.hdd_profile_count.argtypes = [P]
    L.hdd_profile_count.restype = I
    L.hdd_profile_get.argtypes = [P, I, C.POINTER(KernelStat)]
    L.hdd_profile_get.restype = I
    L.hdd_launch_count.argtypes = [P]
    L.hdd_launch_count.restype = C.c_longlong
    L.hdd_setup_batch.argtypes = [P, I]
    L.hdd_setup_batch.restype = I
    L.hdd_autotune.argtypes = [P, C.POINTER(SolveParams), V, C.POINTER(I), C.POINTER(I), C.POINTER(C.c_double)]
    L.hdd_autotune.restype = I
    L.hdd_warmstart_load.argtypes = [P, C.c_char_p]
    L.hdd_warmstart_load.restype = I
    L.hdd_warmstart_save.argtypes = [P, C.c_char_p]
    L.hdd_warmstart_save.restype = I
    L.hdd_num_rhs.argtypes = [P]
    L.hdd_num_rhs.restype = I
    F = C.POINTER(C.c_float)
    L.hdd_cnn_num_params.argtypes = []
    L.hdd_cnn_num_params.restype = I
    L.hdd_stencil_rows.argtypes = [I, C.c_double, I, P, P]
    L.hdd_stencil_rows.restype = I
    L.hdd_cnn_set_params.argtypes = [P, F]
    L.hdd_cnn_set_params.restype = I
    L.hdd_cnn_get_params.argtypes = [P, F]
    L.hdd_cnn_get_params.restype = I
    L.hdd_cnn_forward.argtypes = [P, V, V, V]
    L.hdd_cnn_forward.restype = I
    L.hdd_cnn_infer.argtypes = [P, V, V, V]
    L.hdd_cnn_infer.restype = I
    L.hdd_cnn_loss_grad.argtypes = [P, V, C.POINTER(D), F]
    L.hdd_cnn_loss_grad.restype = I
    L.hdd_cnn_train_step.argtypes = [P, V, C.c_float, C.POINTER(D), V]
    L.hdd_cnn_train_step.restype = I
    L.hdd_get_outer_vector.argtypes = [P, I, V, V]
    L.hdd_get_outer_vector.restype = I
    L.hdd_apply_PA_noalloc.argtypes = [P, V, V, V]
    L.hdd_apply_PA_noalloc.restype = I
    L.hdd_setup_coarse_grid.argtypes = [P, I, V]
    L.hdd_setup_coarse_grid.restype = I
    L.hdd_coarse_grid_op.argtypes = [P, I, I, V, V, V]
    L.hdd_coarse_grid_op.restype = I
    L.hdd_coarse_grid_size.argtypes = [P]
    L.hdd_coarse_grid_size.restype = C.c_longlong
    L.hdd_set_option.argtypes = [P, I, I]
    L.hdd_set_option.restype = I
    _lib = L
    return L
