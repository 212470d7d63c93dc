"""ctypes binding of librsd.so: the C ABI of include/rsd.h, names unchanged.

Argument marshalling only.  Every numerical step runs in the library's CUDA kernels;
there is no Python or CPU fallback, and loading fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsd.so")

RSD_OK = 0
RSD_ERR_ARG = -1
RSD_ERR_PARTITION = -2
RSD_ERR_NOT_SPD = -3
RSD_ERR_NOMEM = -4
RSD_ERR_CUDA = -5
RSD_ERR_TIMEOUT = -6
RSD_ERR_NOCONV = -7

RSD_PREC_FP64 = 0
RSD_PREC_FP32 = 1
RSD_PREC_TF32 = 2
RSD_PREC_FP16 = 3
RSD_PREC_BF16 = 4

RSD_KRYLOV_AUTO = 0
RSD_KRYLOV_PCG = 1
RSD_KRYLOV_FGMRES = 2

RSD_MODE_EXACT = 0
RSD_MODE_PAPER = 1
RSD_MEM_HOST = 0
RSD_MEM_DEVICE = 1

# every function include/rsd.h declares (checked by the tests)
EXPORTS = [
    "rsd_setup", "rsd_apply", "rsd_solve", "rsd_check", "rsd_destroy", "rsd_strerror",
    "rsd_get_info", "rsd_front_dims", "rsd_front_dofs", "rsd_front_map", "rsd_front_factor", "rsd_front_factor16", "rsd_front_dinv",
    "rsd_grid_sizes", "rsd_grid_assemble", "rsd_grid_load", "rsd_grid_partition",
    "rsd_profile", "rsd_launch_count", "rsd_apply_static", "rsd_last_error_detail",
    "rsd_release_cache", "rsd_setup_batched", "rsd_solve_adjoint", "rsd_grid_exp",
    "rsd_grid_coef_grad", "rsd_profile_trace", "rsd_peak_gemm",
    "rsd_inject_drop_sweep_item", "rsd_grid_elastic_sizes", "rsd_grid_elastic_assemble",
    "rsd_grid_elastic_load", "rsd_grid_elastic_partition", "rsd_autotune", "rsd_tune_load",
    "rsd_front_factor_upper",
]


class rsd_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("mem", C.c_int32)]


class rsd_tree(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("parent", C.c_void_p)]


class rsd_options(C.Structure):
    _fields_ = [("mode", C.c_int32), ("prec_leaf", C.c_int32), ("prec_mid", C.c_int32),
                ("prec_root", C.c_int32), ("maxit", C.c_int32), ("stream", C.c_void_p),
                ("profile", C.c_int32), ("wait_cycles", C.c_int64), ("gamma", C.c_int32),
                ("krylov", C.c_int32), ("restart", C.c_int32), ("tune_cache", C.c_char_p),
                ("nonsymmetric", C.c_int32)]


class rsd_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("relres", C.c_double),
                ("relres_recursive", C.c_double), ("history", C.c_double * 64)]


class rsd_info_t(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_nodes", C.c_int32), ("n_levels", C.c_int32),
                ("factor_elems", C.c_int64), ("factor_bytes", C.c_int64),
                ("setup_flops", C.c_double), ("device_bytes", C.c_int64),
                ("notspd_node", C.c_int32), ("promoted", C.c_int32)]


PROFILE_CLASSES = ["assemble", "extend_add", "gemm_tcgen05", "gemm_simt", "diag_factor",
                   "panel_solve_simt", "sweep_up", "sweep_down", "sweep_gather", "krylov", "factor_copy16",
                   "gamma_gmres", "gemm_tcgen05_f16", "gamma_smv", "gamma_iface"]


class rsd_profile_t(C.Structure):
    _fields_ = [("launches", C.c_int64 * 15), ("ms", C.c_double * 15), ("flops", C.c_double * 15),
                ("bytes", C.c_double * 15), ("host_analysis_ms", C.c_double),
                ("host_parts_ms", C.c_double * 6), ("host_issue_ms", C.c_double)]


class rsd_trace_rec(C.Structure):
    _fields_ = [("cls", C.c_int32), ("stream", C.c_int32), ("start_ms", C.c_double),
                ("end_ms", C.c_double), ("flops", C.c_double), ("bytes", C.c_double),
                ("issue_ms", C.c_double)]


_lib = None


def load() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first (paper_1210_6266_gb300/build.py)")
        lib = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sig = {
            "rsd_setup": (C.c_int, [C.POINTER(rsd_csr), P, C.POINTER(rsd_tree), C.POINTER(rsd_options), C.POINTER(P)]),
            "rsd_apply": (C.c_int, [P, P, P]),
            "rsd_apply_static": (C.c_int, [P, P, P]),
            "rsd_solve": (C.c_int, [P, P, P, C.c_double, C.POINTER(rsd_stats)]),
            "rsd_solve_adjoint": (C.c_int, [P, P, P, C.c_double, C.POINTER(rsd_stats)]),
            "rsd_check": (C.c_int, [P]),
            "rsd_inject_drop_sweep_item": (C.c_int, [P, C.c_int32]),
            "rsd_destroy": (None, [P]),
            "rsd_strerror": (C.c_char_p, [C.c_int]),
            "rsd_last_error_detail": (C.c_char_p, []),
            "rsd_get_info": (C.c_int, [P, C.POINTER(rsd_info_t)]),
            "rsd_front_dims": (C.c_int, [P, C.c_int32, P, P, P]),
            "rsd_front_dofs": (C.c_int, [P, C.c_int32, P]),
            "rsd_front_map": (C.c_int, [P, C.c_int32, P]),
            "rsd_front_factor": (C.c_int, [P, C.c_int32, P]),
            "rsd_front_factor16": (C.c_int, [P, C.c_int32, P]),
            "rsd_front_dinv": (C.c_int, [P, C.c_int32, P]),
            "rsd_front_factor_upper": (C.c_int, [P, C.c_int32, P]),
            "rsd_grid_sizes": (C.c_int, [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
            "rsd_grid_assemble": (C.c_int, [C.c_int32, P, P, P, P, P]),
            "rsd_grid_load": (C.c_int, [C.c_int32, P, P, P]),
            "rsd_grid_partition": (C.c_int, [C.c_int32, C.c_int32, P, P, P]),
            "rsd_grid_exp": (C.c_int, [C.c_int32, P, P, P]),
            "rsd_grid_elastic_sizes": (C.c_int, [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
            "rsd_grid_elastic_assemble": (C.c_int, [C.c_int32, C.c_int32, P, C.c_double, P, P, P, P]),
            "rsd_grid_elastic_load": (C.c_int, [C.c_int32, P, P, P]),
            "rsd_grid_elastic_partition": (C.c_int, [C.c_int32, C.c_int32, P, P, P, P]),
            "rsd_grid_coef_grad": (C.c_int, [C.c_int32, P, P, P, P, P, P]),
            "rsd_profile": (C.c_int, [P, C.POINTER(rsd_profile_t), C.c_int32]),
            "rsd_profile_trace": (C.c_int, [P, P, C.c_int64, C.POINTER(C.c_int64)]),
            "rsd_launch_count": (C.c_int64, []),
            "rsd_autotune": (C.c_int, [C.c_char_p, C.POINTER(C.c_double), P]),
            "rsd_tune_load": (C.c_int, [C.c_char_p, C.POINTER(C.c_int32)]),
            "rsd_peak_gemm": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double, P,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "rsd_release_cache": (None, []),
            "rsd_setup_batched": (C.c_int, [C.c_int32, C.POINTER(rsd_csr), P, C.POINTER(rsd_tree),
                                            C.POINTER(rsd_options), C.POINTER(P)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class RSDError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        detail = lib.rsd_last_error_detail().decode()
        super().__init__(f"{where}: {lib.rsd_strerror(code).decode()} ({code}) {detail}")
        self.code = code


def check(code: int, where: str) -> int:
    if code != RSD_OK:
        raise RSDError(code, where)
    return code
