"""ctypes declarations of the C ABI in include/lindblad_ss.h.

Argument marshalling only: every step of the computation runs inside
liblindblad_ss.so.  Loading fails loudly when the library has not been built
or cannot be loaded -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblindblad_ss.so")

SS_OK, SS_ERR_INVALID, SS_ERR_OOM, SS_NOT_CONVERGED, SS_BREAKDOWN, SS_ZERO_PIVOT, SS_ERR_TIMEOUT, \
    SS_ERR_CUDA, SS_ERR_UNSUPPORTED = range(9)
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID", 2: "ERR_OOM", 3: "NOT_CONVERGED", 4: "BREAKDOWN",
                5: "ZERO_PIVOT", 6: "ERR_TIMEOUT", 7: "ERR_CUDA", 8: "ERR_UNSUPPORTED"}
METHODS = {"direct": 0, "iterative-lgmres": 1, "iterative-gmres": 1, "gmres": 1,
           "iterative-bicgstab": 2, "bicgstab": 2, "inverse-power": 3, "auto": 4}
METHOD_NAMES = {0: "direct", 1: "iterative-lgmres", 2: "iterative-bicgstab", 3: "inverse-power", 4: "auto"}
PRECONDS = {"ilu0": 0, "ilut": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}
KRYLOV = {"bicgstab": 0, "gmres": 1}


class CsrView(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("on_device", C.c_int)]


class Options(C.Structure):
    _fields_ = [("method", C.c_int), ("precond", C.c_int), ("precision", C.c_int), ("tol", C.c_double),
                ("maxiter", C.c_int), ("restart", C.c_int), ("drop_tol", C.c_double),
                ("fill_factor", C.c_double), ("w", C.c_double), ("sigma", C.c_double),
                ("use_rcm", C.c_int), ("seed", C.c_uint64), ("inner_rtol", C.c_double), ("lgmres_k", C.c_int),
                ("warm_start", C.c_int), ("autotune", C.c_int)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("outer_iters", C.c_int),
                ("resid_Lrho", C.c_double), ("w_used", C.c_double), ("condest", C.c_double),
                ("n", C.c_int64), ("nnz", C.c_int64), ("bandwidth", C.c_int64), ("profile", C.c_int64),
                ("nnz_factors", C.c_int64), ("levels_lower", C.c_int32), ("levels_upper", C.c_int32),
                ("ms_setup", C.c_double), ("ms_solve", C.c_double), ("method", C.c_int),
                ("bw_modified", C.c_int64), ("bw_shifted", C.c_int64),
                ("tune_lanes_shift", C.c_int32 * 3), ("tune_stage", C.c_int32), ("fp64_fallback", C.c_int32)]

    def as_dict(self) -> dict:
        out = {k: getattr(self, k) for k, _ in self._fields_}
        out["tune_lanes_shift"] = list(self.tune_lanes_shift)
        out["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        out["method_name"] = METHOD_NAMES.get(self.method, str(self.method))
        return out


_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)
_I64P = C.POINTER(C.c_int64)
_I32P = C.POINTER(C.c_int32)
_DP = C.POINTER(C.c_double)

class ServerOptions(C.Structure):
    _fields_ = [("hbm_budget_mb", C.c_double), ("max_waves", C.c_int), ("max_wave_systems", C.c_int),
                ("warm_start", C.c_int)]


_SIGNATURES = {
    "ss_ctx_create": (C.c_int, [C.c_int, _P, _PP]),
    "ss_ctx_destroy": (C.c_int, [_P]),
    "ss_ctx_set_stream": (C.c_int, [_P, _P]),
    "ss_last_error": (C.c_char_p, [_P]),
    "ss_options_default": (None, [C.POINTER(Options)]),
    "assemble_liouvillian": (C.c_int, [_P, C.POINTER(CsrView), C.c_int, C.POINTER(CsrView), _PP]),
    "add_trace_row": (C.c_int, [_P, _P, C.c_double, _PP, _DP]),
    "assemble_trace_batched": (C.c_int, [_P, C.c_int, C.POINTER(CsrView), C.POINTER(C.c_int),
                                         C.POINTER(C.POINTER(CsrView)), C.c_double, C.POINTER(C.c_void_p), _DP]),
    "add_shift": (C.c_int, [_P, _P, C.c_double, _PP]),
    "rcm_permute": (C.c_int, [_P, _P, _P, _I64P, _I64P]),
    "permute": (C.c_int, [_P, _P, _P, _PP]),
    "bandwidth_profile": (C.c_int, [_P, _P, _I64P, _I64P]),
    "ss_mat_shape": (C.c_int, [_P, _I64P, _I64P]),
    "ss_mat_export": (C.c_int, [_P, _P, _P, _P, _P]),
    "ss_mat_import": (C.c_int, [_P, C.POINTER(CsrView), _PP]),
    "ss_mat_free": (None, [_P]),
    "spmv": (C.c_int, [_P, _P, _P, _P]),
    "spmv_f32": (C.c_int, [_P, _P, _P, _P]),
    "ilu_factor": (C.c_int, [_P, _P, C.c_int, C.c_double, C.c_double, C.c_int, _PP, _DP]),
    "precond_apply": (C.c_int, [_P, _P, _P, _P]),
    "precond_apply_f32": (C.c_int, [_P, _P, _P, _P]),
    "ss_prec_info": (C.c_int, [_P, _I64P, _I32P, _I32P]),
    "ss_prec_export": (C.c_int, [_P, _P, _P, _P, _P]),
    "ss_prec_free": (None, [_P]),
    "krylov_solve": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, C.c_double, C.c_int, C.c_int,
                               C.POINTER(C.c_int), _DP]),
    "steady_state_batched": (C.c_int, [_P, C.c_int, C.POINTER(CsrView), C.POINTER(C.c_int),
                                       C.POINTER(C.POINTER(CsrView)), C.POINTER(Options), C.POINTER(C.c_void_p),
                                       C.c_int, C.POINTER(Info)]),
    "ss_profile_enable": (C.c_int, [_P, C.c_int]),
    "ss_profile_read": (C.c_int, [_P, C.c_int, _I64P, _DP]),
    "ss_launch_count": (C.c_ulonglong, []),
    "ss_alloc_count": (C.c_ulonglong, []),
    "ss_set_wait_limit": (C.c_int, [_P, C.c_uint64]),
    "ss_tune_search_host": (C.c_int, [_P, C.c_int32, _P, C.POINTER(C.c_int32)]),
    "ss_diag_prec_skip_row": (C.c_int, [_P, _P, C.c_int64, C.c_int]),
    "ss_diag_batched_stall": (C.c_int, [_P, C.c_int64]),
    "lgmres_solve": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_int, C.c_int, C.c_int,
                               C.POINTER(C.c_int), _DP]),
    "ss_rcm_order_host": (C.c_int, [C.c_int64, _P, _P, _P]),
    "ss_level_sets_host": (C.c_int, [C.c_int64, _P, _P, C.c_int, _P, _P, C.POINTER(C.c_int32)]),
    "ss_ilu0_schedule_host": (C.c_int, [C.c_int64, _P, _P, C.c_int64, _P, _P, _P, _I64P]),
    "ss_ilut_host": (C.c_int, [C.c_int64, _P, _P, _P, C.c_double, C.c_double, C.c_int64, _P, _P, _P,
                               _I64P, _I64P]),
    "ss_mbm_host": (C.c_int, [C.c_int64, _P, _P, _P, _P, _I64P]),
    "krylov_solve_noalloc": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_int, C.POINTER(C.c_int), _DP]),
    "steady_state": (C.c_int, [_P, C.POINTER(CsrView), C.c_int, C.POINTER(CsrView), C.POINTER(Options),
                               _P, C.c_int, C.POINTER(Info)]),
    "ss_server_options_default": (None, [C.POINTER(ServerOptions)]),
    "ss_server_create": (C.c_int, [C.c_int, C.POINTER(Options), C.POINTER(ServerOptions), _PP]),
    "ss_server_destroy": (C.c_int, [_P]),
    "ss_submit": (C.c_int, [_P, C.POINTER(CsrView), C.c_int, C.POINTER(CsrView), _P, C.POINTER(C.c_uint64)]),
    "ss_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_int)]),
    "ss_wait": (C.c_int, [_P, C.c_uint64, C.c_int64, C.POINTER(Info), _DP]),
    "ss_server_stats": (C.c_int, [_P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), _DP, _DP]),
    "ss_server_last_error": (C.c_char_p, [_P]),
}

_lib = None


def exported_names():
    return list(_SIGNATURES)


def load(path: str = LIB_PATH):
    """Load liblindblad_ss.so and declare every signature; raises when absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblindblad_ss.so is not built ({path}); run paper_1504_06768_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
