"""ctypes loader for libsipstokes.so (the C ABI in include/sipstokes.h).

Argument marshalling only.  Importing this module loads the compiled CUDA
library and raises ``ImportError`` when it is missing: there is no CPU
fallback anywhere in the package.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsipstokes.so")

SIP_OK = 0
STATUS_NAMES = {
    0: "SIP_OK", 1: "SIP_ERR_INVALID_ARG", 2: "SIP_ERR_OOM", 3: "SIP_ERR_CUDA",
    4: "SIP_ERR_NOT_CONVERGED", 5: "SIP_ERR_BREAKDOWN", 6: "SIP_ERR_TIMEOUT",
    7: "SIP_ERR_REJECTED", 8: "SIP_ERR_NOT_READY", 9: "SIP_ERR_CANCELLED",
}
BC = {"navier": 0, "neumann": 1, "dirichlet": 2}
PREC = {"fp64": 0, "mixed": 1, "mixed_f32_inner": 2}
COARSE = {"q1": 0, "q0": 1}

c_double_p = ctypes.POINTER(ctypes.c_double)


class ProblemDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("k", ctypes.c_int),
        ("bc", ctypes.c_int * 4),
        ("eta_host", c_double_p),
        ("penalty_scale", ctypes.c_double),
        ("n_hlevels", ctypes.c_int),
        ("cheb_steps_p", ctypes.c_int),
        ("cheb_steps_h", ctypes.c_int),
        ("eig_iters", ctypes.c_int),
        ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int),
        ("coarse", ctypes.c_int),
        ("mixed_fp64_ratio", ctypes.c_double),
    ]


class SolveOpts(ctypes.Structure):
    _fields_ = [
        ("rtol", ctypes.c_double),
        ("max_outer", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("inner_rtol", ctypes.c_double),
        ("max_inner", ctypes.c_int),
        ("inner_loop", ctypes.c_int),
        ("inner_krylov", ctypes.c_int),
        ("inner_norm", ctypes.c_int),
        ("inner_restart", ctypes.c_int),
        ("outer_krylov", ctypes.c_int),
        ("refine", ctypes.c_int),
        ("time_limit_ms", ctypes.c_double),
    ]


class SolveReport(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("outer_its", ctypes.c_int),
        ("inner_total", ctypes.c_int),
        ("inner_max", ctypes.c_int),
        ("inner_avg", ctypes.c_double),
        ("rel_residual", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
        ("lambda_max_p", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
        ("refine_steps", ctypes.c_int),
    ]


_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); every exported entry point of sipstokes.h
SIGNATURES = {
    "sip_problem_desc_default": (None, [ctypes.POINTER(ProblemDesc)]),
    "sip_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_VP)]),
    "sip_ctx_destroy": (None, [_VP]),
    "sip_last_error": (ctypes.c_char_p, [_VP]),
    "sip_problem_create": (ctypes.c_int, [_VP, ctypes.POINTER(ProblemDesc), ctypes.POINTER(_VP)]),
    "sip_problem_destroy": (None, [_VP]),
    "sip_problem_sizes": (ctypes.c_int, [_VP, _I64P, _I64P, _I64P]),
    "sip_problem_schedule": (ctypes.c_int, [_VP, ctypes.c_void_p, ctypes.c_void_p]),
    "sip_problem_set_schedule": (ctypes.c_int, [_VP, ctypes.c_void_p, ctypes.c_void_p]),
    "sip_apply_A": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_apply_A_f32": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_apply_B": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_apply_Bt": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_residual_dd": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sip_problem_setup": (ctypes.c_int, [_VP, _VP]),
    "sip_problem_update_eta": (ctypes.c_int, [_VP, _VP, _VP]),
    "sip_lambda_max": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sip_block_jacobi": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_p_restrict": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_p_prolong_add": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_apply_A1": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_cd_prolong": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_dc_restrict": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_hlevel_dims": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sip_hlevel_stencil": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    "sip_hlevel_apply": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "sip_coarse_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_vcycle": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_vcycle_f32": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "sip_inner_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), _VP]),
    "sip_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
    "sip_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(SolveOpts),
                                 ctypes.POINTER(SolveReport), _VP]),
    "sip_solve_dd": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(SolveOpts),
                                    ctypes.POINTER(SolveReport), _VP]),
    "sip_solve_batch": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP,
                                       ctypes.POINTER(SolveOpts), _VP, ctypes.c_int]),
    "sip_solve_batch_grouped": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP,
                                               ctypes.POINTER(SolveOpts), _VP, ctypes.c_int]),
    "sip_problem_footprint": (ctypes.c_int64, [ctypes.POINTER(ProblemDesc), ctypes.c_int]),
    "sip_server_create": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(_VP)]),
    "sip_server_submit": (ctypes.c_int, [_VP, ctypes.POINTER(ProblemDesc), _VP, ctypes.c_double,
                                         _VP, _VP, ctypes.POINTER(SolveOpts), ctypes.c_uint64]),
    "sip_server_poll": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "sip_server_cancel": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "sip_server_drain": (ctypes.c_int, [_VP]),
    "sip_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), _I64P]),
    "sip_server_destroy": (None, [_VP]),
    "sip_rasterise_inclusions": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, _VP, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, _VP, _VP, _VP]),
    "sip_rasterise_inclusions_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int,
                                                        ctypes.c_double, ctypes.c_double, _VP,
                                                        ctypes.c_int, ctypes.c_double,
                                                        ctypes.c_double, _VP, _VP, _VP]),
    "sip_rhs_body_force": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VP, _VP]),
}

_lib = None


def load():
    """Load the compiled library (once); raise ImportError when absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libsipstokes.so is not built; run `python -m paper_1607_03777_gb300.build` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SipError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
