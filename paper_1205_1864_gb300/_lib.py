"""ctypes declarations of libsghsc.so (include/sghsc.h). Argument marshalling
only: no arithmetic of the method happens in Python. Importing this module
loads the shared library and raises if it has not been built."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsghsc.so")

SG_OK, SG_ERR_INVALID_ARG, SG_ERR_CUDA, SG_ERR_OOM, SG_ERR_NOT_SPD, SG_ERR_BREAKDOWN, \
    SG_ERR_NO_CONVERGENCE, SG_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = {0: "SG_OK", 1: "SG_ERR_INVALID_ARG", 2: "SG_ERR_CUDA", 3: "SG_ERR_OOM", 4: "SG_ERR_NOT_SPD",
                5: "SG_ERR_BREAKDOWN", 6: "SG_ERR_NO_CONVERGENCE", 7: "SG_ERR_UNSUPPORTED"}
SG_F64, SG_F32, SG_F32_ACC64, SG_F32_ACCDF64 = 0, 1, 2, 3
SG_LEGENDRE, SG_HERMITE = 0, 1
SG_PREC_NONE, SG_PREC_MEAN, SG_PREC_HSC, SG_PREC_BGS = 0, 1, 2, 3
SG_M0_VCYCLE, SG_M0_DIAG = 0, 1
SG_MAX_HIST = 1024


class sg_mesh(C.Structure):
    _fields_ = [("ne_x", C.c_int), ("ne_y", C.c_int)]


class sg_prec_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("top_level_f64", C.c_int), ("inner_tol", C.c_double),
                ("inner_maxit", C.c_int), ("inner_fixed_iters", C.c_int), ("nu", C.c_int), ("omega", C.c_double),
                ("m0", C.c_int), ("level_tol", C.c_double), ("level_maxit", C.c_int), ("md_m0", C.c_int),
                ("df64", C.c_int)]


class sg_solve_opts(C.Structure):
    _fields_ = [("precond", C.c_int), ("prec", sg_prec_opts), ("tol", C.c_double), ("maxit", C.c_int),
                ("flexible", C.c_int), ("use_x0", C.c_int), ("check_true_residual", C.c_int),
                ("schur_reduced", C.c_int), ("schur_inner_tol", C.c_double)]


class sg_solve_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("rel_res", C.c_double),
                ("true_rel_res", C.c_double), ("kappa_est", C.c_double), ("inner_iters_total", C.c_longlong),
                ("inner_iters_max", C.c_int), ("solve_ms", C.c_double), ("n_hist", C.c_int),
                ("res_hist", C.c_double * (SG_MAX_HIST + 1)), ("alpha", C.c_double * SG_MAX_HIST),
                ("beta", C.c_double * SG_MAX_HIST)]


class SGError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsghsc.so is not built ({LIB_PATH}); run paper_1205_1864_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    P = C.POINTER
    sig = {
        "sg_setup": (i, [P(sg_mesh), i, i, i, i, i, P(C.c_int), P(C.c_int), P(C.c_double), P(C.c_double), P(vp)]),
        "sg_setup_gpc": (i, [P(sg_mesh), i, i, i, i, i, i, P(C.c_int), P(C.c_int), P(C.c_double), P(C.c_double),
                             P(vp)]),
        "sg_problem_terms": (i, [vp, P(i), P(i)]),
        "sg_destroy": (None, [vp]),
        "sg_set_scales": (i, [vp, P(C.c_double)]),
        "sg_problem_dims": (i, [vp, P(i), P(i), P(i), P(i), P(i)]),
        "sg_chaos_table": (i, [vp, P(C.c_int), P(C.c_int)]),
        "sg_apply": (i, [vp, vp, vp, i, vp]),
        "sg_level_apply": (i, [vp, i, i, vp, vp, vp, i, vp]),
        "sg_vcycle_apply": (i, [vp, vp, vp, i, i, P(sg_prec_opts), vp]),
        "sg_vcycle_apply_static": (i, [vp, vp, vp, i, i, P(sg_prec_opts), vp]),
        "sg_inner_solve": (i, [vp, vp, vp, i, i, P(sg_prec_opts), P(C.c_int), vp]),
        "sg_inner_cluster": (i, [vp]),
        "sg_inner_path": (i, [vp, i, i]),
        "hsc_precond_apply": (i, [vp, vp, vp, P(sg_prec_opts), vp]),
        "mean_precond_apply": (i, [vp, vp, vp, P(sg_prec_opts), vp]),
        "bgs_precond_apply": (i, [vp, vp, vp, P(sg_prec_opts), vp]),
        "sg_solve": (i, [vp, vp, vp, P(sg_solve_opts), P(sg_solve_stats), vp]),
        "sg_solve_host": (i, [vp, vp, vp, P(sg_solve_opts), P(sg_solve_stats), vp]),
        "sg_qoi": (i, [vp, vp, vp, vp, vp]),
        "sg_autotune": (i, [vp, vp]),
        "sg_autotune_result": (i, [vp, P(i), P(i)]),
        "sg_autotune_forms": (i, [vp, P(i), P(i), P(i)]),
        "sg_autotune_outer_result": (i, [vp, P(i)]),
        "sg_autotune_set": (i, [vp, i, i, i, i, i, i]),
        "sg_batch_create": (i, [i, P(vp), P(vp)]),
        "sg_batch_solve": (i, [vp, P(vp), P(vp), P(sg_solve_opts), P(sg_solve_stats), vp]),
        "sg_batch_solve_host": (i, [vp, P(vp), P(vp), P(sg_solve_opts), P(sg_solve_stats), vp]),
        "sg_batch_destroy": (None, [vp]),
        "sg_qoi_grad": (i, [vp, vp, vp, i, P(C.c_double), vp, vp, vp]),
        "sg_measure_alu_peak": (i, [i, i, P(C.c_double), vp]),
        "sg_kl_set_theta": (i, [vp, P(C.c_double)]),
        "sg_kl_qoi_grad": (i, [vp, vp, vp, P(C.c_double), vp, vp, vp]),
        "sg_last_error": (C.c_char_p, []),
        "sg_kernel_launches": (C.c_longlong, []),
        "sg_default_prec_opts": (None, [P(sg_prec_opts)]),
        "sg_default_solve_opts": (None, [P(sg_solve_opts)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def check(status: int, where: str):
    if status != SG_OK:
        msg = LIB.sg_last_error()
        raise SGError(status, where, msg.decode() if msg else "")
    return status


def exported_symbols():
    """Names the header declares (used by the CPU test of the library)."""
    return ["sg_setup", "sg_setup_gpc", "sg_problem_terms", "sg_destroy", "sg_set_scales", "sg_problem_dims", "sg_chaos_table", "sg_apply", "sg_level_apply",
            "sg_vcycle_apply", "sg_vcycle_apply_static", "sg_inner_solve", "sg_inner_cluster", "sg_inner_path", "hsc_precond_apply", "mean_precond_apply", "bgs_precond_apply", "sg_solve", "sg_solve_host", "sg_qoi", "sg_autotune", "sg_autotune_result", "sg_autotune_forms",
            "sg_autotune_outer_result", "sg_autotune_set",
            "sg_batch_create", "sg_batch_solve", "sg_batch_solve_host", "sg_batch_destroy",
            "sg_qoi_grad", "sg_measure_alu_peak", "sg_kl_set_theta", "sg_kl_qoi_grad", "sg_last_error", "sg_kernel_launches", "sg_default_prec_opts", "sg_default_solve_opts"]
