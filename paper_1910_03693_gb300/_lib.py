"""ctypes binding of ``libfrgb.so`` (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module converts
PyTorch tensors to device pointers, passes the current CUDA stream, and turns
error codes into exceptions.  Importing it fails loudly when the library has
not been built: there is no fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfrgb.so")

FR_OK = 0
FR_F64, FR_F32, FR_BF16OP, FR_DF = 0, 1, 2, 3
FR_JV_FD, FR_JV_EXACT = 0, 1
STATUS = {0: "FR_OK", -1: "FR_ERR_INVALID", -2: "FR_ERR_CUDA", -3: "FR_ERR_NOMEM",
          -4: "FR_ERR_NOT_CONVERGED", -5: "FR_ERR_NONFINITE", -6: "FR_ERR_TIMEOUT"}


class MeshDesc(C.Structure):
    _fields_ = [("nd", C.c_int32), ("n_elem", C.c_int32), ("geom_order", C.c_int32),
                ("nodes", C.POINTER(C.c_double)), ("nbr", C.POINTER(C.c_int32)),
                ("nbr_face", C.POINTER(C.c_int8)), ("orient", C.POINTER(C.c_int8)),
                ("p", C.POINTER(C.c_int8))]


class Physics(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mu", C.c_double), ("Pr", C.c_double),
                ("q_inf", C.c_double * 5), ("flux", C.c_int32)]


FLUX = {"rusanov": 0, "roe": 1}


class Limits(C.Structure):
    _fields_ = [("p_min", C.c_int32), ("p_max", C.c_int32)]


class LayoutInfo(C.Structure):
    _fields_ = [("nd", C.c_int32), ("nv", C.c_int32), ("n_elem", C.c_int32),
                ("n_dof", C.c_int64), ("n_dof_capacity", C.c_int64),
                ("bucket_count", C.c_int32 * 6), ("bucket_offset", C.c_int64 * 6),
                ("affine", C.c_int32)]


class ShiftedOp(C.Structure):
    _fields_ = [("sigma", C.c_double), ("q64_dev", C.c_void_p), ("mode", C.c_int),
                ("jv_prec", C.c_int), ("eps", C.c_double), ("precond", C.c_int32)]


class GmresOpts(C.Structure):
    _fields_ = [("m", C.c_int32), ("rtol", C.c_double), ("max_it", C.c_int32), ("reorth", C.c_int32)]


class GmresStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("rel_res", C.c_double)]


class Tableau(C.Structure):
    _fields_ = [("s", C.c_int32), ("A", C.c_double * 36), ("b", C.c_double * 6)]


class NewtonOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("dtau_init", C.c_double), ("dtau_max", C.c_double),
                ("max_newton", C.c_int32), ("max_halvings", C.c_int32), ("mode", C.c_int),
                ("jv_prec", C.c_int), ("eps", C.c_double), ("gmres", GmresOpts), ("low_above", C.c_double),
                ("precond", C.c_int32), ("low_prec", C.c_int)]


class StageStats(C.Structure):
    _fields_ = [("newton_iterations", C.c_int32), ("gmres_iterations", C.c_int32),
                ("halvings", C.c_int32), ("converged", C.c_int32),
                ("norm0", C.c_double), ("norm_final", C.c_double),
                ("low_evaluations", C.c_int32), ("f64_evaluations", C.c_int32)]


class AdaptOpts(C.Structure):
    _fields_ = [("nu_max", C.c_double), ("nu_min", C.c_double),
                ("p_min", C.c_int32), ("p_max", C.c_int32)]


# name -> (restype, argtypes); every function returns fr_status except fr_last_error
SIGNATURES = {
    "fr_create": [C.POINTER(MeshDesc), C.POINTER(Physics), C.POINTER(Limits), C.POINTER(C.c_void_p)],
    "fr_destroy": [C.c_void_p],
    "fr_layout": [C.c_void_p, C.POINTER(LayoutInfo)],
    "fr_get_p": [C.c_void_p, C.POINTER(C.c_int8)],
    "fr_pack": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "fr_unpack": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "fr_residual": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "fr_jvp": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p],
    "fr_jvp_fd_static": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p],
    "fr_vjp": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "gmres_solve": [C.c_void_p, C.POINTER(ShiftedOp), C.c_void_p, C.c_void_p, C.POINTER(GmresOpts),
                    C.POINTER(GmresStats), C.c_void_p],
    "esdirk_stage": [C.c_void_p, C.POINTER(Tableau), C.c_int32, C.c_double, C.c_void_p,
                     C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(NewtonOpts), C.POINTER(StageStats),
                     C.c_void_p],
    "spectral_decay_indicator": [C.c_void_p, C.c_void_p, C.c_int, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_void_p],
    "fr_timing": [C.c_void_p, C.c_int32],
    "fr_timing_select": [C.c_void_p, C.c_char_p],
    "fr_autotune": [C.c_void_p, C.c_void_p, C.c_void_p],
    "fr_tuning_get": [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "fr_tuning_set": [C.c_void_p, C.POINTER(C.c_int32), C.c_int32],
    "fr_esdirk_tableau": [C.c_int32, C.POINTER(Tableau)],
    "fr_timing_report": [C.c_void_p, C.c_char_p, C.c_int64, C.POINTER(C.c_int64)],
    "p_rebucket": [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(AdaptOpts), C.c_void_p, C.c_int,
                   C.c_void_p, C.c_void_p],
    "esdirk_step": [C.c_void_p, C.POINTER(Tableau), C.c_double, C.c_void_p, C.POINTER(NewtonOpts),
                    C.POINTER(StageStats), C.POINTER(AdaptOpts), C.c_int32, C.c_void_p],
    "fr_precond_build": [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p],
    "fr_precond_apply": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "fr_precond_release": [C.c_void_p],
    "fr_filter": [C.c_void_p, C.c_void_p, C.c_double, C.c_int32, C.c_void_p],
    "fr_dfloat_eval": [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p],
    "fr_fma_rate": [C.c_int, C.c_int64, C.POINTER(C.c_double), C.c_void_p],
    "fr_device_status": [C.c_void_p, C.POINTER(C.c_int32), C.c_int32],
}


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1910_03693_gb300.build.build() "
                          "(the FR hot path has no non-CUDA implementation)")
    lib = C.CDLL(path)
    for name, argtypes in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = C.c_int
        fn.argtypes = argtypes
    lib.fr_last_error.restype = C.c_char_p
    lib.fr_last_error.argtypes = []
    return lib


def exported_symbols(lib):
    return [n for n in list(SIGNATURES) + ["fr_last_error"] if hasattr(lib, n)]
