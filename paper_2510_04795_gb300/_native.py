"""ctypes binding of libozdmrg (argument marshalling only; every step runs in the library).

The library is loaded from the package's _lib/ directory.  There is no fallback: a missing or
unloadable library raises, and calls that fail raise OzError with the library's message.
"""
from __future__ import annotations

import ctypes as C
import os

_LIBPATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libozdmrg.so")

OZ_OK, OZ_EINVAL, OZ_ENONFINITE, OZ_ENOCONV, OZ_EVARIATIONAL, OZ_ETIMEOUT, OZ_ECUDA, OZ_ENOMEM = range(8)
OZ_MODE_EAGER, OZ_MODE_NATIVE, OZ_MODE_PERFORMANT = 0, 1, 2
OZ_NFEAT = 20
OZ_SELECT_FIXED, OZ_SELECT_ANALYTIC, OZ_SELECT_LEARNED = 0, 1, 2
STATUS_NAMES = {0: "OZ_OK", 1: "OZ_EINVAL", 2: "OZ_ENONFINITE", 3: "OZ_ENOCONV", 4: "OZ_EVARIATIONAL",
                5: "OZ_ETIMEOUT", 6: "OZ_ECUDA", 7: "OZ_ENOMEM"}


class OzError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class oz_prec(C.Structure):
    _fields_ = [("slices", C.c_int), ("level", C.c_int), ("mode", C.c_int), ("tile", C.c_int)]


OZ_TILE_AUTO, OZ_TILE_CTA, OZ_TILE_PAIR = 0, 1, 2


class oz_task(C.Structure):
    _fields_ = [("src", C.c_int), ("dst", C.c_int), ("coef", C.c_double), ("d_L", C.c_void_p), ("d_R", C.c_void_p)]


class oz_heff_info(C.Structure):
    _fields_ = [("dim", C.c_longlong), ("flops", C.c_longlong), ("carrier_flops", C.c_longlong),
                ("bytes_ops", C.c_longlong), ("bytes_scratch", C.c_longlong), ("gemm1_tiles", C.c_longlong),
                ("gemm2_tiles", C.c_longlong), ("slices", C.c_int), ("level", C.c_int), ("mode", C.c_int),
                ("tile", C.c_int), ("units", C.c_int), ("epilogue1", C.c_int), ("epilogue2", C.c_int)]


class oz_dmrg_step(C.Structure):
    _fields_ = [("sweep", C.c_int), ("dir", C.c_int), ("bond", C.c_int), ("dim", C.c_int), ("nterm", C.c_int),
                ("ntask", C.c_int), ("iters", C.c_int), ("converged", C.c_int), ("kept", C.c_int),
                ("energy", C.c_double), ("discarded", C.c_double), ("energy_fp64", C.c_double),
                ("nonvariational", C.c_int), ("predicted", C.c_int),
                ("rotated", C.c_int)]


_lib = None


def lib_path() -> str:
    return _LIBPATH


def load():
    """Load (once) and declare the C ABI.  Raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        raise OzError(OZ_ECUDA, f"libozdmrg.so not built ({_LIBPATH}); run __graft_entry__.build()")
    L = C.CDLL(_LIBPATH)
    vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "oz_ctx_create": (i, [C.POINTER(vp), i]),
        "oz_ctx_destroy": (i, [vp]),
        "oz_last_error": (C.c_char_p, []),
        "oz_status": (i, [vp, vp]),
        "ozaki_gemm": (i, [vp, i, i, i, d, vp, i, vp, i, d, vp, i, C.POINTER(oz_prec), vp]),
        "oz_performant_choice": (i, [vp, i, i, i, C.POINTER(oz_prec), C.POINTER(i), C.POINTER(C.c_float)]),
        "ozaki_slice": (i, [vp, i, i, vp, i, i, vp, vp, vp]),
        "ozaki_gemm_noalloc": (i, [i, i, i, d, vp, i, vp, i, d, vp, i, i, i, vp]),
        "ozaki_slice_products": (i, [vp, i, i, i, vp, i, vp, i, i, vp, vp]),
        "oz_heff_create": (i, [vp, i, C.POINTER(i), C.POINTER(i), i, C.POINTER(oz_task), C.POINTER(oz_prec),
                               C.POINTER(vp)]),
        "oz_heff_destroy": (i, [vp]),
        "oz_heff_update_ops": (i, [vp, i, vp]),
        "heff_apply": (i, [vp, vp, vp, vp]),
        "oz_heff_info_get": (i, [vp, C.POINTER(oz_heff_info)]),
        "heff_apply_host": (i, [vp, vp, vp, vp]),
        "oz_heff_stage_times": (i, [vp, C.POINTER(C.c_float)]),
        "oz_heff_diag": (i, [vp, vp, vp]),
        "oz_heff_set_levels": (i, [vp, vp, vp]),
        "oz_heff_autotune": (i, [vp, vp, i, vp, vp, vp]),
        "oz_heff_problem_features": (i, [vp, vp, vp, vp, vp]),
        "oz_heff_problem_errors": (i, [vp, vp, i, vp, vp, vp]),
        "oz_heff_select_levels": (i, [vp, vp, i, d, vp, d, vp, vp, vp]),
        "oz_mlp_create": (i, [i, i, i, C.c_ulonglong, C.POINTER(vp)]),
        "oz_mlp_destroy": (i, [vp]),
        "oz_mlp_param_count": (i, [vp]),
        "oz_mlp_nin": (i, [vp]),
        "oz_mlp_nout": (i, [vp]),
        "oz_mlp_get_params": (i, [vp, vp]),
        "oz_mlp_set_params": (i, [vp, vp]),
        "oz_mlp_forward": (i, [vp, vp, i, vp, vp]),
        "oz_mlp_gradient": (i, [vp, vp, vp, vp, i, C.POINTER(C.c_float), vp, vp]),
        "oz_mlp_train": (i, [vp, vp, vp, vp, i, i, i, C.c_float, C.c_ulonglong, C.POINTER(C.c_float), vp]),
        "oz_heff_get_levels": (i, [vp, vp, vp]),
        "oz_davidson_create": (i, [vp, i, d, C.POINTER(vp)]),
        "oz_davidson_destroy": (i, [vp]),
        "davidson_start": (i, [vp, vp, vp]),
        "davidson_step": (i, [vp, C.POINTER(d), C.POINTER(d), C.POINTER(i), vp]),
        "davidson_ritz": (i, [vp, vp, vp]),
        "davidson_solve": (i, [vp, vp, d, i, C.POINTER(d), C.POINTER(i), vp]),
        "lanczos_solve": (i, [vp, vp, d, i, i, C.POINTER(d), C.POINTER(i), vp]),
        "oz_symeig_small": (i, [vp, i, i, vp, vp, i, vp]),
        "oz_mpo_bond_dims": (i, [vp, vp, i, vp]),
        "oz_mpo_dense": (i, [vp, vp, i, vp]),
        "oz_dmrg_create": (i, [vp, vp, vp, i, i, i, i, C.POINTER(oz_prec), d, C.c_ulonglong, C.POINTER(vp)]),
        "oz_dmrg_destroy": (i, [vp]),
        "oz_dmrg_run": (i, [vp, i, vp]),
        "oz_dmrg_set_renorm_prec": (i, [vp, C.POINTER(oz_prec)]),
        "oz_dmrg_set_rdm_prec": (i, [vp, C.POINTER(oz_prec)]),
        "oz_dmrg_set_solver": (i, [vp, i, d, i]),
        "oz_dmrg_set_prediction": (i, [vp, i]),
        "oz_dmrg_steps": (i, [vp, vp, i, C.POINTER(i)]),
        "oz_dmrg_bond_heff": (i, [vp, i, vp, vp, vp, C.POINTER(ll), vp]),
        "oz_dmrg_set_trace": (i, [vp, i]),
        "oz_heff_partition": (i, [i, vp, vp, i, vp, vp, i, vp]),
        "oz_heff_ops_times": (i, [vp, vp, vp]),
        "oz_reduce_ordered": (i, [vp, i, ll, vp, vp]),
        "oz_heff_set_epilogue": (i, [vp, i, i]),
        "oz_heff_apply_streamed": (i, [vp, i, C.POINTER(i), C.POINTER(i), i, C.POINTER(oz_task), C.POINTER(oz_prec),
                                       i, vp, vp, vp]),
        "oz_dmrg_trace": (i, [vp, ll, vp, vp, vp, vp, C.POINTER(ll)]),
        "dmrg_sweep": (i, [vp, vp, vp, i, i, i, i, i, C.POINTER(oz_prec), d, C.c_ulonglong, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(rc: int):
    if rc != OZ_OK:
        raise OzError(rc, load().oz_last_error().decode(errors="replace"))
