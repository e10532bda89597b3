"""ctypes loader for libpyjac_gb.so (the C ABI declared in include/pyjac_gb.h).

Argument marshalling only.  Loading fails loudly when the library has not
been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

PJ_OK, PJ_ERR_ARG, PJ_ERR_MECH, PJ_ERR_CUDA, PJ_ERR_NOMEM, PJ_ERR_UNSUPPORTED, PJ_ERR_TIMEOUT = range(7)
PJ_CONP, PJ_CONV = 0, 1
PJ_CSR, PJ_CSC, PJ_DENSE = 0, 1, 2
PJ_ELEMENTARY, PJ_THIRD_BODY, PJ_LINDEMANN, PJ_TROE, PJ_SRI, PJ_PLOG, PJ_CHEB = range(7)
PJ_OP_SOURCE, PJ_OP_JACOBIAN, PJ_OP_NEWTON, PJ_OP_VJP, PJ_OP_Y, PJ_OP_FD, PJ_OP_LU = 0, 1, 2, 3, 4, 5, 6
PJ_F64, PJ_F32 = 0, 1
PJ_MAX_SP = 4
PJ_JAC_EXACT, PJ_JAC_APPROX = 0, 1
PJ_LAYOUT_PERCORE, PJ_LAYOUT_TMEM, PJ_LAYOUT_COOP = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_vp = C.c_void_p


class pj_mech_desc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_reactions", C.c_int32),
                ("W", _dp), ("T_mid", _dp), ("nasa_low", _dp), ("nasa_high", _dp),
                ("kind", _ip), ("reversible", _ip), ("reac_sp", _ip), ("reac_nu", _ip),
                ("prod_sp", _ip), ("prod_nu", _ip), ("A", _dp), ("beta", _dp), ("Ea", _dp),
                ("A0", _dp), ("beta0", _dp), ("Ea0", _dp), ("troe", _dp), ("troe_n", _ip),
                ("sri", _dp), ("eff_ptr", _ip), ("eff_sp", _ip), ("eff_val", _dp),
                ("chem", _ip), ("rev_explicit", _ip), ("rev_A", _dp), ("rev_beta", _dp), ("rev_Ea", _dp),
                ("plog_ptr", _ip), ("plog", _dp), ("cheb_ptr", _ip), ("cheb_nT", _ip), ("cheb_nP", _ip),
                ("cheb_range", _dp), ("cheb_coef", _dp)]


class pj_batch(C.Structure):
    _fields_ = [("d_param", C.c_void_p), ("d_phi", C.c_void_p), ("n", C.c_int64), ("ld", C.c_int64),
                ("d_out", C.c_void_p), ("d_dphi", C.c_void_p)]


# name -> (restype, argtypes); every entry point declared in include/pyjac_gb.h
SIGNATURES = {
    "pj_last_error": (C.c_char_p, []),
    "pj_version": (C.c_char_p, []),
    "pj_mech_create": (C.c_int, [C.POINTER(pj_mech_desc), C.POINTER(_vp)]),
    "pj_mech_load": (C.c_int, [C.c_char_p, C.POINTER(_vp)]),
    "pj_mech_free": (C.c_int, [_vp]),
    "pj_mech_info": (C.c_int, [_vp, _ip, _ip, _ip]),
    "pj_sparsity": (C.c_int, [_vp, C.c_int, _ip, _ip]),
    "pj_mech_with_jacobian_form": (C.c_int, [_vp, C.c_int, C.POINTER(_vp)]),
    "pj_mech_jacobian_form": (C.c_int, [_vp, _ip]),
    "pj_mech_arrhenius": (C.c_int, [_vp, _dp, _dp, _dp]),
    "pj_jacobian_layout": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int64, _ip]),
    "pj_debug_word": (C.c_int, [_vp, C.POINTER(C.c_uint32), C.c_int]),
    "pj_debug_build": (C.c_int, [_ip]),
    "pj_debug_set_target": (C.c_int, [_vp, C.c_int, C.c_int32, C.c_int32]),
    "pj_mech_with_arrhenius": (C.c_int, [_vp, _dp, _dp, _dp, C.POINTER(_vp)]),
    "pj_eval_source_terms": (C.c_int, [_vp, C.c_int, C.c_int64, _vp, _vp, C.c_int64, _vp, _vp,
                                       _vp, C.c_size_t, _vp]),
    "pj_eval_jacobian_sparse": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int64, _vp, _vp, C.c_int64, _vp,
                                          _vp, _vp, _vp, C.c_size_t, _vp]),
    "pj_eval_jacobian_dense": (C.c_int, [_vp, C.c_int, C.c_int64, _vp, _vp, C.c_int64, _vp, _vp, _vp,
                                         _vp, C.c_size_t, _vp]),
    "pj_eval_jacobian_fd": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int64, _vp, _vp, C.c_int64, _vp,
                                      _vp, _vp, _vp, C.c_size_t, _vp]),
    "pj_lu_info": (C.c_int, [_vp, _ip, _ip]),
    "pj_lu_pattern": (C.c_int, [_vp, _ip, _ip]),
    "pj_lu_factor": (C.c_int, [_vp, C.c_int, C.c_int64, _vp, C.c_int64, _vp, C.c_double, _vp, _vp, _vp,
                               C.c_size_t, _vp]),
    "pj_lu_solve": (C.c_int, [_vp, C.c_int, C.c_int64, _vp, C.c_int64, _vp, _vp, _vp]),
    "pj_workspace_size": (C.c_int, [_vp, C.c_int, C.c_int64, C.POINTER(C.c_size_t)]),
    "pj_eval_y": (C.c_int, [_vp, C.c_int, C.c_int64, _vp, _vp, C.c_int64, _vp, _vp, _vp, C.c_size_t, _vp]),
    "pj_vjp": (C.c_int, [_vp, C.c_int, C.c_int64, _vp, _vp, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                         C.c_size_t, _vp]),
    "pj_newton_matrix_f32": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int64, _vp, _vp, C.c_int64, _vp, C.c_double,
                                       _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "pj_diag_exp": (C.c_int, [_vp, C.c_int64, _vp, _vp, _vp, _vp]),
    "pj_plan_create": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(pj_batch), C.c_int64, _vp,
                                 C.POINTER(_vp)]),
    "pj_plan_free": (C.c_int, [_vp]),
    "pj_plan_set_config": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "pj_plan_get_config": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int)]),
    "pj_plan_autotune": (C.c_int, [_vp, _vp, C.c_char_p, C.c_int]),
    "pj_plan_run": (C.c_int, [_vp, _vp]),
    "pj_plan_capture": (C.c_int, [_vp, _vp]),
    "pj_plan_launch": (C.c_int, [_vp, _vp]),
    "pj_eval_jacobian_sparse_noalloc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int64, _vp, _vp, C.c_int64, _vp,
                                                  _vp, _vp, _vp]),
    "pj_eval_jacobian_sparse_host": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int64, _vp, _vp, _vp, _vp, _vp,
                                               C.c_int64, _vp]),
}

_lib = None


def lib_path() -> str:
    """The library this process loads: the in-tree build, or the one named by
    PYJAC_GB_LIB (e.g. the bounds-checked build libpyjac_gb_dbg.so)."""
    return os.environ.get("PYJAC_GB_LIB") or _build.LIB


def load(build_if_missing: bool = False):
    """Load the shared library once; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libpyjac_gb.so not built ({path}); run "
                               "`python -m paper_1809_01029_gb300.build` (or __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        if not hasattr(lib, name):
            continue
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class PJError(RuntimeError):
    def __init__(self, code, where):
        msg = load().pj_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with code {code}: {msg}")
        self.code = code


def check(code, where):
    if code != PJ_OK:
        raise PJError(code, where)
    return code
