"""ctypes binding of liblbm.so (argument marshalling only).

The shared library is built in-tree by ``paper_1603_09577_gb300.build``. If it
is missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY=checked selects the bounds-checked build (see lbm_debug_flags)
LIB_PATH = os.path.join(HERE, "liblbm_checked.so" if os.environ.get("LBM_LIBRARY") == "checked" else "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_EUNSUPPORTED = range(6)
LBM_F64, LBM_F32, LBM_BF16S = 0, 1, 2
LBM_PERIODIC, LBM_ABB, LBM_NEE = 0, 1, 2
LBM_SCHEME_B, LBM_SCHEME_A = 0, 1
PREC = {"f64": LBM_F64, "f32": LBM_F32, "bf16s": LBM_BF16S}


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


class Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("prec", ctypes.c_int),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("phi_wall", ctypes.c_double * 4), ("steps_per_pass", ctypes.c_int),
                ("per_cell_K", ctypes.c_int), ("kernel_variant", ctypes.c_int),
                ("block_rows", ctypes.c_int), ("scheme", ctypes.c_int)]


class Coeffs(ctypes.Structure):
    _fields_ = [("conv", ctypes.c_int), ("u", ctypes.c_double * 2), ("diff", ctypes.c_int),
                ("K", ctypes.c_double * 3), ("s", ctypes.c_double * 9),
                ("r0", ctypes.c_double), ("r1", ctypes.c_double),
                ("src_family", ctypes.c_int), ("power", ctypes.c_int), ("b", ctypes.c_double),
                ("Dm", ctypes.c_double * 3), ("cfree", ctypes.c_int)]


class Desc3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("prec", ctypes.c_int),
                ("block_rows", ctypes.c_int), ("bc", ctypes.c_int * 3), ("phi_wall", ctypes.c_double * 6)]


class Coeffs3(ctypes.Structure):
    _fields_ = [("conv", ctypes.c_int), ("u", ctypes.c_double * 3), ("diff", ctypes.c_int),
                ("K", ctypes.c_double * 6), ("s0", ctypes.c_double), ("se", ctypes.c_double),
                ("r0", ctypes.c_double), ("r1", ctypes.c_double)]


_lock = threading.Lock()
_lib = None

_VP, _SZ, _I, _DP = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "lbm_workspace_size": [ctypes.POINTER(Desc), ctypes.POINTER(_SZ)],
    "lbm_create": [ctypes.POINTER(_VP), ctypes.POINTER(Desc), _VP, _SZ],
    "lbm_destroy": [_VP],
    "lbm_set_coeffs": [_VP, ctypes.POINTER(Coeffs)],
    "lbm_set_K_field": [_VP, _VP, _VP],
    "lbm_set_phi": [_VP, _VP, _I, _VP],
    "lbm_set_phi_host": [_VP, _VP, _I, _VP],
    "lbm_step": [_VP, _I, _VP],
    "lbm_set_dirichlet": [_VP, _VP, _I],
    "lbm_get_phi": [_VP, _VP, _I, _VP],
    "lbm_get_phi_host": [_VP, _VP, _I, _VP],
    "lbm_reduce": [_VP, _VP, _VP, _VP],
    "lbm_state_bytes": [_VP, ctypes.POINTER(_SZ)],
    "lbm_save": [_VP, _VP, _VP],
    "lbm_load": [_VP, _VP, _VP],
    "lbm_reduce_field_noalloc": [_VP, _VP, ctypes.c_longlong, _VP, _VP],
    "lbm_check_finite": [_VP, ctypes.POINTER(ctypes.c_longlong), _VP],
    "lbm_debug_flags": [_VP, ctypes.POINTER(_I), _VP],
    "lbm_build_checked": [],
    "lbm_debug_wait_probe": [ctypes.c_uint, _VP, _VP],
    "lbm_probe_fp64": [_I, _I, _I, _VP, ctypes.POINTER(ctypes.c_longlong), _VP],
    "lbm_adjoint_workspace_size": [_VP, ctypes.POINTER(_SZ)],
    "lbm_adjoint_begin": [_VP, _VP, _SZ, _VP, _I, _VP],
    "lbm_adjoint_step": [_VP, _VP, _VP],
    "lbm_adjoint_end": [_VP, _VP, _I, _VP, _VP, _VP, _VP],
    "lbm_adjoint_segment": [_VP, _VP, _I, _VP, _SZ, _VP],
    "lbm3_workspace_size": [ctypes.POINTER(Desc3), ctypes.POINTER(_SZ)],
    "lbm3_create": [ctypes.POINTER(_VP), ctypes.POINTER(Desc3), _VP, _SZ],
    "lbm3_destroy": [_VP],
    "lbm3_set_coeffs": [_VP, ctypes.POINTER(Coeffs3)],
    "lbm3_set_phi": [_VP, _VP, _I, _VP],
    "lbm3_step": [_VP, _I, _VP],
    "lbm3_get_phi": [_VP, _VP, _I, _VP],
    "lbm3_state_bytes": [_VP, ctypes.POINTER(_SZ)],
    "lbm3_save": [_VP, _VP, _VP],
    "lbm3_load": [_VP, _VP, _VP],
    "lbm3_reduce": [_VP, _VP, _VP, _VP],
    "lbm3_debug_flags": [_VP, ctypes.POINTER(_I), _VP],
    "lbm_ensemble_workspace_size": [_I, _VP, _VP, ctypes.POINTER(_SZ)],
    "lbm_ensemble_create": [ctypes.POINTER(_VP), _I, _VP, _VP, _VP, _VP, _SZ, _VP],
    "lbm_ensemble_destroy": [_VP],
    "lbm_ensemble_info": [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "lbm_ensemble_set_phi": [_VP, _VP, _I, _VP],
    "lbm_ensemble_step": [_VP, _I, _I, _VP],
    "lbm_ensemble_capture": [_VP, _I, _VP],
    "lbm_ensemble_configure": [_VP, _I],
    "lbm_ensemble_set_persistent": [_VP, _I],
    "lbm_ensemble_set_tiles": [_VP, _I],
    "lbm_ensemble_replay": [_VP, _VP],
    "lbm_ensemble_get_phi": [_VP, _VP, _I, _VP],
    "lbm_ensemble_reduce": [_VP, _VP, _VP, _VP],
    "lbm_ensemble_debug_flags": [_VP, ctypes.POINTER(_I), _VP],
}


def lib():
    """Load liblbm.so; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.lbm_last_error.argtypes = []
            L.lbm_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != LBM_OK:
        raise LBMError(rc, lib().lbm_last_error().decode(errors="replace"))


def declared_symbols() -> list[str]:
    return list(SIGNATURES) + ["lbm_last_error"]
