"""ctypes declarations of the C ABI in include/qmlgb.h.

Loading fails loudly when libqmlgb.so has not been built: there is no
fallback implementation anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
c_char_p = ctypes.c_char_p

QML_OK, QML_EINVAL, QML_ENOTSPD, QML_ENOMEM, QML_ECUDA, QML_ETIMEOUT = range(6)
QML_FP64, QML_SPLIT_BF16 = 0, 1
QML_BASIS_PIXEL, QML_BASIS_HARMONIC, QML_BASIS_AUTO = 0, 1, 2
STATUS_NAMES = {0: "QML_OK", 1: "QML_EINVAL", 2: "QML_ENOTSPD", 3: "QML_ENOMEM", 4: "QML_ECUDA",
                5: "QML_ETIMEOUT"}


class QmlProblem(ctypes.Structure):
    _fields_ = [
        ("has_T", c_int32), ("has_P", c_int32),
        ("npix_T", c_int32), ("npix_P", c_int32),
        ("theta_T", c_void_p), ("phi_T", c_void_p),
        ("theta_P", c_void_p), ("phi_P", c_void_p),
        ("lmin", c_int32), ("lmax", c_int32),
        ("transfer_T", c_void_p), ("transfer_P", c_void_p),
        ("nspec", c_int32), ("spec", c_int32 * 6),
        ("cl_fid", c_void_p), ("N", c_void_p),
        ("precision", c_int32), ("nslices", c_int32),
        ("nbins", c_int32), ("bin_edges", c_void_p),
        ("lmin_sig", c_int32), ("lmax_sig", c_int32), ("basis", c_int32),
    ]


class LnlMask(ctypes.Structure):
    _fields_ = [("prob", QmlProblem), ("maps", c_void_p), ("nmaps", c_int32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "qml_version": (c_int32, []),
    "qml_launch_count": (c_int64, []),
    "qml_last_error": (ctypes.c_char_p, []),
    "qml_ybuild": (c_int32, [ctypes.POINTER(QmlProblem), c_void_p, c_int64, c_void_p]),
    "qml_synthesize": (c_int32, [ctypes.POINTER(QmlProblem), c_void_p, c_void_p, c_int32,
                                 c_void_p, c_void_p]),
    "qml_fisher": (c_int32, [ctypes.POINTER(QmlProblem), c_void_p, ctypes.POINTER(c_void_p),
                             c_void_p]),
    "qml_estimate": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_void_p]),
    "qml_plan_free": (None, [c_void_p]),
    "qml_plan_basis": (c_int32, [c_void_p]),
    "qml_cross": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                            c_void_p, c_void_p]),
    "pix_loglike": (c_int32, [ctypes.POINTER(QmlProblem), c_void_p, c_void_p, c_int32, c_void_p,
                              c_void_p, c_void_p, c_void_p]),
    "pix_loglike_batch": (c_int32, [ctypes.POINTER(LnlMask), c_int32, c_int32, c_void_p, c_void_p,
                                    c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "emu_create": (c_int32, [c_int32, c_void_p, c_void_p, c_int32, c_int32, ctypes.c_uint64,
                             ctypes.POINTER(c_void_p)]),
    "emu_train": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_int32, c_double,
                            c_void_p, c_void_p]),
    "emu_predict": (c_int32, [c_void_p, c_int32, c_void_p, c_double, c_void_p, c_void_p, c_void_p]),
    "emu_param_count": (c_int64, [c_void_p]),
    "qml_tune_set": (c_int32, [c_char_p, c_int64]),
    "qml_tune_get": (c_int32, [c_char_p, c_void_p]),
    "qml_tune_table": (c_int64, [c_void_p, c_int64]),
    "qml_tune_load": (c_int32, [c_char_p]),
    "emu_threshold": (c_int32, [c_void_p, c_double, c_void_p, c_void_p]),
    "emu_params": (c_int32, [c_void_p, c_int32, c_void_p]),
    "emu_baseline": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "emu_loss_grad": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "emu_free": (None, [c_void_p]),
    "qml_potrf": (c_int32, [c_int64, c_void_p, c_int64, c_void_p, c_int32, c_void_p]),
    "qml_potrf_noalloc": (c_int32, [c_int64, c_void_p, c_int64, c_void_p, c_void_p]),
    "qml_trsm": (c_int32, [c_int64, c_int64, c_void_p, c_int64, c_void_p, c_int64, c_int32,
                           c_void_p]),
    "qml_gemm": (c_int32, [c_int32, c_int32, c_int64, c_int64, c_int64, c_double, c_void_p,
                           c_int64, c_void_p, c_int64, c_double, c_void_p, c_int64, c_int32,
                           c_int32, c_void_p]),
}

_lib = None


def load(path: str = LIB) -> ctypes.CDLL:
    """Load libqmlgb.so (once) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is not built; run paper_2605_21149_gb300.build.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(SIGNATURES)
