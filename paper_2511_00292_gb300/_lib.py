"""ctypes binding of libeig3.so (include/eig3.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

# Names of the C ABI (include/eig3.h), in declaration order.
EXPORTS = (
    "eig3_invariants",
    "eig3_eigvals",
    "eig3_eigvals_backward",
    "eig3_eigvals_vjp",
    "eig3_eigprojectors",
    "eig3_mohr_coulomb",
    "eig3_eigvals_variant",
    "eig3_stats_reset",
    "eig3_status_string",
    "eig3_version",
)

GENERAL9, SYM6 = 0, 1
F64, F32 = 0, 1
PREC_F64, PREC_F32_COMP, PREC_F64_GUARDED, PREC_F32_COMP_A64 = 0, 1, 2, 3
VARIANT_PRESENT, VARIANT_NAIVE, VARIANT_NAIVE_TENSOR = 0, 1, 2
STATUS = {0: "EIG3_OK", 1: "EIG3_ERR_ARG", 2: "EIG3_ERR_LAYOUT", 3: "EIG3_ERR_DTYPE",
          4: "EIG3_ERR_ALIGN", 5: "EIG3_ERR_CUDA"}


class Eig3Stats(ctypes.Structure):
    """Mirror of eig3_stats (48 bytes)."""
    _fields_ = [
        ("n_delta_clamped", ctypes.c_ulonglong),
        ("n_j2_clamped", ctypes.c_ulonglong),
        ("n_nonfinite", ctypes.c_ulonglong),
        ("min_disc_ratio", ctypes.c_double),
        ("max_abs_lambda", ctypes.c_double),
        ("n_guarded", ctypes.c_ulonglong),
    ]


class Eig3Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {_lib_status_string(status)}")


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libeig3.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build the CUDA library first "
                "(paper_2511_00292_gb300.build.build() or __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.eig3_invariants.argtypes = [P, I, I, I, I64, P, P]
        lib.eig3_invariants.restype = I
        lib.eig3_eigvals.argtypes = [P, I, I, I, I64, P, P, P, P]
        lib.eig3_eigvals.restype = I
        lib.eig3_eigvals_backward.argtypes = [P, I, I, I, I64, P, P, P, P]
        lib.eig3_eigvals_backward.restype = I
        lib.eig3_eigvals_vjp.argtypes = [P, I, I, I, I64, P, P, P, P, P]
        lib.eig3_eigvals_vjp.restype = I
        lib.eig3_eigprojectors.argtypes = [P, I, I, I, I64, P, P, P]
        lib.eig3_eigprojectors.restype = I
        lib.eig3_mohr_coulomb.argtypes = [P, I, I, I, I64, ctypes.c_double, ctypes.c_double, P,
                                          P, P]
        lib.eig3_mohr_coulomb.restype = I
        lib.eig3_eigvals_variant.argtypes = [P, I, I, I, I64, P, P, P]
        lib.eig3_eigvals_variant.restype = I
        lib.eig3_stats_reset.argtypes = [P, P]
        lib.eig3_stats_reset.restype = I
        lib.eig3_status_string.argtypes = [I]
        lib.eig3_status_string.restype = ctypes.c_char_p
        lib.eig3_version.argtypes = []
        lib.eig3_version.restype = I
        _lib = lib
        return lib


def _lib_status_string(status: int) -> str:
    try:
        return load().eig3_status_string(int(status)).decode()
    except Exception:  # pragma: no cover - only when the library cannot load
        return STATUS.get(int(status), f"status {status}")


def check(status: int, where: str) -> None:
    if status != 0:
        raise Eig3Error(status, where)
