"""FP64 CPU oracle for the closed-form 3x3 eigenvalue method (arXiv 2511.00292).

TEST INFRASTRUCTURE ONLY.  The product (the CUDA library and its Python
binding) never imports this package.  The test suite, the smoke check and the
CPU-baseline leg of ``bench.py`` are its only users.

The arithmetic lives in ``eig3_oracle.c`` (plain scalar C, binary64, no FMA
contraction, evaluated in the paper's order).  This module compiles it with
gcc on first use and marshals numpy arrays through ctypes.

Function map (paper sections):
    invariants        Algorithms 1, 2, 4, 5 -> (I1, J2, J3, Delta)
    invariants_naive  Algorithm 3, the naive J3 monomial sum, 4 J2^3 - 27 J3^2
    eigvals           Algorithm 6 on the stable invariants
    eigvals_naive     Algorithm 6 on the naive invariants
    invariants_naive_tensor / eigvals_naive_tensor
                      tr(S S)/2 and det S of S = dev(A), then Algorithm 6
    eigvals_grad      d lambda_k / dA = l r^T / (l^T r)  (Section 1, E_k^T)
    eigval_jacobians  the three d lambda_k / dA separately
    mohr_coulomb      the yield function of the application section (+ gradient)
    bounds            first-order stability bounds, C = 1, Frobenius norm
    eigvals_mt        eigvals on POSIX threads, for timing on host cores
    eigvals_exact     (oracle/exact.py) the exact eigenvalues of the stored
                      matrix: roots of its exact characteristic polynomial,
                      the reference the stability bounds are stated against
    invariants_exact  (oracle/exact.py) the exact invariants of the stored matrix
    opcount           the operations of one oracle function on one matrix,
                      counted by compiling eig3_oracle.c with an op-counting
                      scalar type (opcount.cpp, g++)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eig3_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libeig3_oracle.so")
_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_LIB = os.path.join(_BUILD, "libeig3_opcount.so")

GENERAL9 = 0
SYM6 = 1
U64 = 2.0 ** -53
U32 = 2.0 ** -24

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _build_opcount() -> str:
    """Compile opcount.cpp (the oracle's source with a counting scalar) with g++."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_OPC_SRC))
    if not os.path.exists(_OPC_LIB) or os.path.getmtime(_OPC_LIB) < newest:
        tmp = _OPC_LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c++17", "-I", _HERE, "-o", tmp, _OPC_SRC, "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OPC_LIB)
    return _OPC_LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            I = ctypes.c_int
            D = ctypes.c_double
            for name in ("eig3o_invariants_batch", "eig3o_invariants_naive_batch",
                         "eig3o_invariants_naive_tensor_batch", "eig3o_eigvals_batch",
                         "eig3o_eigvals_naive_batch", "eig3o_eigvals_naive_tensor_batch"):
                getattr(lib, name).argtypes = [P, I64, I, P]
                getattr(lib, name).restype = None
            lib.eig3o_eigvals_grad_batch.argtypes = [P, P, I64, I, P]
            lib.eig3o_eigvals_grad_batch.restype = None
            lib.eig3o_mohr_coulomb_batch.argtypes = [P, I64, I, D, D, P, P]
            lib.eig3o_mohr_coulomb_batch.restype = None
            lib.eig3o_eigval_jacobians_batch.argtypes = [P, I64, I, P]
            lib.eig3o_eigval_jacobians_batch.restype = None
            lib.eig3o_bounds_batch.argtypes = [P, P, I64, I, D, P]
            lib.eig3o_bounds_batch.restype = None
            lib.eig3o_eigvals_batch_mt.argtypes = [P, I64, I, P, I]
            lib.eig3o_eigvals_batch_mt.restype = I
            _lib = lib
    return _lib


def _as_input(X, layout: int) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    width = 9 if layout == GENERAL9 else 6
    if X.ndim == 1:
        X = X.reshape(1, -1)
    X = X.reshape(-1, width)
    return np.ascontiguousarray(X)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def invariants(X, layout: int = GENERAL9) -> np.ndarray:
    """(n, 4) array of (I1, J2, J3, Delta) by Algorithms 1, 2, 4 and 5."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 4), dtype=np.float64)
    _load().eig3o_invariants_batch(_ptr(X), X.shape[0], layout, _ptr(out))
    return out


def invariants_naive(X, layout: int = GENERAL9) -> np.ndarray:
    """(n, 4) array of (I1, J2, J3, Delta) by the naive monomial sums."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 4), dtype=np.float64)
    _load().eig3o_invariants_naive_batch(_ptr(X), X.shape[0], layout, _ptr(out))
    return out


def invariants_naive_tensor(X, layout: int = GENERAL9) -> np.ndarray:
    """(n, 4) array of (I1, J2, J3, Delta) from S = dev(A): tr(S S)/2, det S."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 4), dtype=np.float64)
    _load().eig3o_invariants_naive_tensor_batch(_ptr(X), X.shape[0], layout, _ptr(out))
    return out


def eigvals(X, layout: int = GENERAL9) -> np.ndarray:
    """(n, 3) ascending eigenvalues by Algorithm 6 on the stable invariants."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 3), dtype=np.float64)
    _load().eig3o_eigvals_batch(_ptr(X), X.shape[0], layout, _ptr(out))
    return out


def eigvals_naive(X, layout: int = GENERAL9) -> np.ndarray:
    """(n, 3) eigenvalues by Algorithm 6 on the naive invariants."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 3), dtype=np.float64)
    _load().eig3o_eigvals_naive_batch(_ptr(X), X.shape[0], layout, _ptr(out))
    return out


def eigvals_naive_tensor(X, layout: int = GENERAL9) -> np.ndarray:
    """(n, 3) eigenvalues by Algorithm 6 on the naive tensor invariants."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 3), dtype=np.float64)
    _load().eig3o_eigvals_naive_tensor_batch(_ptr(X), X.shape[0], layout, _ptr(out))
    return out


def eigvals_grad(X, gbar, layout: int = GENERAL9) -> np.ndarray:
    """Gradient of sum_k gbar_k lambda_k with respect to the stored entries."""
    X = _as_input(X, layout)
    g = np.ascontiguousarray(np.asarray(gbar, dtype=np.float64).reshape(-1, 3))
    if g.shape[0] != X.shape[0]:
        raise ValueError("gbar must have one row of 3 per matrix")
    out = np.empty_like(X)
    _load().eig3o_eigvals_grad_batch(_ptr(X), _ptr(g), X.shape[0], layout, _ptr(out))
    return out


def eigval_jacobians(X, layout: int = GENERAL9) -> np.ndarray:
    """(n, 3, 9): d lambda_k / dA_ij = l_i r_j / (l^T r) for each ascending
    eigenvalue k, with respect to the 9 entries of the (expanded) matrix."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 27), dtype=np.float64)
    _load().eig3o_eigval_jacobians_batch(_ptr(X), X.shape[0], layout, _ptr(out))
    return out.reshape(-1, 3, 9)


def mohr_coulomb(X, s_yc: float = 100.0, m: float = 10.0, layout: int = GENERAL9,
                 grad: bool = False):
    """Mohr-Coulomb yield value per matrix (Section "Application"), literal
    max over the three principal-stress pairs; with grad=True also its
    gradient with respect to the stored entries."""
    X = _as_input(X, layout)
    f = np.empty(X.shape[0], dtype=np.float64)
    g = np.empty_like(X) if grad else None
    _load().eig3o_mohr_coulomb_batch(_ptr(X), X.shape[0], layout, float(s_yc), float(m), _ptr(f),
                                     _ptr(g) if grad else None)
    return (f, g) if grad else f


def bounds(X, kappa=None, layout: int = GENERAL9, u: float = U64) -> np.ndarray:
    """(n, 5) first-order bounds (I1, J2, J3, Delta, lambda), C = 1, Frobenius."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 5), dtype=np.float64)
    if kappa is None:
        kp = None
    else:
        k = np.ascontiguousarray(np.broadcast_to(np.asarray(kappa, dtype=np.float64),
                                                 (X.shape[0],)))
        kp = _ptr(k)
    _load().eig3o_bounds_batch(_ptr(X), kp, X.shape[0], layout, float(u), _ptr(out))
    return out


def eigvals_mt(X, layout: int = GENERAL9, nthreads: int | None = None):
    """eigvals on POSIX threads; returns (lam, threads_used)."""
    X = _as_input(X, layout)
    out = np.empty((X.shape[0], 3), dtype=np.float64)
    nt = int(nthreads or os.cpu_count() or 1)
    used = _load().eig3o_eigvals_batch_mt(_ptr(X), X.shape[0], layout, _ptr(out), nt)
    return out, int(used)


_OPC = {"eigvals": 0, "invariants": 1, "I1": 2, "J2": 3, "J3": 4, "Delta": 5,
        "eigvals_from_invariants": 6}
_OPC_FIELDS = ("add", "mul", "div", "neg", "sqrt", "atan2", "cos", "cmp", "abs")
_opc_lib = None


def opcount(function: str, a) -> tuple[dict, np.ndarray]:
    """(counts, results) of one oracle function on one general 9-entry matrix
    (for "eigvals_from_invariants": the four invariants), from the oracle's
    source compiled with an op-counting scalar type.  counts maps each kind of
    operation (add includes subtraction) to how many the function performed."""
    global _opc_lib
    with _lock:
        if _opc_lib is None:
            lib = ctypes.CDLL(_build_opcount())
            lib.eig3o_opcount.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]
            lib.eig3o_opcount.restype = ctypes.c_int
            _opc_lib = lib
    x = np.zeros(9)
    v = np.asarray(a, dtype=np.float64).reshape(-1)
    x[:v.size] = v
    counts = np.zeros(9, dtype=np.int64)
    res = np.full(4, np.nan)
    if _opc_lib.eig3o_opcount(_OPC[function], _ptr(x), _ptr(counts), _ptr(res)) != 0:
        raise ValueError(function)
    n = {"eigvals": 3, "invariants": 4, "eigvals_from_invariants": 3}.get(function, 1)
    return dict(zip(_OPC_FIELDS, (int(c) for c in counts))), res[:n]


def sym6_to_general9(S) -> np.ndarray:
    """Expand (A00, A11, A22, A12, A02, A01) rows to row-major 9-entry rows."""
    S = np.asarray(S, dtype=np.float64).reshape(-1, 6)
    A = np.empty((S.shape[0], 9), dtype=np.float64)
    A[:, 0] = S[:, 0]; A[:, 1] = S[:, 5]; A[:, 2] = S[:, 4]
    A[:, 3] = S[:, 5]; A[:, 4] = S[:, 1]; A[:, 5] = S[:, 3]
    A[:, 6] = S[:, 4]; A[:, 7] = S[:, 3]; A[:, 8] = S[:, 2]
    return A


from .exact import (eigvals_exact, invariants_exact, map_eigvals_exact,  # noqa: E402
                    map_invariants_exact)  # (pure Python, no compiled part)
