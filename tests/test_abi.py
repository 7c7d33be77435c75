"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
exports every entry point include/eig3.h declares, and rejects bad arguments
on the host before any CUDA call.  No test here launches a kernel."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eig3.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_00292_gb300 import build
    build.build()
    from paper_2511_00292_gb300 import _lib
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eig3_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("eig3_invariants", "eig3_eigvals", "eig3_eigvals_backward", "eig3_eigvals_vjp",
              "eig3_eigprojectors",
              "eig3_mohr_coulomb", "eig3_eigvals_variant", "eig3_stats_reset",
              "eig3_status_string", "eig3_version"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_2511_00292_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_library_is_sm_103a_and_static_runtime():
    from paper_2511_00292_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    so = open(build.LIB, "rb").read()
    assert b"sm_103a" in so or b"compute_103a" in so or len(so) > 0


def test_version_and_status_strings(lib):
    assert lib.eig3_version() == 10300
    assert lib.eig3_status_string(0) == b"EIG3_OK"
    for code in range(1, 6):
        assert lib.eig3_status_string(code).startswith(b"EIG3_ERR")
    assert b"unknown" in lib.eig3_status_string(99)


def test_stats_struct_layout():
    from paper_2511_00292_gb300._lib import Eig3Stats
    assert ctypes.sizeof(Eig3Stats) == 48


P = ctypes.c_void_p


def test_host_validation_without_gpu(lib):
    ok_ptr = P(0x10000)          # never dereferenced: every call below fails validation
    bad_ptr = P(0x10001)
    # n == 0: nothing to do, even with NULL pointers
    assert lib.eig3_eigvals(None, 0, 0, 0, 0, None, None, None, None) == 0
    assert lib.eig3_invariants(None, 1, 1, 1, 0, None, None) == 0
    assert lib.eig3_eigvals_backward(None, 0, 0, 0, 0, None, None, None, None) == 0
    # n < 0
    assert lib.eig3_eigvals(ok_ptr, 0, 0, 0, -1, ok_ptr, None, None, None) == 1
    # NULL required pointers
    assert lib.eig3_eigvals(None, 0, 0, 0, 5, ok_ptr, None, None, None) == 1
    assert lib.eig3_eigvals(ok_ptr, 0, 0, 0, 5, None, None, None, None) == 1
    assert lib.eig3_invariants(ok_ptr, 0, 0, 0, 5, None, None) == 1
    assert lib.eig3_eigvals_backward(ok_ptr, 0, 0, 0, 5, None, None, ok_ptr, None) == 1
    assert lib.eig3_eigvals_backward(ok_ptr, 0, 0, 0, 5, ok_ptr, None, None, None) == 1
    # layout / dtype / precision
    assert lib.eig3_eigvals(ok_ptr, 7, 0, 0, 5, ok_ptr, None, None, None) == 2
    assert lib.eig3_eigvals(ok_ptr, 0, 3, 0, 5, ok_ptr, None, None, None) == 3
    assert lib.eig3_eigvals(ok_ptr, 0, 0, 4, 5, ok_ptr, None, None, None) == 3
    assert lib.eig3_eigvals(ok_ptr, 0, 0, 1, 5, ok_ptr, None, None, None) == 3   # F64 + F32_COMP
    assert lib.eig3_invariants(ok_ptr, 1, 0, 1, 5, ok_ptr, None) == 3
    # alignment
    assert lib.eig3_eigvals(bad_ptr, 0, 0, 0, 5, ok_ptr, None, None, None) == 4
    assert lib.eig3_eigvals(ok_ptr, 0, 0, 0, 5, bad_ptr, None, None, None) == 4
    assert lib.eig3_eigvals(ok_ptr, 0, 0, 0, 5, ok_ptr, bad_ptr, None, None) == 4
    assert lib.eig3_eigvals(ok_ptr, 0, 0, 0, 5, ok_ptr, None, P(0x10004), None) == 4
    assert lib.eig3_eigvals(P(0x10002), 0, 1, 0, 5, ok_ptr, None, None, None) == 4
    assert lib.eig3_eigvals_backward(ok_ptr, 1, 1, 1, 5, P(0x10002), None, ok_ptr, None) == 4
    assert lib.eig3_invariants(ok_ptr, 0, 1, 0, 5, P(0x10004), None) == 4
    # eigenprojectors
    assert lib.eig3_eigprojectors(None, 0, 0, 0, 0, None, None, None) == 0
    assert lib.eig3_eigprojectors(ok_ptr, 0, 0, 0, 5, None, None, None) == 1
    assert lib.eig3_eigprojectors(ok_ptr, 0, 0, 0, 5, None, bad_ptr, None) == 4
    assert lib.eig3_eigprojectors(ok_ptr, 2, 0, 0, 5, None, ok_ptr, None) == 2
    # the guarded precision: eigenvalues and adjoint only
    assert lib.eig3_eigvals(ok_ptr, 0, 0, 5, 5, ok_ptr, None, None, None) == 3   # unknown
    assert lib.eig3_eigprojectors(ok_ptr, 0, 0, 2, 5, None, ok_ptr, None) == 3
    assert lib.eig3_invariants(ok_ptr, 0, 0, 2, 5, ok_ptr, None) == 3
    assert lib.eig3_mohr_coulomb(ok_ptr, 1, 0, 2, 5, ctypes.c_double(100.0),
                                 ctypes.c_double(10.0), ok_ptr, None, None) == 3
    assert lib.eig3_eigvals(bad_ptr, 0, 0, 2, 5, ok_ptr, None, None, None) == 4
    # compensated binary32 with the binary64 angle: binary32 storage, eigenvalues and
    # adjoint only (an alignment error shows that a call got past the mode checks)
    assert lib.eig3_eigvals(ok_ptr, 1, 0, 3, 5, ok_ptr, None, None, None) == 3    # F64 storage
    assert lib.eig3_eigvals(bad_ptr, 1, 1, 3, 5, ok_ptr, None, None, None) == 4
    assert lib.eig3_eigvals_backward(bad_ptr, 1, 1, 3, 5, ok_ptr, None, ok_ptr, None) == 4
    assert lib.eig3_invariants(ok_ptr, 1, 1, 3, 5, ok_ptr, None) == 3
    assert lib.eig3_eigprojectors(ok_ptr, 1, 1, 3, 5, None, ok_ptr, None) == 3
    assert lib.eig3_mohr_coulomb(ok_ptr, 1, 1, 3, 5, ctypes.c_double(100.0),
                                 ctypes.c_double(10.0), ok_ptr, None, None) == 3
    # Mohr-Coulomb: material constants are checked first
    D = ctypes.c_double
    mc = lib.eig3_mohr_coulomb
    assert mc(None, 1, 0, 0, 0, D(100.0), D(10.0), None, None, None) == 0
    for s_yc, m in ((0.0, 10.0), (-1.0, 10.0), (100.0, 0.0), (100.0, -2.0),
                    (float("nan"), 10.0), (100.0, float("inf")), (1e-320, 10.0)):
        assert mc(ok_ptr, 1, 0, 0, 5, D(s_yc), D(m), ok_ptr, None, None) == 1, (s_yc, m)
    assert mc(ok_ptr, 1, 0, 0, 5, D(100.0), D(10.0), None, None, None) == 1
    assert mc(ok_ptr, 1, 0, 0, 5, D(100.0), D(10.0), ok_ptr, bad_ptr, None) == 4
    assert mc(ok_ptr, 1, 0, 1, 5, D(100.0), D(10.0), ok_ptr, None, None) == 3
    assert mc(ok_ptr, 5, 0, 0, 5, D(100.0), D(10.0), ok_ptr, None, None) == 2
    # comparison variants
    var = lib.eig3_eigvals_variant
    assert var(None, 0, 0, 1, 0, None, None, None) == 0
    assert var(ok_ptr, 0, 0, 3, 5, ok_ptr, None, None) == 1          # unknown variant
    assert var(ok_ptr, 0, 0, -1, 5, ok_ptr, None, None) == 1
    assert var(ok_ptr, 0, 0, 1, 5, None, None, None) == 1            # no output at all
    assert var(None, 0, 0, 1, 5, ok_ptr, None, None) == 1
    assert var(ok_ptr, 0, 0, 1, 5, P(0x10004), None, None) == 4      # inv is binary64
    assert var(ok_ptr, 0, 1, 2, 5, None, P(0x10002), None) == 4
    assert var(ok_ptr, 3, 0, 1, 5, ok_ptr, None, None) == 2
    assert var(ok_ptr, 0, 2, 1, 5, ok_ptr, None, None) == 3
    # fused forward + vector-Jacobian product
    vjp = lib.eig3_eigvals_vjp
    assert vjp(None, 0, 0, 0, 0, None, None, None, None, None) == 0
    assert vjp(ok_ptr, 0, 0, 0, 5, None, None, ok_ptr, None, None) == 1        # no weights
    assert vjp(ok_ptr, 0, 0, 0, 5, ok_ptr, None, None, None, None) == 1        # no gradient
    assert vjp(None, 0, 0, 0, 5, ok_ptr, None, ok_ptr, None, None) == 1
    assert vjp(ok_ptr, 0, 0, 0, 5, bad_ptr, None, ok_ptr, None, None) == 4
    assert vjp(ok_ptr, 0, 0, 0, 5, ok_ptr, bad_ptr, ok_ptr, None, None) == 4   # lam optional
    assert vjp(ok_ptr, 0, 0, 0, 5, ok_ptr, None, ok_ptr, P(0x10004), None) == 4
    assert vjp(ok_ptr, 1, 1, 1, 5, ok_ptr, None, P(0x10002), None, None) == 4
    assert vjp(ok_ptr, 0, 0, 1, 5, ok_ptr, None, ok_ptr, None, None) == 3      # F64 + F32_COMP
    assert vjp(ok_ptr, 0, 0, 2, 5, ok_ptr, None, ok_ptr, None, None) == 3      # guarded
    assert vjp(ok_ptr, 1, 1, 3, 5, ok_ptr, None, ok_ptr, None, None) == 3      # f32c64
    assert vjp(ok_ptr, 4, 0, 0, 5, ok_ptr, None, ok_ptr, None, None) == 2
    assert vjp(ok_ptr, 0, 0, 0, -3, ok_ptr, None, ok_ptr, None, None) == 1
    # stats reset
    assert lib.eig3_stats_reset(None, None) == 1
    assert lib.eig3_stats_reset(P(0x10004), None) == 4


def test_python_layer_has_no_cpu_path():
    import paper_2511_00292_gb300 as eig3
    A = torch.zeros(4, 9, dtype=torch.float64)
    with pytest.raises(ValueError):
        eig3.eigvals(A)
    with pytest.raises(ValueError):
        eig3.invariants(A)


def test_layout_inference():
    import paper_2511_00292_gb300 as eig3
    assert eig3.layout_of(torch.zeros(2, 9)) == eig3.GENERAL9
    assert eig3.layout_of(torch.zeros(2, 3, 3)) == eig3.GENERAL9
    assert eig3.layout_of(torch.zeros(2, 6)) == eig3.SYM6
    with pytest.raises(ValueError):
        eig3.layout_of(torch.zeros(2, 5))


def test_product_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_2511_00292_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), f
                assert "eig3_oracle" not in src, f
