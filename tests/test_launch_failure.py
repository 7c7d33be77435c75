"""Failure detection on the host: when a launch fails (here: no usable GPU or
driver, so the CUDA runtime refuses every launch), each entry point returns
EIG3_ERR_CUDA after its argument checks pass -- a status, never a crash or a
hang -- and eig3_status_string explains it.

The calls below pass dummy (aligned) pointers that no kernel may ever
dereference, so the test runs only where no GPU is visible; with one, it is
skipped (the GPU tests cover the successful launches)."""
import ctypes
import glob

import pytest
import torch

P = ctypes.c_void_p
D = ctypes.c_double
ERR_CUDA = 5


def gpu_visible():
    return torch.cuda.is_available() or bool(glob.glob("/dev/nvidia[0-9]*"))


@pytest.fixture(scope="module")
def lib():
    if gpu_visible():
        pytest.skip("dummy-pointer launches must never reach a real GPU")
    from paper_2511_00292_gb300 import build
    build.build()
    from paper_2511_00292_gb300 import _lib
    return _lib.load()


def test_every_entry_point_reports_a_failed_launch(lib):
    ok = P(0x10000)
    calls = {
        "eig3_stats_reset": lambda: lib.eig3_stats_reset(ok, None),
        "eig3_invariants f64": lambda: lib.eig3_invariants(ok, 0, 0, 0, 5, ok, None),
        "eig3_invariants f32c": lambda: lib.eig3_invariants(ok, 1, 1, 1, 5, ok, None),
        "eig3_eigvals f64": lambda: lib.eig3_eigvals(ok, 0, 0, 0, 5, ok, None, None, None),
        "eig3_eigvals f32c": lambda: lib.eig3_eigvals(ok, 1, 1, 1, 5, ok, ok, ok, None),
        "eig3_eigvals f32c64": lambda: lib.eig3_eigvals(ok, 1, 1, 3, 5, ok, None, None, None),
        "eig3_eigvals guarded": lambda: lib.eig3_eigvals(ok, 0, 0, 2, 5, ok, None, None, None),
        "eig3_eigvals_backward": lambda: lib.eig3_eigvals_backward(ok, 0, 0, 0, 5, ok, ok, ok,
                                                                   None),
        "eig3_eigvals_vjp f64": lambda: lib.eig3_eigvals_vjp(ok, 0, 0, 0, 5, ok, ok, ok, ok,
                                                             None),
        "eig3_eigvals_vjp f32c": lambda: lib.eig3_eigvals_vjp(ok, 1, 1, 1, 5, ok, None, ok, None,
                                                              None),
        "eig3_eigprojectors": lambda: lib.eig3_eigprojectors(ok, 0, 0, 0, 5, ok, ok, None),
        "eig3_mohr_coulomb": lambda: lib.eig3_mohr_coulomb(ok, 1, 0, 0, 5, D(100.0), D(10.0),
                                                           ok, ok, None),
        "eig3_eigvals_variant": lambda: lib.eig3_eigvals_variant(ok, 0, 0, 1, 5, ok, ok, None),
    }
    got = {name: call() for name, call in calls.items()}
    assert got == {name: ERR_CUDA for name in calls}
    assert b"launch failed" in lib.eig3_status_string(ERR_CUDA)


def test_argument_errors_still_come_first(lib):
    """The host checks run before any CUDA call: a bad argument is reported as
    such even where every launch would fail."""
    ok, bad = P(0x10000), P(0x10001)
    assert lib.eig3_eigvals(ok, 0, 0, 0, 0, ok, None, None, None) == 0     # n = 0: no launch
    assert lib.eig3_eigvals(bad, 0, 0, 0, 5, ok, None, None, None) == 4   # alignment
    assert lib.eig3_eigvals(ok, 9, 0, 0, 5, ok, None, None, None) == 2    # layout
