"""The integer-pipe binary64 multiplication (csrc/eig3_dmul.cuh), compiled for
the host from the same header, against the host's IEEE 754 multiplication bit
for bit: random bit patterns (every exponent, infinities and NaNs included),
products that overflow or underflow gradually, subnormal operands, exact ties,
the boundary of the normal range and the special values.  A NaN product only
has to be a NaN (IEEE 754 leaves its payload open)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2511_00292_gb300", "csrc")
N = 1 << 20


@pytest.fixture(scope="module")
def dmul(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    so = str(tmp_path_factory.mktemp("dmul") / "libdmul.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "dmul_host.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)

    def f(x, y):
        x = np.ascontiguousarray(x, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        out = np.empty_like(x)
        lib.dmul_batch(x.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p),
                       out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(x.size))
        return out
    return f


def check(dmul, x, y):
    with np.errstate(all="ignore"):
        ref = x * y
    got = dmul(x, y)
    same = (ref.view(np.uint64) == got.view(np.uint64)) | (np.isnan(ref) & np.isnan(got))
    bad = np.flatnonzero(~same)
    assert bad.size == 0, [(x[i].hex(), y[i].hex(), ref[i].hex(), got[i].hex()) for i in bad[:4]]


def test_random_bit_patterns(dmul):
    rng = np.random.default_rng(11)
    x = rng.integers(0, 2 ** 64, N, dtype=np.uint64).view(np.float64)
    y = rng.integers(0, 2 ** 64, N, dtype=np.uint64).view(np.float64)
    check(dmul, x, y)


def test_normal_range(dmul):
    rng = np.random.default_rng(12)
    x = rng.standard_normal(N) * 2.0 ** rng.integers(-200, 200, N)
    y = rng.standard_normal(N) * 2.0 ** rng.integers(-200, 200, N)
    check(dmul, x, y)


def test_gradual_underflow_and_overflow(dmul):
    rng = np.random.default_rng(13)
    e = rng.integers(-1140, -960, N)
    x = rng.uniform(1, 2, N) * 2.0 ** (e // 2)
    y = -rng.uniform(1, 2, N) * 2.0 ** (e - e // 2)
    check(dmul, x, y)
    x = rng.uniform(1, 2, N) * 2.0 ** rng.integers(500, 1024, N)
    y = rng.uniform(1, 2, N) * 2.0 ** rng.integers(0, 1023, N)
    check(dmul, x, y)


def test_subnormal_operands(dmul):
    rng = np.random.default_rng(14)
    bits = rng.integers(1, 2 ** 52, N, dtype=np.uint64)
    bits >>= rng.integers(0, 52, N).astype(np.uint64)  # every leading-bit position
    sub = np.maximum(bits, 1).view(np.float64) * np.where(rng.random(N) < 0.5, -1.0, 1.0)
    y = rng.uniform(1, 2, N) * 2.0 ** rng.integers(-30, 1023, N)
    check(dmul, sub, y)
    check(dmul, y, sub)
    check(dmul, sub, sub[::-1].copy())


def test_ties_and_short_significands(dmul):
    """Products with exactly one bit beyond the 53 kept ones (halfway cases)
    and products that are exact."""
    rng = np.random.default_rng(15)
    a = rng.integers(2 ** 26, 2 ** 27, N).astype(np.float64)
    b = rng.integers(2 ** 26, 2 ** 28, N).astype(np.float64)
    check(dmul, a * 2.0 ** rng.integers(-40, 40, N), b)
    odd = (rng.integers(2 ** 52, 2 ** 53, N, dtype=np.uint64) | np.uint64(1)).astype(np.float64)
    check(dmul, odd, np.full(N, 1.5))
    check(dmul, odd * 2.0 ** -1075, np.full(N, 3.0))  # halfway cases below the normal range


def test_normal_range_boundary(dmul):
    rng = np.random.default_rng(16)
    x = np.nextafter(1.0, 2.0) ** rng.integers(0, 4096, N)
    y = 2.0 ** -1022 * rng.uniform(0.5, 1.0, N)
    check(dmul, x, y)
    big = np.full(N, np.finfo(np.float64).max)
    check(dmul, big, 1.0 - rng.integers(0, 8, N) * 2.0 ** -53)
    check(dmul, big, 1.0 + rng.integers(0, 8, N) * 2.0 ** -52)


def test_special_values(dmul):
    sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 1.0, -1.0, 5e-324, -5e-324,
                   2.2250738585072014e-308, 2.225073858507201e-308, 1.7976931348623157e308,
                   0.5, 2.0, 3.0, 1.0 / 3.0])
    X, Y = np.meshgrid(sp, sp)
    check(dmul, X.ravel(), Y.ravel())
