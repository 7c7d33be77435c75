"""scale2k (csrc/eig3_f64.cuh), the integer-operation x * 2^k of the binary64
kernels' rare rescalings and of the fused adjoint, against the binary64
product itself (numpy's ldexp, which rounds like x * 2^k): bit for bit on
normal, subnormal, zero and non-finite x, for scalings that stay normal,
enter the subnormals (round to nearest even, including ties and the carry
into 2^-1022), underflow to zero and overflow.  The function body is taken
from the header and compiled on the host with plain 64-bit integer types."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2511_00292_gb300", "csrc")

PRELUDE = r"""
#include <stdint.h>
#include <string.h>
#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double x) { long long b; memcpy(&b, &x, 8); return b; }
static inline double __longlong_as_double(long long b) { double x; memcpy(&x, &b, 8); return x; }
static inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
static inline double from_words(int hi, int lo) {
  const unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | (unsigned)lo;
  double x; memcpy(&x, &b, 8); return x;
}
"""


@pytest.fixture(scope="module")
def scale2k(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "eig3_f64.cuh")).read()
    m = re.search(r"__device__ __forceinline__ double scale2k\(double x, int k\) \{", src)
    assert m
    depth, i = 0, m.end() - 1
    for j in range(i, len(src)):
        depth += src[j] == "{"
        depth -= src[j] == "}"
        if depth == 0:
            break
    body = src[m.start():j + 1]
    d = tmp_path_factory.mktemp("s2k")
    (d / "s.cpp").write_text(PRELUDE + body + r"""
extern "C" void run(const double *x, const int *k, double *out, long n) {
  for (long i = 0; i < n; ++i) out[i] = scale2k(x[i], k[i]);
}
""")
    subprocess.run(["g++", "-O2", "-fPIC", "-shared", "-std=c++17", "-o", str(d / "s.so"),
                    str(d / "s.cpp")], check=True)
    lib = ctypes.CDLL(str(d / "s.so"))

    def fn(x, k):
        x = np.ascontiguousarray(x, dtype=np.float64)
        k = np.ascontiguousarray(k, dtype=np.int32)
        out = np.empty_like(x)
        lib.run(x.ctypes.data, k.ctypes.data, out.ctypes.data, ctypes.c_long(x.size))
        return out
    return fn


def same_bits(a, b):
    return np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_random_scalings_bit_for_bit(scale2k):
    rng = np.random.default_rng(5)
    n = 400_000
    mant = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    ex = rng.integers(-1074, 1024, n)
    x = np.ldexp(mant, ex)  # normal, subnormal and zero values
    k = rng.integers(-2100, 2100, n).astype(np.int32)
    with np.errstate(over="ignore", under="ignore"):
        want = np.ldexp(x, k)
    assert same_bits(scale2k(x, k), want)


def test_rounding_into_the_subnormals(scale2k):
    """Ties to even, the carry into the smallest normal, and 2^-1075 (a tie
    at zero) exactly as the product rounds them."""
    tiny = np.float64(2.0 ** -1074)
    x = np.array([1.5, 2.5, 3.5, 1.0, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52, 1.0, 1.5, 1.0,
                  -1.5, -2.5], dtype=np.float64)
    k = np.array([-1074, -1074, -1074, -1075, -1075, -1023, -1022, -1075, -1076,
                  -1074, -1074], dtype=np.int32)
    with np.errstate(under="ignore"):
        want = np.ldexp(x, k)
    got = scale2k(x, k)
    assert same_bits(got, want)
    assert got[0] == 2 * tiny and got[1] == 2 * tiny and got[2] == 4 * tiny   # ties to even
    assert got[5] == 2.0 ** -1022                                            # carry


def test_special_values_unchanged_and_overflow(scale2k):
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0 ** -1074],
                 dtype=np.float64)
    k = np.array([5, -5, -3, 7, 2, 1024, 1500, 2100], dtype=np.int32)
    got = scale2k(x, k)
    assert same_bits(got[:4], x[:4]) and np.isnan(got[4])
    assert got[5] == np.inf and got[6] == -np.inf and got[7] == np.inf


def test_dev_scale_range(scale2k):
    """The rescaling of out-of-range data: every entry of a matrix whose
    largest magnitude is far outside 2^+-150 by 2^-e with e from that
    largest exponent, as the binary64 kernels apply it."""
    rng = np.random.default_rng(6)
    for lo, hi in ((-1074, -880), (880, 1023), (-1074, 1023)):
        v = np.ldexp(rng.uniform(-2, 2, (20000, 9)), rng.integers(lo, hi, (20000, 9)))
        E = np.frexp(np.abs(v).max(axis=1))[1] - 1 + 1023
        e = (np.clip(E, 1, 2045) - 1023).astype(np.int32)
        ke = np.repeat(-e, 9)
        with np.errstate(under="ignore", over="ignore"):
            want = np.ldexp(v.ravel(), ke)
        assert same_bits(scale2k(v.ravel(), ke), want)
