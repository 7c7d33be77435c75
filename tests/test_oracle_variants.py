"""Pins of the oracle's comparison variants (Sections J2, J3, Delta and
Eigenvalues): the naive monomial sums (Algorithm 3 and the naive J3 sum) and
the "naive tensor" forms J2 = tr(S S)/2, J3 = det S of S = dev(A), each
with Delta = 4 J2^3 - 27 J3^2 and Algorithm 6.

Pins: exact values on trace-free integer matrices (every operation exact),
exact rational invariants otherwise, and the qualitative findings the paper
reports for its benchmark paths: both variants fail the stability bounds
near a triple eigenvalue, the tensor form by far less; near a double
eigenvalue the tensor J2 and J3 stay within their bounds while Delta from
them does not; eigenvalues lose about u^(1/3) (naive) near a triple and
u^(1/2) (both) near a double eigenvalue.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W
from tests import refs


def trace_free_integers(n, seed, lo=-20, hi=20):
    rng = np.random.default_rng(seed)
    A = rng.integers(lo, hi + 1, size=(n, 9)).astype(np.float64)
    A[:, 8] = -A[:, 0] - A[:, 4]
    return A


def test_naive_tensor_exact_on_trace_free_integers():
    X = trace_free_integers(500, 7101)
    inv = oracle.invariants_naive_tensor(X)
    for a, v in zip(X, inv):
        I1, J2, J3, D = refs.exact_invariants(a)
        assert Fraction(v[0]) == I1 == 0
        assert Fraction(v[1]) == J2
        assert Fraction(v[2]) == J3
        assert Fraction(v[3]) == D


def test_naive_monomial_sums_on_integers():
    """Integer entries: the monomial sums are exact integers, so J2 and J3 are
    the exact values rounded once by the final division by 3 and 27."""
    rng = np.random.default_rng(7102)
    X = rng.integers(-30, 31, size=(500, 9)).astype(np.float64)
    inv = oracle.invariants_naive(X)
    for a, v in zip(X, inv):
        I1, J2, J3, _ = refs.exact_invariants(a)
        assert v[0] == float(I1)
        assert v[1] == float(J2)          # float(Fraction) rounds to nearest
        assert v[2] == float(J3)


def test_variants_agree_with_exact_invariants_on_random_dyadics():
    rng = np.random.default_rng(7103)
    X = np.ldexp(rng.integers(-2 ** 20, 2 ** 20, size=(300, 9)).astype(np.float64), -20)
    for name in ("invariants_naive", "invariants_naive_tensor"):
        inv = getattr(oracle, name)(X)
        for a, v in zip(X, inv):
            ex = [float(x) for x in refs.exact_invariants(a)]
            nA = np.linalg.norm(a)
            assert abs(v[1] - ex[1]) <= 64 * 2.0 ** -53 * nA ** 2
            assert abs(v[2] - ex[2]) <= 256 * 2.0 ** -53 * nA ** 3


def _ratios(fn, a, b, ex):
    v = fn(a)[0]
    return [abs(v[k] - ex[k]) / b[k] if b[k] > 0 else (0.0 if v[k] == ex[k] else np.inf)
            for k in (1, 2, 3)]


def test_paper_pattern_of_the_invariants():
    deltas = np.logspace(-1, -16, 16)
    worst = {}
    for p in W.paper_paths(deltas=deltas):
        if p["U"] == "u2":
            continue
        a = p["A"]
        ex = [float(x) for x in refs.exact_invariants(a)]
        b = oracle.bounds(a, p["kappa"])[0]
        for name, fn in (("naive", oracle.invariants_naive),
                         ("tensor", oracle.invariants_naive_tensor),
                         ("stable", oracle.invariants)):
            r = _ratios(fn, a[None], b, ex)
            key = (p["path"], name)
            worst[key] = np.maximum(worst.get(key, np.zeros(3)), r)
    # near a triple eigenvalue (D1): both fail, the tensor form much less
    assert worst[("d1", "tensor")][0] > 1e10 and worst[("d1", "tensor")][1] > 1e10
    assert worst[("d1", "naive")][0] > 10 * worst[("d1", "tensor")][0]
    assert worst[("d1", "naive")][1] > 1e10 * worst[("d1", "tensor")][1]
    # near a double eigenvalue (D2): tensor J2, J3 within the bound, Delta not
    assert worst[("d2", "tensor")][0] <= 4 and worst[("d2", "tensor")][1] <= 4
    assert worst[("d2", "tensor")][2] > 1e10
    # the stable invariants stay within their bounds on both paths
    assert max(worst[("d1", "stable")].max(), worst[("d2", "stable")].max()) <= 4


def test_paper_pattern_of_the_eigenvalues():
    pytest.importorskip("mpmath")
    deltas = np.logspace(-1, -16, 16)
    worst = {}
    for p in W.paper_paths(deltas=deltas):
        if p["U"] == "u2":
            continue
        a = p["A"]
        ref = refs.mp_eigvals(a)
        for name, fn in (("naive", oracle.eigvals_naive), ("tensor", oracle.eigvals_naive_tensor)):
            lam = fn(a)[0]
            e = max(abs(complex(lam[k]) - ref[k]) for k in range(3))
            worst[(p["path"], name)] = max(worst.get((p["path"], name), 0.0), e)
    assert 1e-7 < worst[("d1", "naive")] < 1e-4             # u^(1/3) near a triple
    assert 1e-10 < worst[("d1", "tensor")] < 1e-8           # tensor form: far less
    for name in ("naive", "tensor"):
        assert 1e-9 < worst[("d2", name)] < 1e-7            # u^(1/2) near a double


def test_tensor_variant_shares_algorithm_6():
    """Same Algorithm 6 step: on matrices whose tensor invariants equal the
    stable ones bit for bit, the eigenvalues are equal bit for bit."""
    X = trace_free_integers(300, 7104)
    a = oracle.invariants(X)
    b = oracle.invariants_naive_tensor(X)
    same = np.all(a == b, axis=1)
    assert same.sum() > 100
    assert np.array_equal(oracle.eigvals(X)[same], oracle.eigvals_naive_tensor(X)[same])
