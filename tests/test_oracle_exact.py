"""Pins of oracle.eigvals_exact, the exact eigenvalues of the stored matrix
(roots of its exact rational characteristic polynomial).

Independent checks: integer matrices with integer spectra built from
unimodular eigenbases (the roots are integers, so the result is exact);
repeated roots in closed form; symmetric matrices against LAPACK eigvalsh;
50-digit mpmath eigenvalues on the paper's benchmark matrices and on random
general matrices; a complex pair gives NaN.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import refs


def integer_spectrum_matrices(n, seed):
    rng = np.random.default_rng(seed)
    out, lam = [], []
    for _ in range(n):
        V = refs.unimodular(rng, steps=3)
        Vi = refs.exact_inverse_int(V)
        l = np.sort(rng.integers(-40, 41, size=3))
        A = V @ np.diag(l) @ Vi
        out.append(A.reshape(9).astype(np.float64))
        lam.append(l.astype(np.float64))
    return np.array(out), np.array(lam)


def test_integer_spectra_are_exact():
    X, lam = integer_spectrum_matrices(300, 8101)
    assert np.array_equal(oracle.eigvals_exact(X), lam)


def test_repeated_roots_closed_form():
    X = np.array([np.diag([2.0, 2.0, 5.0]).reshape(9), np.diag([-1.0, 3.0, 3.0]).reshape(9),
                  (7.5 * np.eye(3)).reshape(9),
                  np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 4.0]]).reshape(9)])  # Jordan
    want = np.array([[2, 2, 5], [-1, 3, 3], [7.5, 7.5, 7.5], [1, 1, 4]], dtype=np.float64)
    assert np.array_equal(oracle.eigvals_exact(X), want)


def test_complex_pair_gives_nan():
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 2.0]]).reshape(1, 9)
    assert np.all(np.isnan(oracle.eigvals_exact(R)))
    S = np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 1.0], [1e-30, 0.0, 1.0]]).reshape(1, 9)
    assert np.all(np.isnan(oracle.eigvals_exact(S)))          # cube roots of 1e-30


def test_symmetric_against_lapack():
    w1 = W.workload1("cpu")["sym6"].A.numpy()
    X = oracle.sym6_to_general9(w1)
    lam = np.linalg.eigvalsh(X.reshape(-1, 3, 3))
    ex6 = oracle.eigvals_exact(w1, layout=1)
    ex9 = oracle.eigvals_exact(X)
    assert np.array_equal(ex6, ex9)
    nA = np.linalg.norm(X, axis=1)
    assert np.all(np.abs(ex9 - lam).max(axis=1) <= 32 * 2.0 ** -53 * nA)   # LAPACK: p(3) u ||A||


def _mp_eig(a9, dps=60):
    import mpmath
    with mpmath.workdps(dps):
        M = mpmath.matrix(3, 3)
        for i in range(3):
            for j in range(3):
                M[i, j] = mpmath.mpf(float(a9[3 * i + j]))
        ev = mpmath.eig(M, left=False, right=False)
        return sorted(ev, key=lambda z: float(mpmath.re(z)))


def test_against_mpmath():
    """Correct rounding: every value within half an ulp of mpmath's 60-digit
    eigenvalue (ties, which occur for these dyadic matrices, either way)."""
    mpmath = pytest.importorskip("mpmath")
    paths = np.array([p["A"] for p in W.paper_paths(deltas=np.logspace(-1, -16, 16))])
    bt = W.workload2(n=300, device="cpu", seed=8102)
    for X in (paths, bt.A.numpy()):
        ex = oracle.eigvals_exact(X)
        for a, e in zip(X, ex):
            ref = _mp_eig(a)
            scale = max(abs(complex(z)) for z in ref)
            if max(abs(float(mpmath.im(z))) for z in ref) > 1e-40 * max(1.0, scale):
                assert np.all(np.isnan(e))
                continue
            with mpmath.workdps(60):
                for k in range(3):
                    d = abs(mpmath.mpf(float(e[k])) - mpmath.re(ref[k]))
                    assert d <= mpmath.mpf(0.5 * float(np.spacing(abs(e[k])))) * (1 + 1e-9) + 1e-300


def test_oracle_method_within_its_bound_of_the_exact_values():
    bt = W.workload2(n=2000, device="cpu", seed=8103)
    X = bt.A.numpy()
    ex = oracle.eigvals_exact(X)
    ok = np.all(np.isfinite(ex), axis=1)
    b = oracle.bounds(X, bt.kappa.numpy())[:, 4]
    err = np.abs(oracle.eigvals(X) - ex).max(axis=1)
    assert ok.mean() > 0.95
    assert np.all(err[ok] <= 8 * b[ok])


def test_paper_limitation_for_ill_conditioned_eigenbases():
    """Sections J3, Delta and Eigenvalues: with the nearly singular U2(1e-3)
    (kappa ~ 9e3) the closed form exceeds the first-order bound; so it does
    for random eigenbases with kappa up to 1e4, increasingly with kappa."""
    worst = 0.0
    for p in W.paper_paths(deltas=np.logspace(-1, -12, 12)):
        if p["U"] != "u2":
            continue
        a = p["A"][None]
        ex = oracle.eigvals_exact(a)
        if not np.all(np.isfinite(ex)):
            continue
        b = oracle.bounds(a, p["kappa"])[0, 4]
        worst = max(worst, np.abs(oracle.eigvals(a) - ex).max() / b)
    assert worst > 8
    bt = W.illconditioned(1500, "cpu", seed=8104)
    X = bt.A.numpy()
    ex = oracle.eigvals_exact(X)
    ok = np.all(np.isfinite(ex), axis=1)
    r = np.abs(oracle.eigvals(X) - ex).max(axis=1) / oracle.bounds(X, bt.kappa.numpy())[:, 4]
    k = bt.kappa.numpy()
    assert np.mean(r[ok & (k > 1e3)] > 8) > 0.5
    assert np.mean(r[ok & (k < 3)] > 8) < 0.02
