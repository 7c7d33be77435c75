"""Exact eigenvalues of the stored matrices, by their definition.

TEST INFRASTRUCTURE ONLY (part of the oracle package).

The eigenvalues of the binary64 matrix fl(A) are the roots of its
characteristic polynomial

    p(x) = det(x I - A) = x^3 + c2 x^2 + c1 x + c0,
    c2 = -tr A,  c1 = sum of the principal 2x2 minors,  c0 = -det A,

whose coefficients are computed exactly in rational arithmetic (Fraction) from
the stored entries.  Nothing of the paper's method is used: no invariants, no
trigonometric formula.  The sign of the cubic's exact discriminant separates
a complex pair (NaN), repeated roots (closed form in rational arithmetic)
and three simple roots.  For the latter the critical points of p,
x_-/+ = (-c2 -/+ sqrt(c2^2 - 3 c1)) / 3, split the real line into three
intervals on each of which p is monotone and has exactly one root; each root
is found by bisection in decimal arithmetic with 60 significant digits
(Python's decimal module).  Every root is rounded once to binary64.

This is the reference the stability bounds of the paper are stated against
(the exact eigenvalues of fl(A)); it is slow (milliseconds per matrix) and
meant for samples of a few thousand matrices.

invariants_exact gives the exact invariants of fl(A) from the same exact
coefficients: with I1 = -c2, I2 = c1 and I3 = -c0 (trace, sum of the
principal minors, determinant),

    J2 = I1^2/3 - I2,   J3 = 2 I1^3/27 - I1 I2/3 + I3,   Delta = 4 J2^3 - 27 J3^2,

the invariants of the deviator S = A - (I1/3) I (J2 = tr(S^2)/2 and
J3 = det S, since S has the characteristic polynomial of A shifted by I1/3),
each rounded once to binary64.  The map_* helpers spread either over worker
processes started with spawn (safe beside a CUDA context).
"""
from __future__ import annotations

from decimal import Decimal, localcontext
from fractions import Fraction

import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np

DIGITS = 60


def charpoly(a9):
    """Exact (c2, c1, c0) of det(x I - A) for a 9-entry row-major matrix."""
    A = [[Fraction(float(a9[3 * i + j])) for j in range(3)] for i in range(3)]
    tr = A[0][0] + A[1][1] + A[2][2]
    minors = ((A[0][0] * A[1][1] - A[0][1] * A[1][0])
              + (A[0][0] * A[2][2] - A[0][2] * A[2][0])
              + (A[1][1] * A[2][2] - A[1][2] * A[2][1]))
    det = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
           - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
           + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]))
    return -tr, minors, -det


def _dec(q: Fraction) -> Decimal:
    return Decimal(q.numerator) / Decimal(q.denominator)


def _roots(c2: Fraction, c1: Fraction, c0: Fraction):
    """Ascending real roots as Decimals, or None for a complex pair.

    The exact discriminant of the cubic, b^2 c^2 - 4 c^3 - 4 b^3 d - 27 d^2 +
    18 b c d (leading coefficient 1), decides the case: negative -> a complex
    pair; zero -> a repeated root, given in closed form by rational
    arithmetic (the double root (9 d - b c) / (2 (b^2 - 3 c)) and the simple
    root (4 b c - 9 d - b^3) / (b^2 - 3 c), or the triple root -b/3);
    positive -> three simple roots: with d = 0 the root 0 and those of
    x^2 + b x + c, otherwise bisected."""
    b, c, d = c2, c1, c0
    disc_p = b * b * c * c - 4 * c ** 3 - 4 * b ** 3 * d - 27 * d * d + 18 * b * c * d
    if disc_p < 0:
        return None
    q = b * b - 3 * c                        # (tr A)^2 - 3 c1 = 3 J2
    if disc_p == 0:
        if q == 0:
            r = _dec(-b / 3)
            return [r, r, r]
        xd = (9 * d - b * c) / (2 * q)
        xs = (4 * b * c - 9 * d - b ** 3) / q
        return [_dec(x) for x in sorted((xd, xd, xs))]
    if d == 0:                               # p = x (x^2 + b x + c): a root at 0 exactly
        sq = _dec(b * b - 4 * c).sqrt()      # > 0: the roots are simple here
        return sorted([Decimal(0), (-_dec(b) - sq) / 2, (-_dec(b) + sq) / 2])
    D2, D1, D0 = _dec(b), _dec(c), _dec(d)

    def p(x):
        return ((x + D2) * x + D1) * x + D0

    s = _dec(q).sqrt()
    xm = (-D2 - s) / 3                       # local maximum of p
    xp = (-D2 + s) / 3                       # local minimum of p
    bound = 1 + max(abs(D2), abs(D1), abs(D0))   # Cauchy: every root is within it

    def bisect(lo, hi, increasing):
        # p is monotone on [lo, hi] with a sign change there, and the root is
        # not 0: stop at a relative width of 10^-(DIGITS - 12)
        eps = Decimal(10) ** (-(DIGITS - 12))
        for _ in range(8000):
            if hi - lo <= eps * max(abs(lo), abs(hi)):
                break
            mid = (lo + hi) / 2
            v = p(mid)
            if v == 0:
                return mid
            if (v < 0) == increasing:
                lo = mid
            else:
                hi = mid
        return (lo + hi) / 2

    # p(xm) > 0 > p(xp) exactly; a sign lost at DIGITS digits means two roots
    # closer than that resolution, which then coincide at binary64 precision
    pm, pp = p(xm), p(xp)
    r1 = bisect(-bound, xm, True) if pm > 0 else xm
    r2 = xm if pm <= 0 else (xp if pp >= 0 else bisect(xm, xp, False))
    r3 = bisect(xp, bound, True) if pp < 0 else xp
    return [r1, r2, r3]


def eigvals_exact(X, layout: int = 0) -> np.ndarray:
    """(n, 3) ascending exact eigenvalues of the stored matrices, rounded once
    to binary64; NaN rows for matrices with a complex pair of eigenvalues.
    layout 0: (n, 9) row-major; layout 1: (n, 6) symmetric (A00, A11, A22,
    A12, A02, A01)."""
    X = np.asarray(X, dtype=np.float64)
    if layout == 1:
        S = X.reshape(-1, 6)
        X = np.stack([S[:, 0], S[:, 5], S[:, 4], S[:, 5], S[:, 1], S[:, 3],
                      S[:, 4], S[:, 3], S[:, 2]], axis=1)
    X = X.reshape(-1, 9)
    out = np.empty((X.shape[0], 3))
    with localcontext() as ctx:
        ctx.prec = DIGITS
        for i, a in enumerate(X):
            if not np.all(np.isfinite(a)):
                out[i] = np.nan
                continue
            r = _roots(*charpoly(a))
            out[i] = np.nan if r is None else [float(x) for x in r]
    return out


def _general9(X, layout: int) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    if layout == 1:
        S = X.reshape(-1, 6)
        X = np.stack([S[:, 0], S[:, 5], S[:, 4], S[:, 5], S[:, 1], S[:, 3],
                      S[:, 4], S[:, 3], S[:, 2]], axis=1)
    return X.reshape(-1, 9)


def invariants_exact(X, layout: int = 0) -> np.ndarray:
    """(n, 4) exact (I1, J2, J3, Delta) of the stored matrices, each rounded
    once to binary64 (NaN rows for non-finite input)."""
    X = _general9(X, layout)
    out = np.empty((X.shape[0], 4))
    for i, a in enumerate(X):
        if not np.all(np.isfinite(a)):
            out[i] = np.nan
            continue
        c2, c1, c0 = charpoly(a)
        I1, I2, I3 = -c2, c1, -c0
        J2 = I1 * I1 / 3 - I2
        J3 = 2 * I1 ** 3 / 27 - I1 * I2 / 3 + I3
        out[i] = [float(I1), float(J2), float(J3), float(4 * J2 ** 3 - 27 * J3 ** 2)]
    return out


def _chunked(fn, X, layout: int, processes: int) -> np.ndarray:
    X = _general9(X, layout)
    k = max(1, int(processes))
    if k == 1 or X.shape[0] < 64:
        return fn(X, 0)
    parts = np.array_split(X, 4 * k)
    with ProcessPoolExecutor(max_workers=k, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(fn, parts, [0] * len(parts)))
    return np.concatenate(res, axis=0)


def map_eigvals_exact(X, layout: int = 0, processes: int = 1) -> np.ndarray:
    """eigvals_exact over `processes` spawned worker processes."""
    return _chunked(eigvals_exact, X, layout, processes)


def map_invariants_exact(X, layout: int = 0, processes: int = 1) -> np.ndarray:
    """invariants_exact over `processes` spawned worker processes."""
    return _chunked(invariants_exact, X, layout, processes)
