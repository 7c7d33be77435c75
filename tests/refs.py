"""Independent references used to pin the oracle (test side only).

Nothing here follows the paper's algorithms.  Each function is a plain
definition evaluated exactly or at high precision:

* exact_invariants: I1 = tr A, J2 = (1/2) tr(S^2), J3 = det S with
  S = A - (tr A / 3) I, and Delta = 4 J2^3 - 27 J3^2, all in rational
  arithmetic on the binary64 entries (so the result is the exact value at
  fl(A), as the paper's error definition requires).
* parlett_discriminant: det B with B_ij = tr(A^(i-1) A^(j-1)) (Parlett's
  form of the discriminant, Section "Discriminant Delta"), exact.
* mp_eigvals: eigenvalues of fl(A) at high precision (mpmath), sorted by
  real part; complex values are kept.
* spectral invariants of a known spectrum (the symmetric functions of the
  eigenvalues).
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np


def _exact_matrix(a9):
    return [[Fr(float(a9[3 * i + j])) for j in range(3)] for i in range(3)]


def det3(M):
    return (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
            - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
            + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]))


def matmul3(X, Y):
    return [[sum(X[i][k] * Y[k][j] for k in range(3)) for j in range(3)] for i in range(3)]


def exact_invariants(a9):
    """Exact (I1, J2, J3, Delta) of the binary64 matrix a9, as Fractions."""
    A = _exact_matrix(a9)
    I1 = A[0][0] + A[1][1] + A[2][2]
    S = [[A[i][j] - (I1 / 3 if i == j else 0) for j in range(3)] for i in range(3)]
    S2 = matmul3(S, S)
    J2 = (S2[0][0] + S2[1][1] + S2[2][2]) / 2
    J3 = det3(S)
    return I1, J2, J3, 4 * J2 ** 3 - 27 * J3 ** 2


def parlett_discriminant(a9):
    """Exact det B, B_ij = tr(A^(i-1) A^(j-1)), i, j = 1..3."""
    A = _exact_matrix(a9)
    I = [[Fr(int(i == j)) for j in range(3)] for i in range(3)]
    P = [I, A, matmul3(A, A)]
    B = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            M = matmul3(P[i], P[j])
            B[i][j] = M[0][0] + M[1][1] + M[2][2]
    return det3(B)


def spectral_invariants(lam):
    """(I1, J2, J3, Delta) as symmetric functions of a known spectrum (Fractions)."""
    l1, l2, l3 = [Fr(x) for x in lam]
    I1 = l1 + l2 + l3
    m = I1 / 3
    J2 = ((l1 - l2) ** 2 + (l1 - l3) ** 2 + (l2 - l3) ** 2) / 6
    J3 = (l1 - m) * (l2 - m) * (l3 - m)
    D = ((l1 - l2) * (l1 - l3) * (l2 - l3)) ** 2
    return I1, J2, J3, D


def mp_eigvals(a9, dps: int = 50):
    """Eigenvalues of the binary64 matrix a9 at `dps` digits, sorted by real part."""
    import mpmath
    with mpmath.workdps(dps):
        M = mpmath.matrix(3, 3)
        for i in range(3):
            for j in range(3):
                M[i, j] = mpmath.mpf(float(a9[3 * i + j]))
        ev = mpmath.eig(M, left=False, right=False)
        ev = sorted(ev, key=lambda z: (float(mpmath.re(z)), float(mpmath.im(z))))
        return [complex(z) for z in ev]


def mp_charpoly_roots(a9, dps: int = 60):
    """Roots of the exact characteristic polynomial of fl(A) (exact rational
    coefficients, mpmath polyroots at `dps` digits), sorted by real part."""
    import mpmath
    A = _exact_matrix(a9)
    I1 = A[0][0] + A[1][1] + A[2][2]
    I2 = (A[0][0] * A[1][1] - A[0][1] * A[1][0] + A[0][0] * A[2][2] - A[0][2] * A[2][0]
          + A[1][1] * A[2][2] - A[1][2] * A[2][1])
    I3 = det3(A)
    with mpmath.workdps(dps):
        coeffs = [mpmath.mpf(1), -mpmath.mpf(I1.numerator) / I1.denominator,
                  mpmath.mpf(I2.numerator) / I2.denominator,
                  -mpmath.mpf(I3.numerator) / I3.denominator]
        roots = mpmath.polyroots(coeffs, maxsteps=400, extraprec=4 * dps)
        roots = sorted(roots, key=lambda z: (float(mpmath.re(z)), float(mpmath.im(z))))
        return [complex(z) for z in roots]


def unimodular(rng: np.random.Generator, steps: int = 3) -> np.ndarray:
    """Random integer 3x3 matrix with det = +-1 (product of integer shears and
    a permutation), so its inverse is an integer matrix too."""
    V = np.eye(3, dtype=np.int64)
    for _ in range(steps):
        i, j = rng.choice(3, size=2, replace=False)
        E = np.eye(3, dtype=np.int64)
        E[i, j] = rng.choice([-1, 1])
        V = V @ E
    return V[rng.permutation(3)]


def exact_inverse_int(V: np.ndarray) -> np.ndarray:
    """Inverse of an integer unimodular matrix (adjugate / det), as integers."""
    M = [[Fr(int(V[i, j])) for j in range(3)] for i in range(3)]
    d = det3(M)
    adj = np.zeros((3, 3), dtype=np.int64)
    for i in range(3):
        for j in range(3):
            minor = [[M[r][c] for c in range(3) if c != i] for r in range(3) if r != j]
            cof = minor[0][0] * minor[1][1] - minor[0][1] * minor[1][0]
            val = (-1) ** (i + j) * cof / d
            assert val.denominator == 1
            adj[i, j] = int(val)
    return adj
