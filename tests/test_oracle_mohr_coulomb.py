"""Pins of the oracle's Mohr-Coulomb yield function (Section "Application").

The oracle evaluates the definition literally: the largest of the three pair
terms |s_i - s_j| + K (s_i + s_j) over its own eigenvalues, scaled by
(m+1)/(2 S_yc), minus one; the gradient chains d f/d s of the maximising pair
with the eigenvector form of d lambda/dA.  Nothing here re-types that
formula.  The pins are facts that hold independently of it:

* the yield surface passes through uniaxial compression -S_yc and uniaxial
  tension S_yt = S_yc/m (what m = S_yc/S_yt means), through pure shear
  tau = S_yc/(m+1) and through the hydrostatic apex p = S_yc/(m-1);
* for m > 0 the maximising pair is the extreme pair, so
  f = (m s_max - s_min)/S_yc - 1 with LAPACK's eigenvalues (numpy.eigvalsh);
* the gradient of a symmetric sigma is (m n3 n3^T - n1 n1^T)/S_yc with
  LAPACK's eigenvectors, and agrees with central finite differences;
* the Lode-angle sweep of the paper's figure: the present eigenvalue method
  keeps the absolute error of f near machine precision at every angle, the
  naive invariants reach errors of order u^(1/2) near the angles with two
  coalescing principal stresses (multiples of 60 degrees), and f changes sign
  six times over the sweep (the second set of angles where f approaches 0).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests import refs

U = 2.0 ** -53
S_YC, M = 100.0, 10.0        # MPa; S_yt = 10 MPa (Section "Application")
C_LAM = 8.0                  # the eigenvalue bound's constant used throughout the tests


def rotations(n, seed):
    g = torch.Generator().manual_seed(seed)
    return W.haar_o3(n, g, "cpu").numpy()


def rotate_diag(Q, s):
    A = Q @ np.diag(s) @ Q.T
    return (0.5 * (A + A.T)).reshape(9)


def f_tol(X, layout=0, s_yc=S_YC, m=M):
    """|f - f_exact| <= (m + 1)/S_yc * C b_lambda + 4 u (1 + |f|-scale)."""
    b = oracle.bounds(X, None, layout=layout)[:, 4]
    return (m + 1.0) / s_yc * C_LAM * b + 8.0 * U * (1.0 + m)


@pytest.mark.parametrize("s_yc,m", [(100.0, 10.0), (250.0, 2.0), (40.0, 4.5)])
def test_surface_passes_through_uniaxial_shear_and_apex(s_yc, m):
    Q = rotations(64, 5101)
    pts = []
    for q in Q:
        pts.append(rotate_diag(q, [-s_yc, 0.0, 0.0]))              # uniaxial compression
        pts.append(rotate_diag(q, [0.0, s_yc / m, 0.0]))           # uniaxial tension, S_yt
        tau = s_yc / (m + 1.0)
        pts.append(rotate_diag(q, [tau, -tau, 0.0]))               # pure shear
        p = s_yc / (m - 1.0) if m != 1.0 else None
        if p is not None:
            pts.append(rotate_diag(q, [p, p, p]))                  # hydrostatic apex
    X = np.array(pts)
    f = oracle.mohr_coulomb(X, s_yc=s_yc, m=m)
    assert np.all(np.abs(f) <= f_tol(X, s_yc=s_yc, m=m)), np.abs(f).max()
    # just inside / just outside the surface along uniaxial compression
    f_in = oracle.mohr_coulomb(np.diag([-0.99 * s_yc, 0, 0]).reshape(1, 9), s_yc=s_yc, m=m)
    f_out = oracle.mohr_coulomb(np.diag([-1.01 * s_yc, 0, 0]).reshape(1, 9), s_yc=s_yc, m=m)
    assert f_in[0] == pytest.approx(-0.01, abs=1e-14) and f_out[0] == pytest.approx(0.01, abs=1e-14)


def test_extreme_pair_form_against_lapack():
    bt = W.stress_field(4000, "cpu", seed=5102)
    X6 = bt.A.numpy()
    X9 = oracle.sym6_to_general9(X6)
    for s_yc, m in ((S_YC, M), (30.0, 0.5), (500.0, 1.0)):
        lam = np.linalg.eigvalsh(X9.reshape(-1, 3, 3))
        ref = (m * lam[:, 2] - lam[:, 0]) / s_yc - 1.0
        tol = f_tol(X9, s_yc=s_yc, m=m) + 4 * U * np.abs(lam).max(axis=1) * (m + 1) / s_yc
        f9 = oracle.mohr_coulomb(X9, s_yc=s_yc, m=m)
        f6 = oracle.mohr_coulomb(X6, s_yc=s_yc, m=m, layout=oracle.SYM6)
        assert np.all(np.abs(f9 - ref) <= tol)
        assert np.array_equal(f6, f9)


def test_general_matrices_with_real_spectrum():
    """The definition only needs the eigenvalues: general matrices with a real
    spectrum (kappa_2(V) <= 10) against numpy.linalg.eigvals."""
    bt = W.workload2(n=3000, device="cpu", seed=5103)
    X = bt.A.numpy()
    lam = np.sort(np.linalg.eigvals(X.reshape(-1, 3, 3)).real, axis=1)
    sep = np.minimum(lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 1]) > 1e-3
    ref = (M * lam[:, 2] - lam[:, 0]) / S_YC - 1.0
    f = oracle.mohr_coulomb(X)
    b = oracle.bounds(X, bt.kappa.numpy(), layout=0)[:, 4]
    tol = 2 * (M + 1) / S_YC * C_LAM * b + 16 * U
    assert np.all(np.abs(f - ref)[sep] <= tol[sep])


def test_gradient_against_lapack_eigenvectors():
    bt = W.stress_field(3000, "cpu", seed=5104)
    X6 = bt.A.numpy()
    X9 = oracle.sym6_to_general9(X6)
    lam, V = np.linalg.eigh(X9.reshape(-1, 3, 3))
    gap = np.minimum(lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 1])
    nA = np.linalg.norm(X9, axis=1)
    sel = gap > 1e-6 * nA
    n1, n3 = V[:, :, 0], V[:, :, 2]
    ref = (M * np.einsum("ni,nj->nij", n3, n3) - np.einsum("ni,nj->nij", n1, n1)) / S_YC
    ref = ref.reshape(-1, 9)
    _, g9 = oracle.mohr_coulomb(X9, grad=True)
    _, g6 = oracle.mohr_coulomb(X6, layout=oracle.SYM6, grad=True)
    tol = 64 * U * (M + 1) / S_YC * (1 + nA / np.maximum(gap, 1e-300))
    err = np.abs(g9 - ref).max(axis=1)
    assert np.all(err[sel] <= tol[sel])
    # symmetric storage: diagonal entries once, off-diagonals G_ij + G_ji
    R = g9.reshape(-1, 3, 3)
    want6 = np.stack([R[:, 0, 0], R[:, 1, 1], R[:, 2, 2], R[:, 1, 2] + R[:, 2, 1],
                      R[:, 0, 2] + R[:, 2, 0], R[:, 0, 1] + R[:, 1, 0]], axis=1)
    assert np.allclose(g6, want6, rtol=0, atol=1e-15)


def test_gradient_against_central_differences():
    bt = W.gradient_batch(n=6, device="cpu", seed=5105)      # general, separated spectra
    X = 50.0 * bt.A.numpy()
    _, G = oracle.mohr_coulomb(X, grad=True)
    h = 1e-5
    for i in range(len(X)):
        fd = np.empty(9)
        for j in range(9):
            e = np.zeros(9)
            e[j] = h
            fp = oracle.mohr_coulomb((X[i] + e)[None])[0]
            fm = oracle.mohr_coulomb((X[i] - e)[None])[0]
            fd[j] = (fp - fm) / (2 * h)
        assert np.allclose(G[i], fd, rtol=1e-6, atol=1e-8), (G[i], fd)


def naive_f(lam, s_yc=S_YC, m=M):
    """The definition evaluated on given eigenvalues (used for the naive
    invariants' eigenvalues, as in the paper's comparison)."""
    K = (m - 1.0) / (m + 1.0)
    out = np.empty(len(lam))
    for r, s in enumerate(lam):
        out[r] = max(abs(s[i] - s[j]) + K * (s[i] + s[j]) for i in range(3)
                     for j in range(i + 1, 3))
    return (m + 1.0) / (2.0 * s_yc) * out - 1.0


def test_lode_sweep_stable_vs_naive():
    """Figure of Section "Application": J2 = 150 MPa^2, sigma = U_symm diag(s) U_symm^T."""
    pytest.importorskip("mpmath")
    n = 720                                   # half-degree steps
    X9 = oracle.sym6_to_general9(W.lode_sweep(n))
    exact = np.array([naive_f([sorted(z.real for z in refs.mp_eigvals(a))])[0] for a in X9])
    f = oracle.mohr_coulomb(X9)
    fn = naive_f(oracle.eigvals_naive(X9))
    err, err_n = np.abs(f - exact), np.abs(fn - exact)
    assert np.all(err <= f_tol(X9)), err.max()
    assert err.max() < 1e-14
    theta = np.degrees(np.arange(n) * 2 * np.pi / n)
    dist60 = np.abs(((theta + 30.0) % 60.0) - 30.0)      # distance to the nearest multiple of 60
    near, far = dist60 <= 2.0, dist60 >= 10.0
    assert err_n[near].max() > 1e-9                       # order u^(1/2)
    assert err_n[near].max() < 1e-6
    assert err_n[far].max() < 1e-13
    # f changes sign six times over the sweep (zeros between the coalescence angles)
    assert np.count_nonzero(np.diff(np.sign(f)) != 0) == 6
    assert f.min() < -0.1 and f.max() > 0.4


def test_lode_sweep_principal_stresses_have_the_prescribed_j2():
    X9 = oracle.sym6_to_general9(W.lode_sweep(96))
    inv = oracle.invariants(X9)
    assert np.allclose(inv[:, 0], 0.0, atol=1e-13)
    assert np.allclose(inv[:, 1], 150.0, rtol=1e-14)


def test_value_only_equals_value_with_gradient():
    bt = W.stress_field(500, "cpu", seed=5106)
    X6 = bt.A.numpy()
    f0 = oracle.mohr_coulomb(X6, layout=oracle.SYM6)
    f1, _ = oracle.mohr_coulomb(X6, layout=oracle.SYM6, grad=True)
    assert np.array_equal(f0, f1)


def test_stress_field_recipe():
    bt = W.stress_field(20000, "cpu", seed=5107)
    lam = bt.lam_nominal.numpy()
    p = lam.mean(axis=1)
    assert -200.0 <= p.min() and p.max() <= 100.0
    rad = np.sqrt(1.5 * ((lam - p[:, None]) ** 2).sum(axis=1))   # sqrt(3 J2) of the spectrum
    assert rad.min() >= 0.1 * (1 - 1e-12) and rad.max() <= 100.0 * (1 + 1e-12)
    X9 = oracle.sym6_to_general9(bt.A.numpy())
    assert np.allclose(X9.reshape(-1, 3, 3), np.transpose(X9.reshape(-1, 3, 3), (0, 2, 1)))
    frac_yield = float(np.mean(oracle.mohr_coulomb(X9) > 0))
    assert 0.2 < frac_yield < 0.8, frac_yield          # elastic and yielding states both common
