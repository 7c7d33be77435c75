"""Pins for the FP64 oracle (CPU only).

The oracle is checked against things fixed by the paper and by mathematics,
never against itself: exact rational invariants of fl(A) (plain definitions),
known spectra built exactly, high-precision eigenvalues, the paper's worked
example, special cases, the paper's qualitative findings on its test paths,
finite differences for the gradient and library eigenvectors.
"""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest
import torch

import workloads as W
from tests import refs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = 2.0 ** -53
C_INV = 4.0      # invariants vs exact, well-conditioned eigenbasis (observed <= 2.31)
C_LAM = 8.0      # eigenvalues vs exact: the constant C of the eigenvalue bound (observed <= 7.4)


def _ratio(err, bound):
    err = np.asarray(err, dtype=np.float64)
    bound = np.asarray(bound, dtype=np.float64)
    out = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), np.where(err == 0, 0.0, np.inf))
    return out


def _exact_errors(oracle_mod, A, kappa=1.0):
    A = np.asarray(A, dtype=np.float64).reshape(-1, 9)
    inv = oracle_mod.invariants(A)
    b = oracle_mod.bounds(A, kappa)
    err = np.zeros((A.shape[0], 4))
    for i in range(A.shape[0]):
        ex = refs.exact_invariants(A[i])
        for k in range(4):
            err[i, k] = abs(Fr(float(inv[i, k])) - ex[k])
    return err, b


# --------------------------------------------------------------------------
# Invariants against exact rational values of fl(A)
# --------------------------------------------------------------------------

def test_invariants_exact_random_dyadic(oracle_mod):
    rng = np.random.default_rng(11)
    A = rng.integers(-4096, 4097, size=(300, 9)).astype(np.float64) / 1024.0
    err, b = _exact_errors(oracle_mod, A)
    r = _ratio(err, b[:, :4])
    assert r.max() <= C_INV, r.max(axis=0)


def test_invariants_exact_general_kappa10(oracle_mod):
    bt = W.workload2(n=600, device="cpu", seed=77)
    A = bt.A.numpy()
    err, b = _exact_errors(oracle_mod, A, bt.kappa.numpy())
    r = _ratio(err, b[:, :4])
    # I1 and J2 are backward stable for any eigenbasis (Sections I1 and J2);
    # J3 and Delta only for a well-conditioned one, kappa <= 10 here.
    assert r[:, 0].max() <= C_INV
    assert r[:, 1].max() <= C_INV
    assert r[:, 2].max() <= 16.0 * 10.0
    assert r[:, 3].max() <= 16.0 * 10.0


def test_parlett_form_matches_definition():
    rng = np.random.default_rng(5)
    for _ in range(40):
        a = rng.integers(-9, 10, size=9).astype(np.float64) / 8.0
        assert refs.parlett_discriminant(a) == refs.exact_invariants(a)[3]


def test_paper_paths_stability_pattern(oracle_mod):
    """Reproduces the paper's findings on its test paths: all four stable
    invariants within their bounds for U1 and U_symm; J2 within its bound
    even for U2(1e-3); J3 and Delta exceeding theirs for U2."""
    worst = {}
    for p in W.paper_paths():
        err, b = _exact_errors(oracle_mod, p["A"], p["kappa"])
        r = _ratio(err, b[:, :4])[0]
        key = p["U"]
        worst[key] = np.maximum(worst.get(key, np.zeros(4)), r)
    for u in ("symm", "u1"):
        assert worst[u].max() <= C_INV, (u, worst[u])
    assert worst["u2"][1] <= C_INV
    assert worst["u2"][2] > 10.0 and worst["u2"][3] > 10.0


def test_lemma_dev_norm_vs_J2(oracle_mod):
    """(2/(9 kappa^2)) J2 <= ||dev A||_F^2 <= 18 kappa^2 J2 (Lemma, Section J2)."""
    bt = W.workload2(n=2000, device="cpu", seed=78)
    A = bt.A.numpy()
    kap = bt.kappa.numpy()
    J2 = oracle_mod.invariants(A)[:, 1]
    nS2 = oracle_mod.bounds(A, kap)[:, 1] / U64
    keep = J2 > 1e-200
    lo = 2.0 / (9.0 * kap ** 2) * J2
    hi = 18.0 * kap ** 2 * J2
    assert np.all(nS2[keep] >= lo[keep] * (1 - 1e-9))
    assert np.all(nS2[keep] <= hi[keep] * (1 + 1e-9))


# --------------------------------------------------------------------------
# Known spectra, built exactly
# --------------------------------------------------------------------------

SPECTRA = [
    (Fr(1, 4), Fr(3, 8), Fr(-5, 2)),
    (Fr(1), Fr(1) + Fr(1, 2 ** 30), Fr(2)),
    (Fr(1), Fr(1) + Fr(1, 2 ** 20), Fr(1) + Fr(1, 2 ** 19)),
    (Fr(2), Fr(2), Fr(5)),
    (Fr(-3), Fr(-3), Fr(-3)),
    (Fr(7, 2), Fr(-1, 16), Fr(0)),
    (Fr(1), Fr(1) + Fr(1, 2 ** 40), Fr(1) + Fr(1, 2 ** 39)),
]


@pytest.mark.parametrize("lam", SPECTRA)
def test_known_spectrum_exact(oracle_mod, lam):
    rng = np.random.default_rng(abs(hash(tuple(lam))) % (2 ** 32))
    for trial in range(6):
        V = refs.unimodular(rng, steps=2 + trial % 3)
        Vi = refs.exact_inverse_int(V)
        Aex = [[sum(Fr(int(V[i, k])) * lam[k] * Fr(int(Vi[k, j])) for k in range(3))
                for j in range(3)] for i in range(3)]
        a9 = np.array([float(Aex[i][j]) for i in range(3) for j in range(3)])
        assert all(Fr(float(Aex[i][j])) == Aex[i][j] for i in range(3) for j in range(3))
        assert refs.exact_invariants(a9) == refs.spectral_invariants(lam)
        kappa = float(np.linalg.cond(V.astype(np.float64), 2))
        err, b = _exact_errors(oracle_mod, a9, kappa)
        # bound-relative check with kappa-scaled constant for J3 and Delta
        r = _ratio(err, b[:, :4])[0]
        assert r[0] <= C_INV and r[1] <= C_INV, r
        assert r[2] <= C_INV * kappa ** 2 and r[3] <= C_INV * kappa ** 2, (r, kappa)
        got = oracle_mod.eigvals(a9)[0]
        want = np.array([float(x) for x in sorted(lam)])
        assert np.all(np.abs(got - want) <= C_LAM * b[0, 4]), (got, want, b[0, 4])


# --------------------------------------------------------------------------
# Eigenvalues against high-precision references
# --------------------------------------------------------------------------

def _lam_ratio(oracle_mod, A, kappa, ref_fn):
    A = np.asarray(A, dtype=np.float64).reshape(-1, 9)
    lam = oracle_mod.eigvals(A)
    b = oracle_mod.bounds(A, kappa)[:, 4]
    worst = 0.0
    for i in range(A.shape[0]):
        ref = ref_fn(A[i])
        err = max(abs(complex(lam[i, k]) - ref[k]) for k in range(3))
        worst = max(worst, err / b[i])
    return worst


def test_eigvals_vs_mpmath_symmetric(oracle_mod):
    pytest.importorskip("mpmath")
    w1 = W.workload1("cpu")["general9"]
    idx = np.r_[np.arange(0, 4096, 16), np.arange(4096, 4160)]
    A = w1.A.numpy()[idx]
    assert _lam_ratio(oracle_mod, A, 1.0, refs.mp_eigvals) <= C_LAM


def test_eigvals_vs_mpmath_general(oracle_mod):
    pytest.importorskip("mpmath")
    bt = W.workload2(n=300, device="cpu", seed=79)
    # complex spectra of fl(A) (near-double cases) are compared in modulus
    assert _lam_ratio(oracle_mod, bt.A.numpy(), bt.kappa.numpy(), refs.mp_eigvals) <= C_LAM


def test_eigvals_vs_charpoly_roots(oracle_mod):
    pytest.importorskip("mpmath")
    bt = W.workload2(n=24, device="cpu", seed=80)
    assert _lam_ratio(oracle_mod, bt.A.numpy(), bt.kappa.numpy(), refs.mp_charpoly_roots) <= C_LAM


def test_eigvals_vs_lapack_symmetric(oracle_mod):
    w1 = W.workload1("cpu")["general9"]
    A = w1.A.numpy()
    lam = oracle_mod.eigvals(A)
    ref = np.linalg.eigvalsh(A.reshape(-1, 3, 3))
    b = oracle_mod.bounds(A, 1.0)[:, 4]
    assert np.all(np.abs(lam - ref).max(axis=1) <= 2 * C_LAM * b)


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            out[k.strip()] = v.split()
    return out


def test_worked_example(oracle_mod):
    g = _read_golden("worked_example.txt")
    a9 = np.array([float(x) for x in g["matrix"]])
    delta = float(g["delta"][0])
    # the generator's construction reproduces the printed matrix
    built = W.paper_matrix(W.paper_U("u1"), W.paper_D("d2", delta))
    assert np.allclose(built, a9, rtol=0, atol=4 * U64)
    assert abs(np.linalg.cond(W.paper_U("u1"), 2) - float(g["kappa2_U1"][0])) < 1e-12
    lam = oracle_mod.eigvals(a9)[0]
    nominal = np.array([float(x) for x in g["nominal_eigenvalues"]])
    assert np.all(np.abs(lam - nominal) <= 1e-15)
    mpmath = pytest.importorskip("mpmath")
    ref = refs.mp_eigvals(a9)
    err = max(abs(complex(lam[k]) - ref[k]) for k in range(3))
    # "on the order of machine precision, about 1e-16": same order of magnitude,
    # and within the eigenvalue bound kappa ||A||_F u with kappa2(U1) = 2
    assert err < 10 * float(g["reported_abs_error"][0]), err
    b = oracle_mod.bounds(a9, float(g["kappa2_U1"][0]))[0, 4]
    assert err <= C_LAM * b
    # the ordering lambda_1 <= lambda_2 <= lambda_3 resolves the 1e-14 gap
    assert lam[0] < lam[1] < lam[2]


def test_paper_kappas():
    g = _read_golden("paper_facts.txt")
    assert abs(np.linalg.cond(W.paper_U("symm"), 2) - float(g["kappa2_symm"][0])) < 1e-12
    assert abs(np.linalg.cond(W.paper_U("u1"), 2) - float(g["kappa2_u1"][0])) < 1e-12
    k2 = np.linalg.cond(W.paper_U("u2", 1e-3), 2)
    assert 0.9 * float(g["kappa2_u2_gamma1e-3_approx"][0]) < k2 < 1.1 * float(g["kappa2_u2_gamma1e-3_approx"][0])


def test_naive_vs_stable_paper_paths(oracle_mod):
    """The paper's eigenvalue comparison: the naive closed form loses about
    u^(1/3) near a triple and u^(1/2) near a double eigenvalue, the stable
    one stays within its bound (U1, U_symm)."""
    pytest.importorskip("mpmath")
    worst_naive = {"d1": 0.0, "d2": 0.0}
    worst_stable = 0.0
    for p in W.paper_paths(deltas=np.logspace(-1, -16, 16)):
        if p["U"] == "u2":
            continue
        a9 = p["A"]
        ref = refs.mp_eigvals(a9)
        st = oracle_mod.eigvals(a9)[0]
        nv = oracle_mod.eigvals_naive(a9)[0]
        b = oracle_mod.bounds(a9, p["kappa"])[0, 4]
        worst_stable = max(worst_stable, max(abs(complex(st[k]) - ref[k]) for k in range(3)) / b)
        worst_naive[p["path"]] = max(worst_naive[p["path"]],
                                     max(abs(complex(nv[k]) - ref[k]) for k in range(3)))
    assert worst_stable <= C_LAM
    assert worst_naive["d1"] > 1e-7      # order u^(1/3)
    assert worst_naive["d2"] > 3e-9      # order u^(1/2)


# --------------------------------------------------------------------------
# Special cases
# --------------------------------------------------------------------------

def test_scaled_identity_exact(oracle_mod):
    for alpha in (0.0, 1.0, -0.1, 3.7e-200, 1e300, 7.0):
        a9 = np.array([alpha, 0, 0, 0, alpha, 0, 0, 0, alpha], dtype=np.float64)
        inv = oracle_mod.invariants(a9)[0]
        assert inv[1] == 0.0 and inv[2] == 0.0 and inv[3] == 0.0
        lam = oracle_mod.eigvals(a9)[0]
        assert np.all(np.abs(lam - alpha) <= 2 * np.spacing(abs(alpha)))


def test_diagonal_cases(oracle_mod):
    a9 = np.diag([1.0, 2.0, 3.0]).reshape(9)
    inv = oracle_mod.invariants(a9)[0]
    assert inv[2] == 0.0 and inv[3] == 4.0 and inv[1] == 1.0
    assert np.array_equal(oracle_mod.eigvals(a9)[0].round(14), [1.0, 2.0, 3.0])
    for d in (1e-3, 1e-8, 1e-15):
        a9 = np.diag([1.0, 1.0, 1.0 + d]).reshape(9)
        assert oracle_mod.invariants(a9)[0, 3] == 0.0
    perm = np.diag([3.0, -1.0, 2.0]).reshape(9)
    lam = oracle_mod.eigvals(perm)[0]
    assert np.allclose(lam, [-1.0, 2.0, 3.0], atol=8 * U64 * 3)


def test_ordering_random(oracle_mod):
    bt = W.workload2(n=20000, device="cpu", seed=81)
    A = bt.A.numpy()
    lam = oracle_mod.eigvals(A)
    b = oracle_mod.bounds(A, bt.kappa.numpy())[:, 4]
    # lambda_1 <= lambda_2 <= lambda_3 holds up to rounding: where two eigenvalues
    # agree to within the error bound their computed order may swap by a few ulps
    assert np.all(lam[:, 0] - lam[:, 1] <= C_LAM * b)
    assert np.all(lam[:, 1] - lam[:, 2] <= C_LAM * b)
    far = (lam[:, 1] - lam[:, 0] > C_LAM * b) | (lam[:, 2] - lam[:, 1] > C_LAM * b)
    assert far.mean() > 0.5


def test_sym6_layout_matches_general(oracle_mod):
    w1 = W.workload1("cpu")
    g = oracle_mod.eigvals(w1["general9"].A.numpy())
    s = oracle_mod.eigvals(w1["sym6"].A.numpy(), layout=oracle_mod.SYM6)
    assert np.array_equal(g, s)
    gi = oracle_mod.invariants(w1["general9"].A.numpy())
    si = oracle_mod.invariants(w1["sym6"].A.numpy(), layout=oracle_mod.SYM6)
    assert np.array_equal(gi, si)


def test_threaded_matches_serial(oracle_mod):
    bt = W.workload2(n=10007, device="cpu", seed=82)
    A = bt.A.numpy()
    lam, used = oracle_mod.eigvals_mt(A, nthreads=4)
    assert used >= 1
    assert np.array_equal(lam, oracle_mod.eigvals(A))


# --------------------------------------------------------------------------
# Gradient oracle and bound calculator
# --------------------------------------------------------------------------

def test_gradient_oracle_vs_central_fd(oracle_mod):
    bt = W.gradient_batch(n=40, device="cpu", seed=83)
    A = bt.A.numpy()
    rng = np.random.default_rng(3)
    gbar = rng.standard_normal((A.shape[0], 3))
    G = oracle_mod.eigvals_grad(A, gbar)
    h = 1e-6
    for i in range(A.shape[0]):
        fd = np.zeros(9)
        for j in range(9):
            ap = A[i].copy(); am = A[i].copy()
            ap[j] += h; am[j] -= h
            fd[j] = (gbar[i] @ oracle_mod.eigvals(ap)[0] - gbar[i] @ oracle_mod.eigvals(am)[0]) / (2 * h)
        assert np.max(np.abs(fd - G[i])) <= 1e-6 * max(1.0, np.max(np.abs(G[i]))), (i, fd, G[i])


def test_gradient_oracle_vs_lapack_eigenvectors(oracle_mod):
    bt = W.gradient_batch(n=200, device="cpu", seed=84)
    A = bt.A.numpy()
    rng = np.random.default_rng(4)
    gbar = rng.standard_normal((A.shape[0], 3))
    G = oracle_mod.eigvals_grad(A, gbar)
    for i in range(A.shape[0]):
        M = A[i].reshape(3, 3)
        w, R = np.linalg.eig(M)
        order = np.argsort(w.real)
        w, R = w[order].real, R[:, order].real
        L = np.linalg.inv(R)          # rows are left eigenvectors, L R = I
        ref = sum(gbar[i, k] * np.outer(L[k], R[:, k]) for k in range(3)).reshape(9)
        assert np.max(np.abs(ref - G[i])) <= 1e-9 * max(1.0, np.max(np.abs(ref)))


def test_gradient_oracle_sym6(oracle_mod):
    w1 = W.workload1("cpu")["sym6"]
    S = w1.A.numpy()[:30]
    rng = np.random.default_rng(6)
    gbar = rng.standard_normal((S.shape[0], 3))
    G = oracle_mod.eigvals_grad(S, gbar, layout=oracle_mod.SYM6)
    h = 1e-6
    for i in range(S.shape[0]):
        for j in range(6):
            sp = S[i].copy(); sm = S[i].copy()
            sp[j] += h; sm[j] -= h
            fd = (gbar[i] @ oracle_mod.eigvals(sp, oracle_mod.SYM6)[0]
                  - gbar[i] @ oracle_mod.eigvals(sm, oracle_mod.SYM6)[0]) / (2 * h)
            assert abs(fd - G[i, j]) <= 1e-6 * max(1.0, np.max(np.abs(G[i])))


def _exact_grad_norm(fn_index, a9, h=Fr(1, 2 ** 40)):
    g = []
    for j in range(9):
        ap = [Fr(float(x)) for x in a9]
        am = list(ap)
        ap[j] += h
        am[j] -= h
        fp = _exact_inv_fr(ap)[fn_index]
        fm = _exact_inv_fr(am)[fn_index]
        g.append(float((fp - fm) / (2 * h)))
    return float(np.linalg.norm(g))


def _exact_inv_fr(afr):
    A = [[afr[3 * i + j] for j in range(3)] for i in range(3)]
    I1 = A[0][0] + A[1][1] + A[2][2]
    S = [[A[i][j] - (I1 / 3 if i == j else 0) for j in range(3)] for i in range(3)]
    S2 = refs.matmul3(S, S)
    J2 = (S2[0][0] + S2[1][1] + S2[2][2]) / 2
    J3 = refs.det3(S)
    return I1, J2, J3, 4 * J2 ** 3 - 27 * J3 ** 2


def test_bound_jacobian_norms(oracle_mod):
    """The bound calculator's Jacobian norms equal the norms of finite-difference
    gradients of the exact invariants (Jacobians of J2, J3, Delta in the paper)."""
    rng = np.random.default_rng(9)
    for _ in range(8):
        a9 = rng.standard_normal(9)
        b = oracle_mod.bounds(a9, 1.0)[0]
        nS = np.sqrt(b[1] / U64)
        assert abs(_exact_grad_norm(1, a9) - nS) <= 1e-9 * nS
        assert abs(_exact_grad_norm(2, a9) - b[2] / (nS * U64)) <= 1e-9 * b[2] / (nS * U64)
        assert abs(_exact_grad_norm(3, a9) - b[3] / (nS * U64)) <= 1e-9 * b[3] / (nS * U64)
