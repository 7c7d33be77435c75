"""GPU tests of the guarded binary64 precision (EIG3_PREC_F64_GUARDED, "f64g"),
the library's answer to the limitation that Sections J3, Delta and
Eigenvalues report for ill-conditioned eigenbases.

Reference: oracle.eigvals_exact, the exact eigenvalues of the stored matrix.
Bound: b = kappa ||A||_F u (the first-order eigenvalue bound, C = 1); the
tolerance is 8 b, as for the binary64 path on well-conditioned input.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests import gpu_util as U

pytestmark = pytest.mark.gpu
C = 8.0


@pytest.fixture(scope="module")
def eig3():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_00292_gb300 as m
    return m


def dev():
    return torch.device("cuda:0")


def err_over_bound(lam, exact, X, kappa):
    b = oracle.bounds(X, kappa)[:, 4]
    return np.abs(lam - exact).max(axis=1) / b


def test_paper_u2_paths(eig3):
    """The nearly singular U2(1e-3) (kappa ~ 9e3) on both paths: the binary64
    path exceeds the bound (as the paper reports), the guarded one does not."""
    P = [p for p in W.paper_paths(deltas=np.logspace(-1, -12, 23))]
    X = np.array([p["A"] for p in P])
    kap = np.array([p["kappa"] for p in P])
    ex = oracle.eigvals_exact(X)
    ok = np.all(np.isfinite(ex), axis=1)
    A = torch.as_tensor(X, device=dev())
    st = eig3.Stats(dev())
    lg = U.to_np(eig3.eigvals(A, precision="f64g", stats=st))
    lp = U.to_np(eig3.eigvals(A))
    rg = err_over_bound(lg, ex, X, kap)
    rp = err_over_bound(lp, ex, X, kap)
    u2 = np.array([p["U"] == "u2" for p in P])
    print(f"[guard] U2 paths: plain max {rp[ok & u2].max():.3g} bounds, "
          f"guarded max {rg[ok & u2].max():.3g}; switched {st.read()['n_guarded']}")
    assert rp[ok & u2].max() > C
    assert np.all(rg[ok] <= C)
    assert st.read()["n_guarded"] >= u2.sum() // 2


def test_ill_conditioned_batch(eig3):
    bt = W.illconditioned(3000, "cpu", seed=9101, log10_kappa_max=5.0)
    X = bt.A.numpy()
    ex = oracle.eigvals_exact(X)
    ok = np.all(np.isfinite(ex), axis=1)
    A = bt.A.to(dev())
    st = eig3.Stats(dev())
    lg = U.to_np(eig3.eigvals(A, precision="f64g", stats=st))
    lp = U.to_np(eig3.eigvals(A))
    k = bt.kappa.numpy()
    rg = err_over_bound(lg, ex, X, k)
    rp = err_over_bound(lp, ex, X, k)
    n_ref = st.read()["n_guarded"]
    print(f"[guard] kappa <= 1e5: plain beyond {C:g} bounds {np.mean(rp[ok] > C):.3f}, "
          f"max {rp[ok].max():.3g}; guarded max {rg[ok].max():.3g}; switched {n_ref}/{len(X)}")
    assert np.mean(rp[ok] > C) > 0.3
    assert np.all(rg[ok] <= C)
    # every row on which the binary64 path fails its bound was switched
    changed = np.any(lg != lp, axis=1)
    assert np.all(changed[ok & (rp > C)])
    assert 0 < n_ref <= len(X)


def test_unswitched_rows_are_the_binary64_results(eig3):
    bt = W.workload2(n=200_003, device="cpu", seed=9102)
    X = bt.A.numpy()
    A = bt.A.to(dev())
    st = eig3.Stats(dev())
    lg = eig3.eigvals(A, precision="f64g", stats=st)
    lp = eig3.eigvals(A)
    diff = (lg != lp).any(dim=1).cpu().numpy()
    n_ref = st.read()["n_guarded"]
    # rho = ||dev A||_F^2 / tr(dev(A)^2); rows clearly below the threshold of 32
    M = X.reshape(-1, 3, 3)
    S = M - np.trace(M, axis1=1, axis2=2)[:, None, None] / 3 * np.eye(3)
    trS2 = np.einsum("nij,nji->n", S, S)
    rho = (S * S).sum(axis=(1, 2)) / np.where(trS2 > 0, trS2, np.nan)
    # where tr(S^2) is at the level of rounding noise (spectra coalesced to a
    # few ulps) the computed ratio is noise too, on either side
    noise = ~(trS2 > 1e-29 * (X * X).sum(axis=1))
    print(f"[guard] workload 2: switched {n_ref} of {len(X)}, rows changed {diff.sum()}, "
          f"noise-level rows {noise.sum()}")
    assert diff.sum() <= n_ref
    assert not diff[(rho < 30) & ~noise].any()
    assert n_ref <= np.count_nonzero((rho > 31) | noise)


def test_symmetric_input_is_never_switched(eig3):
    S = W.workload1("cpu")["sym6"].A.to(dev())
    st = eig3.Stats(dev())
    assert torch.equal(eig3.eigvals(S, precision="f64g", stats=st), eig3.eigvals(S))
    assert st.read()["n_guarded"] == 0
    X9 = torch.as_tensor(oracle.sym6_to_general9(S.cpu().numpy()), device=dev())
    st.reset()
    assert torch.equal(eig3.eigvals(X9, precision="f64g", stats=st), eig3.eigvals(X9))
    assert st.read()["n_guarded"] == 0


def test_guarded_precision_is_for_eigenvalues_only(eig3):
    A = W.workload2(n=100, device="cpu", seed=9103).A.to(dev())
    with pytest.raises(eig3.Eig3Error):
        eig3.invariants(A, precision="f64g")
    with pytest.raises(eig3.Eig3Error):
        eig3.eigprojectors(A, precision="f64g")


def test_switched_adjoint_inputs_match_the_gaps(eig3):
    """For a switched matrix the adjoint inputs come from the QR eigenvalues:
    the gaps of the trigonometric form, (2 r / sqrt3) sigma1 and
    (2 r / sqrt3) sigma2, reproduce lambda2 - lambda1 and lambda3 - lambda2."""
    bt = W.illconditioned(5000, "cpu", seed=9105, log10_kappa_max=4.0)
    A = bt.A.to(dev())
    lam, aux = eig3.eigvals(A, precision="f64g", return_aux=True)
    lam, aux = U.to_np(lam), U.to_np(aux)
    r, s1, s2 = aux[:, 0], aux[:, 1], aux[:, 2]
    g12 = 2 * r / np.sqrt(3) * s1
    g23 = 2 * r / np.sqrt(3) * s2
    scale = np.abs(lam).max(axis=1)
    ok = np.isfinite(lam).all(axis=1)
    assert np.all(np.abs(g12 - (lam[:, 1] - lam[:, 0]))[ok] <= 64 * U.U64 * scale[ok])
    assert np.all(np.abs(g23 - (lam[:, 2] - lam[:, 1]))[ok] <= 64 * U.U64 * scale[ok])
    assert np.all(np.abs(s1 * s1 + s1 * s2 + s2 * s2 - 0.75)[ok & (r > 0)] <= 1e-14)


def test_binary32_storage_and_backward(eig3):
    bt = W.illconditioned(2000, "cpu", seed=9104, log10_kappa_max=4.0)
    A32 = bt.A.float().to(dev())
    X = A32.double().cpu().numpy()
    ex = oracle.eigvals_exact(X)
    ok = np.all(np.isfinite(ex), axis=1)
    lg = U.to_np(eig3.eigvals(A32, precision="f64g"))
    b = C * oracle.bounds(X, bt.kappa.numpy())[:, 4]
    tol = b[:, None] + 0.5 * np.spacing(np.maximum(np.abs(ex), np.abs(lg)).astype(np.float32))
    assert np.all((np.abs(lg - ex) <= tol)[ok])
    # the adjoint: with the guarded adjoint inputs, or recomputing them
    A = bt.A.to(dev())
    w = torch.randn(A.shape[0], 3, dtype=torch.float64, device=dev())
    lam, aux = eig3.eigvals(A, precision="f64g", return_aux=True)
    g1 = eig3.eigvals_backward(A, w, aux=aux, precision="f64g")
    g2 = eig3.eigvals_backward(A, w, precision="f64g")
    assert torch.equal(g1, g2)
    assert torch.isfinite(g1[torch.as_tensor(ok, device=dev())]).all()


def test_switched_adjoint_against_lapack_eigenvectors(eig3):
    """The adjoint on the rows the guard switches to QR (strongly non-normal,
    kappa up to 1e4): the chain-rule gradient from the QR eigenvalue gaps
    against d lambda_k / dA_ij = (V^-1)_ki V_jk from LAPACK's eigenvectors V,
    where the spectrum is real and the relative gap >= 1e-4.  The oracle's
    own eigenvector form is not used here: it starts from the closed-form
    eigenvalues, which are what lose accuracy on these matrices.  Tolerance:
    the gradient's sensitivity, kappa^2 (1 + ||A|| / gap) u per unit weight,
    with the divided differences' own amplification (||A|| / gap)^2."""
    bt = W.illconditioned(20_000, "cpu", seed=9106, log10_kappa_max=4.0)
    X = bt.A.numpy()
    S = X.reshape(-1, 3, 3) - np.einsum("nii->n", X.reshape(-1, 3, 3))[:, None, None] / 3 * np.eye(3)
    fro2 = (S * S).sum(axis=(1, 2))
    trS2 = np.einsum("nij,nji->n", S, S)
    switched = fro2 > 40.0 * np.maximum(trS2, 0.0)          # beyond the guard's 32, with margin
    ex = oracle.eigvals_exact(X[switched])
    real = np.all(np.isfinite(ex), axis=1)
    scale = np.abs(ex).max(axis=1)
    gap = np.minimum(ex[:, 1] - ex[:, 0], ex[:, 2] - ex[:, 1])
    sel = real & (gap >= 1e-4 * scale)
    idx = np.nonzero(switched)[0][sel]
    assert idx.size > 500
    A = torch.as_tensor(X[idx], device=dev())
    w = torch.randn(idx.size, 3, dtype=torch.float64, device=dev(),
                    generator=torch.Generator(dev()).manual_seed(11))
    st = eig3.Stats(dev())
    lam, aux = eig3.eigvals(A, precision="f64g", return_aux=True, stats=st)
    assert st.read()["n_guarded"] == idx.size
    G = U.to_np(eig3.eigvals_backward(A, w, aux=aux, precision="f64g"))
    wn = w.cpu().numpy()
    M = X[idx].reshape(-1, 3, 3)
    ev, V = np.linalg.eig(M)
    order = np.argsort(ev.real, axis=1)
    ev = np.take_along_axis(ev, order, axis=1)
    V = np.take_along_axis(V, order[:, None, :], axis=2)
    Vi = np.linalg.inv(V)
    ref = np.einsum("nk,nki,njk->nij", wn, Vi, V).real.reshape(-1, 9)
    nA = np.linalg.norm(X[idx], axis=1)
    g = gap[sel]
    k2 = bt.kappa.numpy()[idx] ** 2
    tol = 64.0 * U.U64 * np.abs(wn).sum(axis=1) * (k2 * (1.0 + nA / g) + (nA / g) ** 2)
    err = np.abs(G - ref).max(axis=1)
    print(f"[guard] switched adjoint on {idx.size} rows: max err/tol {np.max(err / tol):.3g}, "
          f"max |G| {np.abs(ref).max():.3g}")
    assert np.all(err <= tol)
