"""Eigenprojectors (eig3_eigprojectors) against the oracle's eigenvector form
(E_k = r_k l_k^T / (l_k^T r_k), the transpose of d lambda_k / dA) and against
the identities that hold at any size: sum_k E_k = I, A E_k = lambda_k E_k,
E_k^2 = E_k, and symmetry for symmetric input."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eig3():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_00292_gb300 as m
    return m


def dev():
    return torch.device("cuda:0")


def gap_of(lam):
    lam = np.sort(lam, axis=1)
    return np.minimum(lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 1])


def test_projectors_vs_eigenvector_form(eig3):
    bt = W.workload2(n=60_001, device="cpu", seed=2300)
    An = bt.A.numpy()
    P, lam = eig3.eigprojectors(bt.A.to(dev()), return_eigvals=True)
    P = U.to_np(P).reshape(-1, 3, 9)
    lam = U.to_np(lam)
    assert np.array_equal(lam, U.to_np(eig3.eigvals(bt.A.to(dev()))))
    gap = gap_of(lam)
    sel = gap / np.abs(lam).max(axis=1) >= 1e-4
    Jt = oracle.eigval_jacobians(An[sel]).reshape(-1, 3, 3, 3).transpose(0, 1, 3, 2).reshape(-1, 3, 9)
    err = np.abs(P[sel] - Jt).max(axis=(1, 2))
    k = bt.kappa.numpy()[sel]
    tol = 64 * U.U64 * k ** 2 * (1 + np.linalg.norm(An[sel], axis=1) / gap[sel]) * \
        np.maximum(1.0, np.abs(Jt).max(axis=(1, 2)))
    print(f"[proj] n={sel.sum()} max err/tol {np.max(err / tol):.3g}")
    assert np.all(err <= tol)


def test_projector_identities_any_size(eig3):
    bt = W.workload2(n=1 << 20, device=dev(), seed=2301)
    P, lam = eig3.eigprojectors(bt.A, return_eigvals=True)
    A = bt.A.reshape(-1, 3, 3)
    E = P                                                   # (n, 3, 3, 3)
    I = torch.eye(3, dtype=torch.float64, device=dev())
    lamn = lam.cpu().numpy()
    gap = torch.as_tensor(gap_of(lamn), device=dev())
    nA0 = torch.linalg.matrix_norm(A)
    # sum_k E_k = I holds for any spectrum; the terms of each E_k are of size
    # ~ ||A|| / gap and cancel, so rounding enters at u ||A|| / gap
    resid_sum = (E.sum(dim=1) - I).abs().amax(dim=(1, 2))
    tol_sum = 64 * U.U64 * (1 + nA0 / gap.clamp_min(1e-300))
    assert bool((resid_sum <= tol_sum).all()), float((resid_sum / tol_sum).max())
    # A E_k = lambda_k E_k and E_k^2 = E_k where the spectrum is separated
    scale = lam.abs().amax(dim=1)
    sep = gap / scale >= 1e-3
    As, Es, ls = A[sep], E[sep], lam[sep]
    nA = torch.linalg.matrix_norm(As).unsqueeze(1)
    kap = bt.kappa[sep].unsqueeze(1)
    r1 = (As.unsqueeze(1) @ Es - ls.unsqueeze(-1).unsqueeze(-1) * Es).abs().amax(dim=(2, 3))
    tol1 = 256 * U.U64 * kap ** 2 * nA * (1 + nA / gap[sep].unsqueeze(1)) * \
        Es.abs().amax(dim=(2, 3))
    assert bool((r1 <= tol1).all()), float((r1 / tol1).max())
    r2 = (Es @ Es - Es).abs().amax(dim=(2, 3))
    tol2 = 256 * U.U64 * kap ** 2 * (1 + nA / gap[sep].unsqueeze(1)) * Es.abs().amax(dim=(2, 3)) ** 2
    assert bool((r2 <= tol2).all()), float((r2 / tol2).max())


def test_projectors_symmetric_and_sym6(eig3):
    """Both layouts give the same projectors, and symmetric ones, where they are
    well conditioned: for separated spectra all three, for a near-repeated pair
    the projector of the isolated eigenvalue (the pair's own ones depend on its
    splitting at the level u / gap)."""
    w1 = W.workload1("cpu")
    Pg = U.to_np(eig3.eigprojectors(w1["general9"].A.to(dev())))
    Ps = U.to_np(eig3.eigprojectors(w1["sym6"].A.to(dev())))
    lam = np.sort(oracle.eigvals(w1["general9"].A.numpy()), axis=1)
    thr = 1e-3
    lo = lam[:, 1] - lam[:, 0] >= thr
    hi = lam[:, 2] - lam[:, 1] >= thr
    both = lo & hi
    assert np.abs(Pg[both] - Ps[both]).max() <= 1e-10
    assert np.abs(Ps[both] - Ps[both].transpose(0, 1, 3, 2)).max() <= 1e-10
    iso3 = ~lo & hi            # lambda_1 ~ lambda_2: E_3 is well conditioned
    iso1 = lo & ~hi            # lambda_2 ~ lambda_3: E_1 is
    assert iso3.sum() > 10 and iso1.sum() >= 0
    assert np.abs(Pg[iso3, 2] - Ps[iso3, 2]).max() <= 1e-10
    if iso1.any():
        assert np.abs(Pg[iso1, 0] - Ps[iso1, 0]).max() <= 1e-10
    # the pair's projector is I - E_3 (well conditioned); E_1 + E_2 summed from
    # the individual ones carries their u ||A|| / gap rounding
    I = np.eye(3)
    gap = (lam[:, 1] - lam[:, 0])[iso3]
    nA = np.linalg.norm(w1["general9"].A.numpy()[iso3], axis=1)
    resid = np.abs(Ps[iso3, 0] + Ps[iso3, 1] + Ps[iso3, 2] - I).max(axis=(1, 2))
    assert np.all(resid <= 256 * U.U64 * (1 + nA / np.maximum(gap, 1e-300)))


def _diag_rows(vals):
    A = np.zeros((len(vals), 9))
    for i, v in enumerate(vals):
        A[i, [0, 4, 8]] = v
    return A


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_exact_coalescence_takes_the_cluster_mean(eig3, prec):
    """Where two computed eigenvalues coincide exactly the individual
    eigenvalues have no derivative; the library gives each the mean of the
    pair's weights, i.e. the gradient of the pair's mean.  Diagonal matrices
    make the computed gap exactly zero."""
    dt = torch.float64 if prec == "f64" else torch.float32
    A = torch.as_tensor(_diag_rows([(1.0, 1.0, 2.0), (1.0, 2.0, 2.0), (-3.0, 0.5, 0.5)]),
                        dtype=dt, device=dev())
    g = torch.tensor([[1.0, 3.0, 5.0]] * 3, dtype=dt, device=dev())
    G = U.to_np(eig3.eigvals_backward(A, g, precision=prec)).reshape(-1, 3, 3)
    want = np.stack([np.diag([2.0, 2.0, 5.0]), np.diag([1.0, 4.0, 4.0]), np.diag([1.0, 4.0, 4.0])])
    tol = 1e-12 if prec == "f64" else 1e-5
    assert np.abs(G - want).max() <= tol, G
    P = U.to_np(eig3.eigprojectors(A, precision=prec))
    E12 = np.diag([0.5, 0.5, 0.0])
    assert np.abs(P[0, 0] - E12).max() <= tol and np.abs(P[0, 1] - E12).max() <= tol
    assert np.abs(P[0, 2] - np.diag([0.0, 0.0, 1.0])).max() <= tol
    assert np.abs(P[1, 0] - np.diag([1.0, 0.0, 0.0])).max() <= tol
    assert np.abs(P[1, 1] - np.diag([0.0, 0.5, 0.5])).max() <= tol


def test_projectors_f32c(eig3):
    S = W.workload3(n=50_001, device="cpu", seed=2302).A
    P = U.to_np(eig3.eigprojectors(S.to(dev()), precision="f32c"))
    S64 = S.double().numpy()
    lam = np.sort(oracle.eigvals(S64, layout=oracle.SYM6), axis=1)
    gap = gap_of(lam) / np.maximum(np.abs(lam).max(axis=1), 1e-300)
    sel = gap >= 1e-2
    Jt = oracle.eigval_jacobians(S64[sel], layout=oracle.SYM6).reshape(-1, 3, 3, 3)
    Jt = Jt.transpose(0, 1, 3, 2)
    err = np.abs(P[sel] - Jt).max(axis=(1, 2, 3))
    tol = 64 * U.U32 / gap[sel]
    print(f"[proj] f32c n={sel.sum()} max err/tol {np.max(err / tol):.3g}")
    assert np.all(err <= tol)


@pytest.mark.parametrize("layout", ["sym6", "general9"])
def test_projectors_f32c_output_alignment_and_ragged_tiles(eig3, layout):
    """The binary32 kernel writes each tile's outputs back through shared
    memory: with 16-byte stores when the output is 16-byte aligned, element
    stores otherwise.  Both give the same bytes, for every tile size."""
    S = W.workload3(n=3 * 256 + 77, device="cpu", seed=2303).A
    X = S if layout == "sym6" else torch.as_tensor(oracle.sym6_to_general9(S.double().numpy()),
                                                    dtype=torch.float32)
    Xd = X.to(dev())
    n = Xd.shape[0]
    P, lam = eig3.eigprojectors(Xd, layout=layout, precision="f32c", return_eigvals=True)
    bufP = torch.full((n * 27 + 1,), float("nan"), dtype=torch.float32, device=dev())
    bufL = torch.full((n * 3 + 1,), float("nan"), dtype=torch.float32, device=dev())
    P1, lam1 = eig3.eigprojectors(Xd, layout=layout, precision="f32c", return_eigvals=True,
                                  out=bufP[1:].view(n, 3, 3, 3), lam_out=bufL[1:].view(n, 3))
    assert torch.equal(P, P1) and torch.equal(lam, lam1)
    assert torch.isnan(bufP[0]) and torch.isnan(bufL[0])
    assert torch.equal(lam, eig3.eigvals(Xd, layout=layout, precision="f32c"))
    for m in (1, 255, 256, 257):
        Pm = eig3.eigprojectors(Xd[:m], layout=layout, precision="f32c")
        assert torch.equal(Pm, P[:m])
