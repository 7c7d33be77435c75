"""GPU parity of the adjoint kernel (eig3_eigvals_backward) against the
oracle's eigenvector form l r^T / (l^T r), finite differences, and the
gradient of cluster sums near repeated eigenvalues."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests import gpu_util as U

pytestmark = pytest.mark.gpu
GEN, SYM = 0, 1


@pytest.fixture(scope="module")
def eig3():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_00292_gb300 as m
    return m


def dev():
    return torch.device("cuda:0")


def rel_gap(lam):
    lam = np.sort(lam, axis=1)
    g = np.minimum(lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 1])
    return g / np.maximum(np.abs(lam).max(axis=1), 1e-300)


def grad_tol(A, kappa, lam, gbar):
    """Gradient error bound: the eigenprojector's sensitivity ~ kappa^2 ||A|| u / gap."""
    lam = np.sort(lam, axis=1)
    gap = np.minimum(lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 1])
    nA = np.linalg.norm(A, axis=1)
    scale = np.abs(gbar).sum(axis=1) * np.asarray(kappa) ** 2
    return 64.0 * U.U64 * scale * (1.0 + nA / np.maximum(gap, 1e-300))


@pytest.mark.parametrize("with_aux", [True, False])
def test_backward_vs_eigenvector_form(eig3, with_aux):
    bt = W.workload4(n=50_001, device="cpu", seed=1404)
    A = bt.A.to(dev())
    w = bt.extra["w"].to(dev())
    lam, aux = eig3.eigvals(A, return_aux=True)
    G = U.to_np(eig3.eigvals_backward(A, w, aux=aux if with_aux else None))
    An = bt.A.numpy()
    lam_n = U.to_np(lam)
    sel = rel_gap(lam_n) >= 1e-4
    assert sel.sum() > 10_000
    ref = oracle.eigvals_grad(An[sel], bt.extra["w"].numpy()[sel])
    err = np.abs(G[sel] - ref).max(axis=1)
    tol = grad_tol(An[sel], bt.kappa.numpy()[sel], lam_n[sel], bt.extra["w"].numpy()[sel])
    print(f"[grad] aux={with_aux} n={sel.sum()} max err/tol {np.max(err / tol):.3g}")
    assert np.all(err <= tol)


def test_autograd_function_and_gradcheck(eig3):
    bt = W.gradient_batch(n=64, device="cpu", seed=1405)
    A = bt.A.to(dev()).requires_grad_(True)
    w = torch.randn(64, 3, dtype=torch.float64, device=dev())
    lam = eig3.eigvals_ad(A)
    (lam * w).sum().backward()
    ref = oracle.eigvals_grad(bt.A.numpy(), w.cpu().numpy())
    assert np.abs(U.to_np(A.grad) - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
    # torch's central finite differences, eps = 1e-6 (the workload's h)
    A2 = bt.A[:8].to(dev()).clone().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: eig3.eigvals_ad(x), (A2,), eps=1e-6, atol=1e-6,
                                    rtol=1e-5)


def test_cluster_sums_near_repeated(eig3):
    """Below the 1e-4 gap the individual eigenvalue gradients are ill-posed; the
    gradient of a cluster's sum is not.  With equal weights inside the cluster
    the adjoint must match I - (gradient of the isolated eigenvalue) terms."""
    bt = W.workload2(n=60_000, device="cpu", seed=1406)
    kinds = bt.extra["kinds"].numpy()
    An = bt.A.numpy()
    lam = np.sort(oracle.eigvals(An), axis=1)
    lo = lam[:, 1] - lam[:, 0]
    hi = lam[:, 2] - lam[:, 1]
    scale = np.maximum(np.abs(lam).max(axis=1), 1e-300)
    # pair (lambda_1, lambda_2) nearly equal, lambda_3 well separated
    s12 = (kinds == 1) & (lo / scale < 1e-4) & (hi / scale > 1e-2)
    s23 = (kinds == 1) & (hi / scale < 1e-4) & (lo / scale > 1e-2)
    rng = np.random.default_rng(0)
    for sel, iso in ((s12, 2), (s23, 0)):
        m = int(sel.sum())
        assert m > 100
        w_iso = rng.standard_normal(m)
        gbar = np.ones((m, 3))
        gbar[:, iso] = w_iso
        A = torch.as_tensor(An[sel], device=dev())
        G = U.to_np(eig3.eigvals_backward(A, torch.as_tensor(gbar, device=dev())))
        # sum(lambda) = I1 -> gradient I; the isolated eigenvalue adds (w - 1) G_iso
        # (only the isolated eigenvalue's Jacobian is well defined here)
        G_iso = oracle.eigval_jacobians(An[sel])[:, iso, :]
        ref = (w_iso - 1.0)[:, None] * G_iso
        ref[:, [0, 4, 8]] += 1.0
        err = np.abs(G - ref).max(axis=1)
        nA = np.linalg.norm(An[sel], axis=1)
        k = bt.kappa.numpy()[sel]
        gap_iso = np.where(iso == 2, hi[sel], lo[sel])
        tol = 64.0 * U.U64 * k ** 2 * (1 + np.abs(w_iso)) * (1.0 + nA / gap_iso)
        print(f"[grad] cluster iso={iso} m={m} max err/tol {np.max(err / tol):.3g}")
        assert np.all(err <= tol)


def test_backward_sym6_and_f32(eig3):
    w1 = W.workload1("cpu")["sym6"]
    S = w1.A.to(dev())
    g = torch.randn(S.shape[0], 3, dtype=torch.float64, device=dev())
    lam = U.to_np(eig3.eigvals(S))
    G = U.to_np(eig3.eigvals_backward(S, g))
    sel = rel_gap(lam) >= 1e-3
    ref = oracle.eigvals_grad(w1.A.numpy()[sel], g.cpu().numpy()[sel], layout=SYM)
    assert np.abs(G[sel] - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
    # binary32 storage: binary64 adjoint rounded once, and the compensated one
    S32 = S.float()
    g32 = g.float()
    S32n = S32.double().cpu().numpy()
    g32n = g32.double().cpu().numpy()
    for prec in ("f64", "f32c"):
        lam32, aux = eig3.eigvals(S32, precision=prec, return_aux=True)
        G32 = U.to_np(eig3.eigvals_backward(S32, g32, aux=aux, precision=prec))
        lam32n = U.to_np(lam32)
        sel32 = sel & (rel_gap(lam32n) >= 1e-3)
        r = oracle.eigvals_grad(S32n[sel32], g32n[sel32], layout=SYM)
        err = np.abs(G32[sel32] - r).max(axis=1)
        scale = np.abs(g32n[sel32]).sum(axis=1)
        gap = rel_gap(lam32n[sel32])
        tol = 64.0 * U.U32 * scale / gap
        print(f"[grad] sym6 f32 {prec}: max err/tol {np.max(err / tol):.3g}")
        assert np.all(err <= tol)
