"""GPU results against the exact values of the stored matrices
(oracle.eigvals_exact, oracle.invariants_exact: rational and 60-digit
arithmetic), in units of the paper's first-order bounds (Lemma of Section
"Eigenvalues": kappa ||A||_F u; Sections I1, J2, J3, Delta for the
invariants).  Unlike the parity tests, which allow the oracle's own error
beside the GPU's, these bound the GPU's distance from the exact result alone:
eigenvalues within C = 8 bounds (binary64; the compensated binary32 path
within 8 bounds at u = 2^-24 plus its final rounding), invariants within 16
bounds, J3 and Delta kappa^2-scaled as the paper shows them only
conditionally stable."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests import gpu_util as U

pytestmark = pytest.mark.gpu
GEN, SYM = 0, 1
N = 1 << 13


@pytest.fixture(scope="module")
def eig3():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2511_00292_gb300 as m
    return m


def dev():
    return torch.device("cuda:0")


def cases():
    w1 = W.workload1("cpu")
    b2 = W.workload2(n=N, device="cpu", seed=2202)
    b4 = W.workload4(n=N, device="cpu", seed=2204)
    w5 = W.workload5(n=2 * N, device="cpu", seed=2205)
    return [
        ("workload1 general9", w1["general9"].A.numpy(), GEN, np.ones(w1["general9"].n)),
        ("workload1 sym6", w1["sym6"].A.numpy(), SYM, np.ones(w1["sym6"].n)),
        ("workload2", b2.A.numpy(), GEN, b2.kappa.numpy()),
        ("workload4", b4.A.numpy(), GEN, b4.kappa.numpy()),
        ("workload5 general half", w5["general9"].A.numpy(), GEN, w5["general9"].kappa.numpy()),
    ]


@pytest.mark.parametrize("case", range(5))
def test_binary64_eigenvalues_within_8_bounds_of_exact(eig3, case):
    name, A, lay, kappa = cases()[case]
    X = torch.as_tensor(A, device=dev())
    lam = U.to_np(eig3.eigvals(X, layout=lay))
    ex = oracle.map_eigvals_exact(A, lay, 8)
    real = np.all(np.isfinite(ex), axis=1)            # complex spectra of fl(A) are NaN
    b = oracle.bounds(A, kappa, layout=lay)[:, 4]
    err = np.abs(lam - ex)[real].max(axis=1)
    tol = 8.0 * b[real] + 2.0 * np.spacing(np.abs(ex[real]).max(axis=1))
    r = err / tol
    print(f"[exact] {name}: {real.sum()} real spectra, max err/(8 bounds) {r.max():.3g}, "
          f"p99.9 {np.quantile(r, 0.999):.3g}")
    assert np.all(err <= tol)
    # the fused path's eigenvalues are the same numbers
    if lay == GEN:
        w = torch.zeros(X.shape[0], 3, dtype=torch.float64, device=dev())
        assert torch.equal(eig3.eigvals_vjp(X, w)[0], eig3.eigvals(X))


def test_compensated_binary32_within_8_bounds_of_exact(eig3):
    """Workload 3 and the symmetric half of workload 5, both binary32: the
    exact eigenvalues of the stored binary32 matrices."""
    for name, S in (("workload3", W.workload3(n=N, device="cpu", seed=2203).A),
                    ("workload5 symmetric half", W.workload5(n=2 * N, device="cpu",
                                                             seed=2205)["sym6"].A)):
        lam = U.to_np(eig3.eigvals(S.to(dev()), precision="f32c"))
        A = S.double().numpy()
        ex = oracle.map_eigvals_exact(A, SYM, 8)
        b = oracle.bounds(A, 1.0, layout=SYM, u=U.U32)[:, 4]
        ulp = np.spacing(np.abs(ex).max(axis=1).astype(np.float32)).astype(np.float64)
        err = np.abs(lam - ex).max(axis=1)
        tol = 8.0 * b + 2.0 * ulp
        print(f"[exact] {name} f32c: max err/tol {np.max(err / tol):.3g}, "
              f"max {np.max(err / np.where(ulp > 0, ulp, 1)):.2f} ulp")
        assert np.all(err <= tol)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_invariants_within_16_bounds_of_exact(eig3, prec):
    if prec == "f64":
        b2 = W.workload2(n=N, device="cpu", seed=2206)
        A, lay, kappa, u = b2.A.numpy(), GEN, b2.kappa.numpy(), U.U64
        X = torch.as_tensor(A, device=dev())
    else:
        S = W.workload3(n=N, device="cpu", seed=2207).A
        A, lay, kappa, u = S.double().numpy(), SYM, np.ones(N), U.U32 ** 2
        X = S.to(dev())
    inv = U.to_np(eig3.invariants(X, layout=lay, precision=prec))
    ex = oracle.map_invariants_exact(A, lay, 8)
    b = oracle.bounds(A, kappa, layout=lay, u=u)[:, :4]
    k2 = np.asarray(kappa) ** 2
    scale = np.stack([np.ones(N), np.ones(N), k2, k2], axis=1)
    err = np.abs(inv - ex)
    tol = 16.0 * scale * b
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(err == 0, 0.0, err / tol)
    print(f"[exact] invariants {prec}: max err/tol per (I1, J2, J3, Delta) "
          f"{[float(x) for x in r.max(axis=0)]}")
    assert np.all(err <= tol)
