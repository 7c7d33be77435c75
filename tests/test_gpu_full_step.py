"""The benchmark's step at its full size, in its launch configuration: the
mixed workload of 2^28 matrices (2^27 symmetric binary32 through the
compensated kernel, 2^27 general binary64 through the binary64 kernel),
forward + vector-Jacobian product fused per half (eig3_eigvals_vjp) with the
binary32 launch on a second stream beside the binary64 one, run three times
(statistics over the last two).  Sampled outputs of both halves are compared
with the oracle (eigenvalues on 2^20 samples per half, eigenvector-form
gradients on 2^18), and the statistics with properties that hold at any
size."""
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


def rel_gap(lam):
    lam = np.sort(lam, axis=1)
    g = np.minimum(lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 1])
    return g / np.maximum(np.abs(lam).max(axis=1), 1e-300)


def test_full_size_mixed_step(eig3):
    dev = torch.device("cuda:0")
    w5 = W.workload5(n=1 << 28, device=dev)
    S, G = w5["sym6"], w5["general9"]
    lamS = torch.empty(S.n, 3, dtype=torch.float32, device=dev)
    gS = torch.empty_like(S.A)
    lamG = torch.empty(G.n, 3, dtype=torch.float64, device=dev)
    gG = torch.empty_like(G.A)
    st = eig3.Stats(dev)
    s64, s32 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def step():
        cur = torch.cuda.current_stream(dev)
        s64.wait_stream(cur)
        s32.wait_stream(cur)
        with torch.cuda.stream(s64):
            eig3.eigvals_vjp(G.A, G.extra["w"], precision="f64", out=lamG, grad_out=gG, stats=st)
        with torch.cuda.stream(s32):
            eig3.eigvals_vjp(S.A, S.extra["w"], precision="f32c", out=lamS, grad_out=gS,
                             stats=st)
        cur.wait_stream(s64)
        cur.wait_stream(s32)

    step()
    torch.cuda.synchronize()
    st.reset()
    step()
    step()
    torch.cuda.synchronize()
    stats = st.read()
    assert stats["n_nonfinite"] == 0
    assert 0.0 <= stats["min_disc_ratio"] <= 4.0
    maxabs = max(float(lamS.abs().max()), float(lamG.abs().max()))
    assert stats["max_abs_lambda"] == pytest.approx(maxabs, rel=1e-6)

    # binary64 half: eigenvalues and gradients on samples
    idx = torch.as_tensor(W.sample_indices(G.n, 1 << 20, seed=9201), device=dev)
    XG = U.to_np(G.A[idx])
    kG = U.to_np(G.kappa[idx])
    err, tol, bad = U.check_eig_f64(U.to_np(lamG[idx]), XG, kG, GEN)
    print(f"[full step] binary64 eigenvalues on {idx.numel()}: max err/tol {np.max(err / tol):.3g}")
    assert not bad.any()
    idx = idx[:1 << 18]
    XG, kG = XG[:1 << 18], kG[:1 << 18]
    wG = U.to_np(G.extra["w"][idx])
    lam_ref = oracle.eigvals(XG)
    sel = rel_gap(lam_ref) >= 1e-4
    gref = oracle.eigvals_grad(XG[sel], wG[sel])
    nA = np.linalg.norm(XG[sel], axis=1)
    lam_s = np.sort(lam_ref[sel], axis=1)
    gap = np.minimum(lam_s[:, 1] - lam_s[:, 0], lam_s[:, 2] - lam_s[:, 1])
    gtol = 64.0 * U.U64 * np.abs(wG[sel]).sum(axis=1) * kG[sel] ** 2 * (1.0 + nA / gap)
    gerr = np.abs(U.to_np(gG[idx])[sel] - gref).max(axis=1)
    print(f"[full step] binary64 gradients: max err/tol {np.max(gerr / gtol):.3g} on {sel.sum()}")
    assert np.all(gerr <= gtol)

    # compensated binary32 half
    idx = torch.as_tensor(W.sample_indices(S.n, 1 << 20, seed=9202), device=dev)
    XS = U.to_np(S.A[idx])
    err, tol, _ = U.check_eig_f32c(U.to_np(lamS[idx]), XS, 1.0, SYM)
    print(f"[full step] binary32 eigenvalues on {idx.numel()}: max err/tol {np.max(err / tol):.3g}")
    assert np.all(err <= tol)
    idx = idx[:1 << 18]
    XS = XS[:1 << 18]
    wS = U.to_np(S.extra["w"][idx])
    lam_ref = oracle.eigvals(XS, layout=SYM)
    sel = rel_gap(lam_ref) >= 1e-3
    gref = oracle.eigvals_grad(XS[sel], wS[sel], layout=SYM)
    gerr = np.abs(U.to_np(gS[idx])[sel] - gref).max(axis=1)
    gtol = 64.0 * U.U32 * np.abs(wS[sel]).sum(axis=1) / rel_gap(lam_ref[sel]) * (
        1.0 + np.abs(gref).max(axis=1))
    print(f"[full step] binary32 gradients: max err/tol {np.max(gerr / gtol):.3g} on {sel.sum()}")
    assert np.all(gerr <= gtol)
