"""GPU edge cases: empty and ragged batches, degenerate matrices, non-finite
entries, extreme scales, misaligned pointers, output guard bands, the
statistics struct, and capture of the whole forward + backward step in a
CUDA graph."""
import ctypes

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


def test_empty_batch(eig3):
    for prec, dt in (("f64", torch.float64), ("f32c", torch.float32)):
        A = torch.empty(0, 9, dtype=dt, device=dev())
        assert eig3.eigvals(A, precision=prec).shape == (0, 3)
        assert eig3.invariants(A, precision=prec).shape == (0, 4)
        g = torch.empty(0, 3, dtype=dt, device=dev())
        assert eig3.eigvals_backward(A, g, precision=prec).shape == (0, 9)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 256, 257, 1025, 38913])
def test_ragged_sizes(eig3, n):
    bt = W.workload2(n=n, device="cpu", seed=1500 + n)
    lam = U.to_np(eig3.eigvals(bt.A.to(dev())))
    err, tol, bad = U.check_eig_f64(lam, bt.A.numpy(), bt.kappa.numpy(), GEN)
    assert not bad.any()
    S = W.workload3(n=n, device="cpu", seed=1600 + n)
    lc = U.to_np(eig3.eigvals(S.A.to(dev()), precision="f32c"))
    err, tol, _ = U.check_eig_f32c(lc, S.A.double().numpy(), 1.0, SYM)
    assert np.all(err <= tol)


def test_scaled_identity_and_zero(eig3):
    alphas = [0.0, 1.0, -0.1, 7.0, 3.7e-200, 1e300, -2.5e-30]
    A = np.zeros((len(alphas), 9))
    for i, a in enumerate(alphas):
        A[i, [0, 4, 8]] = a
    inv = U.to_np(eig3.invariants(torch.as_tensor(A, device=dev())))
    assert np.all(inv[:, 1:] == 0.0)          # J2 = J3 = Delta = 0 exactly (Section J2 remark)
    lam = U.to_np(eig3.eigvals(torch.as_tensor(A, device=dev())))
    al = np.array(alphas)[:, None]
    assert np.all(np.abs(lam - al) <= 2 * np.spacing(np.abs(al)))
    A32 = torch.as_tensor(A[[0, 1, 2, 3, 6]], device=dev()).float()
    for prec in ("f64", "f32c"):
        lam32 = U.to_np(eig3.eigvals(A32, precision=prec))
        a32 = A32[:, 0:1].double().cpu().numpy()
        assert np.all(np.abs(lam32 - a32) <= 2 * np.spacing(np.abs(a32).astype(np.float32)))
        inv32 = U.to_np(eig3.invariants(A32, precision=prec))
        assert np.all(inv32[:, 1:] == 0.0)


def test_diagonal_special_cases(eig3):
    A = np.stack([np.diag([1.0, 2.0, 3.0]).reshape(9), np.diag([3.0, -1.0, 2.0]).reshape(9),
                  np.diag([1.0, 1.0, 1.0 + 1e-8]).reshape(9)])
    inv = U.to_np(eig3.invariants(torch.as_tensor(A, device=dev())))
    assert inv[0, 2] == 0.0 and inv[0, 3] == 4.0     # J3 = 0, Delta = (d0 d1 d2)^2
    assert inv[2, 3] == 0.0                          # exact double eigenvalue
    lam = U.to_np(eig3.eigvals(torch.as_tensor(A, device=dev())))
    ref = np.sort(np.diagonal(A.reshape(-1, 3, 3), axis1=1, axis2=2), axis=1)
    assert np.all(np.abs(lam - ref) <= 8 * U.U64 * 3)


def test_nonfinite_inputs_give_nan_not_trap(eig3):
    A = np.tile(np.eye(3).reshape(1, 9), (6, 1))
    A[0, 1] = np.nan
    A[1, 4] = np.inf
    A[2, 0] = -np.inf
    st = eig3.Stats(dev())
    lam = U.to_np(eig3.eigvals(torch.as_tensor(A, device=dev()), stats=st))
    assert np.all(~np.isfinite(lam[:3]).all(axis=1))
    assert np.all(np.abs(lam[3:] - 1.0) <= 4 * U.U64)
    s = st.read()
    assert s["n_nonfinite"] == 3
    A32 = torch.as_tensor(A, device=dev()).float()
    lam32 = U.to_np(eig3.eigvals(A32, precision="f32c"))
    assert np.all(~np.isfinite(lam32[:3]).all(axis=1))
    torch.cuda.synchronize()   # the context is still healthy
    assert bool(torch.isfinite(eig3.eigvals(torch.eye(3, device=dev(), dtype=torch.float64)
                                            .reshape(1, 9))).all())


@pytest.mark.parametrize("expo", [-30, -12, 12, 30])
def test_extreme_scales_f32c(eig3, expo):
    S = W.workload3(n=20_000, device="cpu", seed=1700 + expo)
    A = (S.A.double() * 10.0 ** (expo - np.log10(np.abs(S.A.double().numpy()).max()))).float()
    lam = U.to_np(eig3.eigvals(A.to(dev()), precision="f32c"))
    err, tol, ulps = U.check_eig_f32c(lam, A.double().numpy(), 1.0, SYM)
    print(f"[edge] f32c scale 1e{expo}: max ulp {ulps.max():.2f}")
    assert np.all(err <= tol)


@pytest.mark.parametrize("expo", [-30, 30])
def test_large_and_small_scales_f64(eig3, expo):
    """Within the oracle's exponent range (its Delta, of degree 6, neither
    under- nor overflows) the results match it."""
    bt = W.workload2(n=20_000, device="cpu", seed=1800)
    A = bt.A.numpy() * 10.0 ** expo
    lam = U.to_np(eig3.eigvals(torch.as_tensor(A, device=dev())))
    err, tol, bad = U.check_eig_f64(lam, A, bt.kappa.numpy(), GEN)
    assert not bad.any()


@pytest.mark.parametrize("k", [-900, -170, -60, 60, 170, 900])
def test_power_of_two_scale_equivariance_f64(eig3, k):
    """Beyond the oracle's range (Delta of a literal evaluation under- or
    overflows once ||dev A|| leaves about [1e-51, 1e51]) the library scales the
    deviatoric data by powers of two, which makes it exactly equivariant:
    lambda(2^k A) = 2^k lambda(A) bit for bit, and likewise the gradient is
    scale invariant.  The unit-scale results are pinned to the oracle above."""
    bt = W.workload2(n=30_000, device="cpu", seed=1801)
    A = torch.as_tensor(bt.A.numpy(), device=dev())
    A = A[(A.abs().amax(dim=1) > 2.0 ** -60)]      # keep 2^k A free of subnormals
    lam0, aux0 = eig3.eigvals(A, return_aux=True)
    lamk, auxk = eig3.eigvals(A * 2.0 ** k, return_aux=True)
    assert torch.equal(lamk, lam0 * 2.0 ** k)
    g = torch.randn(A.shape[0], 3, dtype=torch.float64, device=dev())
    G0 = eig3.eigvals_backward(A, g, aux=aux0)
    Gk = eig3.eigvals_backward(A * 2.0 ** k, g, aux=auxk)
    assert torch.equal(G0, Gk)
    for lay, X in (("sym6", W.workload1("cpu")["sym6"].A),):
        X = torch.as_tensor(X.numpy(), device=dev())
        assert torch.equal(eig3.eigvals(X * 2.0 ** k), eig3.eigvals(X) * 2.0 ** k)


def test_r_is_a_faithful_square_root(eig3):
    """r = sqrt(3 J2+) (the first adjoint input) comes from a binary32 seed and a
    series correction, not from the correctly rounded sqrt: it must lie within
    one unit in the last place of the exact square root of 3 times the
    kernel's own J2 (evaluated in extended precision), over a wide range of
    exponents."""
    bt = W.workload2(n=50_000, device="cpu", seed=1810)
    g = torch.Generator().manual_seed(1811)
    scale = 2.0 ** torch.randint(-120, 121, (bt.n, 1), generator=g).double()
    A = torch.as_tensor(bt.A.numpy(), device=dev()) * scale.to(dev())
    J2 = U.to_np(eig3.invariants(A))[:, 1]
    _, aux = eig3.eigvals(A, return_aux=True)
    r = U.to_np(aux)[:, 0]
    pos = J2 > 0
    assert pos.mean() > 0.9
    ref = np.sqrt(np.longdouble(3.0) * J2[pos].astype(np.longdouble))
    d = np.abs(r[pos].astype(np.longdouble) - ref)
    ulp = np.spacing(r[pos]).astype(np.longdouble)
    print(f"[edge] r: {np.mean(r[pos] == ref.astype(np.float64)):.3f} correctly rounded, "
          f"max error {float(np.max(d / ulp)):.3f} ulp")
    assert np.all(d < ulp)
    assert np.all(r[~pos] == 0.0)


@pytest.mark.parametrize("k", [-100, -40, 40, 100])
def test_power_of_two_scale_equivariance_f32c(eig3, k):
    S = W.workload3(n=30_000, device="cpu", seed=1802).A
    S = torch.as_tensor(S.numpy(), device=dev())
    big = S.abs().amax(dim=1)
    keep = (big * 2.0 ** k < 2.0 ** 120) & (S.abs().amin(dim=1) * 2.0 ** k > 2.0 ** -120) & \
        (S.abs().amin(dim=1) > 0)
    S = S[keep]
    lam0, aux0 = eig3.eigvals(S, precision="f32c", return_aux=True)
    lamk = eig3.eigvals(S * 2.0 ** k, precision="f32c")
    # exact equivariance needs every result (and r) to stay out of the binary32
    # subnormal range at both scales
    tiny = 2.0 ** -125
    ok = (lam0.abs().amin(dim=1) * min(1.0, 2.0 ** k) > tiny) & \
        (aux0[:, 0] * min(1.0, 2.0 ** k) > tiny)
    assert int(ok.sum()) > 10_000
    assert torch.equal(lamk[ok], lam0[ok] * 2.0 ** k)


def test_misaligned_pointer_rejected(eig3):
    """A device pointer off its element alignment is refused on the host
    (EIG3_ERR_ALIGN) before anything is launched."""
    buf = torch.zeros(9 * 4 + 2, dtype=torch.float32, device=dev())
    out = torch.zeros(16, dtype=torch.float64, device=dev())
    lib = eig3.load()
    base = buf.data_ptr()
    st = lib.eig3_eigvals(ctypes.c_void_p(base + 4), 0, 0, 0, 4, ctypes.c_void_p(out.data_ptr()),
                          None, None, None)
    assert st == 4
    st = lib.eig3_eigvals(ctypes.c_void_p(base + 2), 0, 1, 1, 4, ctypes.c_void_p(out.data_ptr()),
                          None, None, None)
    assert st == 4
    torch.cuda.synchronize()


def test_guard_bands_untouched(eig3):
    n = 1001
    bt = W.workload2(n=n, device="cpu", seed=1900)
    A = bt.A.to(dev())
    canary = -12345.678
    for prec, dt in (("f64", torch.float64), ("f32c", torch.float32)):
        X = A.to(dt)
        lam_buf = torch.full((n + 64, 3), canary, dtype=dt, device=dev())
        aux_buf = torch.full((n + 64, 4), canary, dtype=dt, device=dev())
        eig3.eigvals(X, precision=prec, return_aux=True, out=lam_buf[32:32 + n],
                     aux_out=aux_buf[32:32 + n])
        g_buf = torch.full((n + 64, 9), canary, dtype=dt, device=dev())
        eig3.eigvals_backward(X, torch.ones(n, 3, dtype=dt, device=dev()),
                              aux=aux_buf[32:32 + n], precision=prec, out=g_buf[32:32 + n])
        for b in (lam_buf, aux_buf, g_buf):
            assert bool((b[:32] == canary).all()) and bool((b[32 + n:] == canary).all())
            assert bool((b[32:32 + n] != canary).any())


def test_stats_struct(eig3):
    bt = W.workload2(n=200_000, device="cpu", seed=2000)
    A = bt.A.to(dev())
    st = eig3.Stats(dev())
    lam = eig3.eigvals(A, stats=st)
    inv = eig3.invariants(A)
    s = st.read()
    invn = U.to_np(inv)
    assert s["n_delta_clamped"] == int((invn[:, 3] < 0).sum())
    assert s["n_j2_clamped"] == int((invn[:, 1] < 0).sum())
    assert s["n_nonfinite"] == 0
    assert s["max_abs_lambda"] == float(lam.abs().max())
    J2 = np.maximum(invn[:, 1], 0)
    ratio = np.maximum(invn[:, 3], 0)[J2 > 0] / J2[J2 > 0] ** 3
    # binary32 diagnostic from the angle: relative accuracy of a few binary32 ulps
    assert abs(s["min_disc_ratio"] - ratio.min()) <= 1e-5 * ratio.min() + 1e-30
    assert s["n_delta_clamped"] > 0          # the near-double cases of this workload


def test_cuda_graph_mixed_step(eig3):
    """A small copy of the mixed workload: forward + backward on a symmetric
    FP32 (compensated) half and a general FP64 half, captured once and
    replayed; replays reproduce the eager results bit for bit."""
    w5 = W.workload5(n=1 << 16, device=dev())
    S, G = w5["sym6"], w5["general9"]
    lamS = torch.empty(S.n, 3, dtype=torch.float32, device=dev())
    auxS = torch.empty(S.n, 4, dtype=torch.float32, device=dev())
    gS = torch.empty_like(S.A)
    lamG = torch.empty(G.n, 3, dtype=torch.float64, device=dev())
    auxG = torch.empty(G.n, 4, dtype=torch.float64, device=dev())
    gG = torch.empty_like(G.A)
    st = eig3.Stats(dev())

    def step():
        eig3.eigvals(S.A, precision="f32c", return_aux=True, out=lamS, aux_out=auxS, stats=st)
        eig3.eigvals_backward(S.A, S.extra["w"], aux=auxS, precision="f32c", out=gS)
        eig3.eigvals(G.A, precision="f64", return_aux=True, out=lamG, aux_out=auxG, stats=st)
        eig3.eigvals_backward(G.A, G.extra["w"], aux=auxG, precision="f64", out=gG)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            step()
    torch.cuda.current_stream().wait_stream(s)
    eager = [t.clone() for t in (lamS, gS, lamG, gG)]
    for t in (lamS, gS, lamG, gG):
        t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(2):
            step()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, (lamS, gS, lamG, gG)):
        assert torch.equal(a, b)
    # the graph's results are the library's results: check them against the oracle
    err, tol, bad = U.check_eig_f64(U.to_np(lamG), U.to_np(G.A), U.to_np(G.kappa), GEN)
    assert not bad.any()
    err, tol, _ = U.check_eig_f32c(U.to_np(lamS), U.to_np(S.A), 1.0, SYM)
    assert np.all(err <= tol)


def test_zero_copy_pinned_host_buffers(eig3):
    """Kernels reading and writing page-locked host memory directly give the
    same bits as on device-resident buffers."""
    bt = W.workload2(n=70_001, device="cpu", seed=2100)
    hA = bt.A.pin_memory()
    dA = bt.A.to(dev())
    lam_h, aux_h = eig3.eigvals(hA, return_aux=True, device=dev())
    torch.cuda.synchronize()
    assert not lam_h.is_cuda and lam_h.is_pinned()
    lam_d, aux_d = eig3.eigvals(dA, return_aux=True)
    assert torch.equal(lam_h, lam_d.cpu())
    hw = torch.randn(bt.n, 3, dtype=torch.float64).pin_memory()
    g_h = eig3.eigvals_backward(hA, hw, aux=aux_h, device=dev())
    torch.cuda.synchronize()
    g_d = eig3.eigvals_backward(dA, hw.to(dev()), aux=aux_d)
    assert torch.equal(g_h, g_d.cpu())
    S = W.workload3(n=50_001, device="cpu", seed=2101).A
    l_h = eig3.eigvals(S.pin_memory(), precision="f32c", device=dev())
    torch.cuda.synchronize()
    assert torch.equal(l_h, eig3.eigvals(S.to(dev()), precision="f32c").cpu())
    # the fused entry point on host pointers, both precisions
    lv_h, gv_h = eig3.eigvals_vjp(hA, hw, device=dev())
    torch.cuda.synchronize()
    assert not gv_h.is_cuda and gv_h.is_pinned()
    lv_d, gv_d = eig3.eigvals_vjp(dA, hw.to(dev()))
    assert torch.equal(lv_h, lv_d.cpu()) and torch.equal(gv_h, gv_d.cpu())
    wS = torch.randn(S.shape[0], 3, dtype=torch.float32).pin_memory()
    ls_h, gs_h = eig3.eigvals_vjp(S.pin_memory(), wS, precision="f32c", device=dev())
    torch.cuda.synchronize()
    ls_d, gs_d = eig3.eigvals_vjp(S.to(dev()), wS.to(dev()), precision="f32c")
    assert torch.equal(ls_h, ls_d.cpu()) and torch.equal(gs_h, gs_d.cpu())
    with pytest.raises(ValueError):
        eig3.eigvals(bt.A)          # pageable host memory is refused


def test_huge_page_pinned_buffers(eig3):
    """host.pinned_empty / pinned_copy (registered huge-page host memory) serve
    the zero-copy path and HostPipeline with the device results bit for bit,
    and dropping them releases their registration (allocating many in turn
    keeps working)."""
    from paper_2511_00292_gb300 import host
    from paper_2511_00292_gb300.host import HostPipeline
    bt = W.workload4(n=30_011, device="cpu", seed=2204)
    hA, hw = host.pinned_copy(bt.A), host.pinned_copy(bt.extra["w"])
    assert hA.is_pinned() and hw.is_pinned() and torch.equal(hA, bt.A)
    dA = bt.A.to(dev())
    l_d, a_d = eig3.eigvals(dA, return_aux=True)
    g_d = eig3.eigvals_backward(dA, bt.extra["w"].to(dev()), aux=a_d)
    lam_h = eig3.eigvals(hA, device=dev())
    torch.cuda.synchronize()
    assert torch.equal(lam_h, l_d.cpu())
    lam = host.pinned_empty((bt.n, 3), torch.float64)
    grad = host.pinned_empty(hA.shape, torch.float64)
    HostPipeline(dev(), chunk=4096, depth=3).forward_backward(hA, hw, lam, grad)
    torch.cuda.synchronize()
    # the pipeline runs the fused kernel (eig3_eigvals_vjp)
    lv, gv = eig3.eigvals_vjp(dA, bt.extra["w"].to(dev()))
    assert torch.equal(lam, l_d.cpu()) and torch.equal(lam, lv.cpu())
    assert torch.equal(grad, gv.cpu())
    for _ in range(8):
        x = host.pinned_empty((1 << 24,), torch.float64)   # 128 MiB each
        x[::4096].fill_(1.0)
        y = torch.empty(1 << 24, dtype=torch.float64, device=dev())
        y.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        del x, y
    assert host.pinned_empty((0, 9)).shape == (0, 9)


@pytest.mark.parametrize("depth", [2, 3])
def test_host_pipeline_matches_device(eig3, depth):
    """Chunked host-to-device streaming gives the device results (of the fused
    kernel it runs) bit for bit, including a ragged last chunk and more chunks
    than device slots."""
    from paper_2511_00292_gb300.host import HostPipeline
    bt = W.workload4(n=10_007, device="cpu", seed=2200)
    hA, hw = bt.A.pin_memory(), bt.extra["w"].pin_memory()
    lam = torch.empty(bt.n, 3, dtype=torch.float64).pin_memory()
    grad = torch.empty_like(hA).pin_memory()
    pipe = HostPipeline(dev(), chunk=1024, depth=depth)
    pipe.forward_backward(hA, hw, lam, grad)
    torch.cuda.synchronize()
    dA = bt.A.to(dev())
    l_d, g_d = eig3.eigvals_vjp(dA, bt.extra["w"].to(dev()))   # the kernel the pipeline runs
    assert torch.equal(lam, l_d.cpu()) and torch.equal(grad, g_d.cpu())
    S = W.workload3(n=5_003, device="cpu", seed=2201).A
    wS = torch.randn(S.shape[0], 3, dtype=torch.float32)
    lS = torch.empty(S.shape[0], 3, dtype=torch.float32).pin_memory()
    gS = torch.empty_like(S).pin_memory()
    pipe.forward_backward(S.pin_memory(), wS.pin_memory(), lS, gS, precision="f32c")
    torch.cuda.synchronize()
    l2, g2 = eig3.eigvals_vjp(S.to(dev()), wS.to(dev()), precision="f32c")
    assert torch.equal(lS, l2.cpu()) and torch.equal(gS, g2.cpu())


def test_host_pipeline_graph_replay(eig3):
    """The captured pipeline (one graph launch per step) gives the results of
    the direct run bit for bit, replay after replay, with both jobs in it."""
    from paper_2511_00292_gb300.host import HostPipeline
    bt = W.workload4(n=9_001, device="cpu", seed=2202)
    S = W.workload3(n=7_003, device="cpu", seed=2203).A
    wS = torch.randn(S.shape[0], 3, dtype=torch.float32)
    hA, hw, hS, hwS = (t.pin_memory() for t in (bt.A, bt.extra["w"], S, wS))
    outs = [torch.empty(bt.n, 3, dtype=torch.float64).pin_memory(),
            torch.empty_like(hA).pin_memory(),
            torch.empty(S.shape[0], 3, dtype=torch.float32).pin_memory(),
            torch.empty_like(hS).pin_memory()]
    jobs = [(hS, hwS, outs[2], outs[3], None, "f32c"), (hA, hw, outs[0], outs[1], None, "f64")]
    pipe = HostPipeline(dev(), chunk=2048, depth=3)
    pipe.run(jobs)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    g = pipe.capture(jobs)
    for o in outs:
        o.zero_()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert all(torch.equal(o, r) for o, r in zip(outs, ref))



def test_supplied_outputs_are_checked_before_any_launch(eig3):
    """The kernels write through raw pointers, so the binding refuses outputs of
    the wrong size, dtype or memory kind instead of letting a kernel write past
    them."""
    A = W.workload2(n=1000, device="cpu", seed=2204).A.to(dev())
    S = W.workload3(n=1000, device="cpu", seed=2205).A.to(dev())
    small = torch.empty(999, 3, dtype=torch.float64, device=dev())
    with pytest.raises(ValueError):
        eig3.eigvals(A, out=small)
    with pytest.raises(ValueError):
        eig3.eigvals(A, out=torch.empty(1000, 3, dtype=torch.float32, device=dev()))
    with pytest.raises(ValueError):
        eig3.eigvals(A, out=torch.empty(1000, 3, dtype=torch.float64))          # pageable host
    with pytest.raises(ValueError):
        eig3.eigvals(A, return_aux=True, aux_out=torch.empty(1000, 3, dtype=torch.float64,
                                                             device=dev()))
    with pytest.raises(ValueError):
        eig3.eigvals_backward(A, torch.zeros(1000, 3, dtype=torch.float64, device=dev()),
                              out=torch.empty(1000, 6, dtype=torch.float64, device=dev()))
    with pytest.raises(ValueError):
        eig3.eigprojectors(A, out=torch.empty(1000, 26, dtype=torch.float64, device=dev()))
    with pytest.raises(ValueError):
        eig3.mohr_coulomb(S, grad=True, grad_out=torch.empty(1000, 9, dtype=torch.float32,
                                                             device=dev()))
    with pytest.raises(ValueError):
        eig3.eigvals_variant(A, "naive", inv_out=torch.empty(1000, 4, dtype=torch.float32,
                                                             device=dev()))
    wide = torch.empty(1000, 6, dtype=torch.float64, device=dev())[:, :3]  # not contiguous
    with pytest.raises(ValueError):
        eig3.eigvals(A, out=wide)
    # correct outputs are used as given
    lam = torch.empty(1000, 3, dtype=torch.float64, device=dev())
    assert eig3.eigvals(A, out=lam).data_ptr() == lam.data_ptr()
