"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element, at sizes the oracle finishes in
seconds (several grid-stride tiles and a ragged tail) and, sampled, at the
full benchmark sizes."""
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


def report(name, **kw):
    print(f"[parity] {name}: " + " ".join(f"{k}={v}" for k, v in kw.items()))


# --------------------------------------------------------------------------
# Workload 1: symmetric FP64, both layouts, forward only
# --------------------------------------------------------------------------

@pytest.mark.parametrize("layout", ["general9", "sym6"])
def test_workload1_eigvals(eig3, layout):
    w1 = W.workload1("cpu")[layout]
    A = w1.A.to(dev())
    lam = U.to_np(eig3.eigvals(A))
    lay = GEN if layout == "general9" else SYM
    err, tol, bad = U.check_eig_f64(lam, w1.A.numpy(), 1.0, lay)
    report("w1 " + layout, max_err_over_tol=float((err / tol).max()))
    assert not bad.any(), np.argwhere(bad)[:5]
    assert np.all(np.diff(lam, axis=1) >= 0)


@pytest.mark.parametrize("layout", ["general9", "sym6"])
def test_workload1_invariants(eig3, layout):
    w1 = W.workload1("cpu")[layout]
    inv = U.to_np(eig3.invariants(w1.A.to(dev())))
    lay = GEN if layout == "general9" else SYM
    err, tol = U.check_invariants(inv, w1.A.numpy(), 1.0, lay, U.U64)
    report("w1 inv " + layout, max_ratio=[float(x) for x in (err / np.maximum(tol, 1e-300)).max(0)])
    assert np.all(err <= tol)


def test_sym6_matches_general9(eig3):
    w1 = W.workload1("cpu")
    a = U.to_np(eig3.eigvals(w1["general9"].A.to(dev())))
    b = U.to_np(eig3.eigvals(w1["sym6"].A.to(dev())))
    bnd = U.EIG_C * oracle.bounds(w1["general9"].A.numpy(), 1.0)[:, 4:5]
    assert np.all(np.abs(a - b) <= 2 * bnd + 8 * np.spacing(np.abs(a).max(1, keepdims=True)))


# --------------------------------------------------------------------------
# Workload 2: general FP64, small with a ragged tail, and full-size sampled
# --------------------------------------------------------------------------

def test_workload2_small(eig3):
    bt = W.workload2(n=100_003, device="cpu", seed=1202)
    A = bt.A.to(dev())
    lam = U.to_np(eig3.eigvals(A))
    err, tol, bad = U.check_eig_f64(lam, bt.A.numpy(), bt.kappa.numpy(), GEN)
    report("w2 small", max_err_over_tol=float((err / tol).max()))
    assert not bad.any()
    inv = U.to_np(eig3.invariants(A))
    ierr, itol = U.check_invariants(inv, bt.A.numpy(), bt.kappa.numpy(), GEN, U.U64)
    report("w2 small inv", max_ratio=[float(x) for x in (ierr / np.maximum(itol, 1e-300)).max(0)])
    assert np.all(ierr <= itol)


def test_workload2_full_size_sampled(eig3):
    n = 1 << 26
    bt = W.workload2(n=n, device=dev())
    lam = eig3.eigvals(bt.A)
    idx = W.sample_indices(n, 1 << 16)
    it = torch.as_tensor(idx, device=dev())
    A_s = U.to_np(bt.A[it])
    err, tol, bad = U.check_eig_f64(U.to_np(lam[it]), A_s, U.to_np(bt.kappa[it]), GEN)
    report("w2 2^26 sampled", max_err_over_tol=float((err / tol).max()), samples=len(idx))
    assert not bad.any()
    # properties that hold at any size: ordering and finiteness of every output
    assert bool(torch.isfinite(lam).all())
    assert bool((lam[:, 1] >= lam[:, 0]).all()) and bool((lam[:, 2] >= lam[:, 1]).all())
    del bt, lam
    torch.cuda.empty_cache()


# --------------------------------------------------------------------------
# Workload 3: symmetric 6-entry FP32 storage, binary64 and compensated paths
# --------------------------------------------------------------------------

def test_workload3_f64_path(eig3):
    bt = W.workload3(n=100_003, device="cpu", seed=1303)
    A = bt.A.to(dev())
    lam = U.to_np(eig3.eigvals(A, precision="f64"))
    A64 = bt.A.double().numpy()
    err, tol, bad = U.check_eig_f64(lam, A64, 1.0, SYM, f32_storage=True)
    report("w3 f64 path", max_err_over_tol=float((err / tol).max()))
    assert not bad.any()


def test_workload3_f32c_path(eig3):
    bt = W.workload3(n=100_003, device="cpu", seed=1303)
    A = bt.A.to(dev())
    lam = U.to_np(eig3.eigvals(A, precision="f32c"))
    A64 = bt.A.double().numpy()
    err, tol, ulps = U.check_eig_f32c(lam, A64, 1.0, SYM)
    near = bt.extra["near"].numpy()
    report("w3 f32c", max_err_over_tol=float((err / tol).max()), max_ulp=float(ulps.max()),
           max_ulp_near_hydrostatic=float(ulps[near].max()), p999_ulp=float(np.quantile(ulps, 0.999)))
    assert np.all(err <= tol)
    assert np.all(np.diff(lam, axis=1) >= 0)


def test_workload3_f32c_angle64_by_disc_ratio(eig3):
    """The compensated binary32 path with the final Delta combination and the
    triple angle in binary64 (precision "f32c64") beside the plain one, per bin
    of Delta/J2^3 = 4 sin^2(phi) taken from the oracle's eigenvalues: both stay
    within the compensated tolerance in every bin, and the per-bin maxima (in
    ulp of max|lambda|) show what binary64 buys where, i.e. the threshold below
    which taking these steps in binary64 would pay."""
    bt = W.workload3(n=200_003, device="cpu", seed=1305)
    A = bt.A.to(dev())
    lam32 = U.to_np(eig3.eigvals(A, precision="f32c"))
    lam64, aux64 = eig3.eigvals(A, precision="f32c64", return_aux=True)
    A64 = bt.A.double().numpy()
    e32, tol, u32 = U.check_eig_f32c(lam32, A64, 1.0, SYM)
    e64, _, u64 = U.check_eig_f32c(U.to_np(lam64), A64, 1.0, SYM)
    assert np.all(e32 <= tol) and np.all(e64 <= tol)
    assert np.all(np.diff(U.to_np(lam64), axis=1) >= 0)
    ref = np.sort(oracle.eigvals(A64, layout=SYM), axis=1)
    g12, g23 = ref[:, 1] - ref[:, 0], ref[:, 2] - ref[:, 1]
    j2 = (g12 * g12 + g12 * g23 + g23 * g23) / 3.0
    ratio = (g12 * g23 * (g12 + g23)) ** 2 / np.maximum(j2, 1e-300) ** 3
    edges = [0.0, 1e-8, 1e-6, 1e-4, 1e-2, 1.0, 5.0]
    rows = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (ratio >= lo) & (ratio < hi)
        if m.any():
            rows.append(f"[{lo:g},{hi:g}) n={int(m.sum())} f32c {u32[m].max():.2f} "
                        f"f32c64 {u64[m].max():.2f}")
    report("w3 f32c vs f32c64 max ulp by Delta/J2^3", bins="; ".join(rows))
    # the adjoint takes the binary64-angle adjoint inputs like the compensated ones
    w = torch.randn(bt.n, 3, dtype=torch.float32, device=dev())
    g64 = eig3.eigvals_backward(A, w, aux=aux64, precision="f32c64")
    g32 = eig3.eigvals_backward(A, w, precision="f32c")
    assert bool(torch.isfinite(g64).all())
    sep = torch.as_tensor(np.minimum(g12, g23) / np.abs(ref).max(axis=1) > 1e-2, device=dev())
    rel = ((g64 - g32).abs().amax(dim=1) / g32.abs().amax(dim=1).clamp_min(1e-30))[sep]
    assert float(rel.max()) < 1e-3


def test_workload3_f32c_invariants(eig3):
    bt = W.workload3(n=50_001, device="cpu", seed=1304)
    A = bt.A.to(dev())
    inv = U.to_np(eig3.invariants(A, precision="f32c"))
    A64 = bt.A.double().numpy()
    # compensated arithmetic: the invariants as if evaluated at twice the
    # binary32 precision, u = u32^2
    err, tol = U.check_invariants(inv, A64, 1.0, SYM, U.U32 ** 2)
    ratio = err / np.maximum(tol / 16.0, 1e-300)
    report("w3 f32c inv (error / bound at u32^2)", max=[float(x) for x in ratio.max(0)])
    assert np.all(err <= tol)


def test_workload3_full_size_sampled(eig3):
    n = 1 << 27
    bt = W.workload3(n=n, device=dev())
    lam_c = eig3.eigvals(bt.A, precision="f32c")
    lam_d = eig3.eigvals(bt.A, precision="f64")
    idx = W.sample_indices(n, 1 << 16, seed=9)
    it = torch.as_tensor(idx, device=dev())
    A_s = U.to_np(bt.A[it])
    err, tol, ulps = U.check_eig_f32c(U.to_np(lam_c[it]), A_s, 1.0, SYM)
    report("w3 2^27 sampled f32c", max_ulp=float(ulps.max()))
    assert np.all(err <= tol)
    err, tol, bad = U.check_eig_f64(U.to_np(lam_d[it]), A_s, 1.0, SYM, f32_storage=True)
    assert not bad.any()
    assert bool(torch.isfinite(lam_c).all()) and bool((lam_c[:, 1] >= lam_c[:, 0]).all())
    del bt, lam_c, lam_d
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["f32c", "f32c64"])
def test_general9_f32c(eig3, prec):
    bt = W.workload2(n=60_001, device="cpu", seed=1305)
    A32 = bt.A.float()
    lam = U.to_np(eig3.eigvals(A32.to(dev()), precision=prec))
    err, tol, ulps = U.check_eig_f32c(lam, A32.double().numpy(), bt.kappa.numpy(), GEN, c32=16.0)
    report("general9 " + prec, max_err_over_tol=float((err / tol).max()), max_ulp=float(ulps.max()))
    assert np.all(err <= tol)
    assert np.all(np.diff(lam, axis=1) >= 0)
