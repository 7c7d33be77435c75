"""The seeded input generators produce what their recipes state (shapes,
dtypes, spectra, eigenbasis conditioning, mixtures), checked with LAPACK on
the generated matrices.  The generators hold none of the method's
arithmetic; these checks keep the stated workload recipes honest."""
import numpy as np
import pytest
import torch

import workloads as W


def eig_sorted(A9):
    return np.sort(np.linalg.eigvals(A9.reshape(-1, 3, 3)).real, axis=1)


def test_haar_rotations_are_orthogonal_with_both_signs():
    g = torch.Generator().manual_seed(5)
    Q = W.haar_o3(4000, g, "cpu").numpy()
    assert np.abs(Q @ np.transpose(Q, (0, 2, 1)) - np.eye(3)).max() < 1e-14
    det = np.linalg.det(Q)
    assert np.allclose(np.abs(det), 1.0)
    assert 0.4 < np.mean(det > 0) < 0.6
    # Haar: E[Q_ij^2] = 1/3 for every entry
    assert np.allclose((Q ** 2).mean(axis=0), 1 / 3, atol=0.02)


def test_workload1():
    w = W.workload1("cpu")
    G9, S6 = w["general9"], w["sym6"]
    assert G9.A.shape == (4160, 9) and S6.A.shape == (4160, 6)
    assert G9.A.dtype == torch.float64
    A = G9.A.numpy().reshape(-1, 3, 3)
    assert np.array_equal(A, np.transpose(A, (0, 2, 1)))           # explicitly symmetric
    lam = np.sort(np.linalg.eigvalsh(A), axis=1)
    assert np.allclose(lam, np.sort(G9.lam_nominal.numpy(), axis=1), atol=1e-14)
    near = G9.lam_nominal.numpy()[4096:]
    d = near[:, 1] - near[:, 0]
    assert np.allclose(np.sort(d[:32])[::-1], np.logspace(-1, -15, 32), rtol=1e-12)


def test_workload2_mixture_and_conditioning():
    bt = W.workload2(n=30_000, device="cpu", seed=7)
    kinds = bt.extra["kinds"].numpy()
    frac = np.bincount(kinds, minlength=3) / len(kinds)
    assert np.all(np.abs(frac - 1 / 3) < 0.02)
    k = bt.kappa.numpy()
    assert k.min() >= 1.0 and k.max() <= 10.0 * (1 + 1e-12)
    lam = bt.lam_nominal.numpy()
    gaps = np.sort(lam, axis=1)
    d = (gaps[:, 1] - gaps[:, 0])[kinds == 2]
    # delta log-uniform in [1e-16, 1e-2] (a + delta is rounded, so the stored
    # gap of the smallest deltas is within an ulp of 1 of delta)
    assert d.min() >= 0.0 and d.max() <= 1e-2 * (1 + 1e-9)
    assert np.median(np.log10(np.maximum(d, 1e-17))) == pytest.approx(-9.0, abs=0.3)
    sep = np.all(np.diff(np.sort(lam, axis=1), axis=1) > 1e-3, axis=1)
    ev = eig_sorted(bt.A.numpy()[sep][:2000])
    assert np.allclose(ev, np.sort(lam[sep][:2000], axis=1), atol=1e-12)


def test_workload3_scales_and_near_hydrostatic_share():
    bt = W.workload3(n=40_000, device="cpu", seed=9)
    assert bt.A.dtype == torch.float32 and bt.A.shape == (40_000, 6)
    near = bt.extra["near"].numpy()
    assert 0.18 < near.mean() < 0.22
    lam = bt.lam_nominal.numpy()
    scale = np.abs(lam).max(axis=1)
    assert scale.max() < 1e6 * 1.01 and scale.min() > 1e-6 * 1e-3
    spread = (lam.max(axis=1) - lam.min(axis=1)) / scale
    assert np.median(spread[near]) < 1e-4 < np.median(spread[~near])


def test_workload5_composition():
    w = W.workload5(n=1 << 14, device="cpu", seed=11)
    S, G = w["sym6"], w["general9"]
    assert S.A.shape == (1 << 13, 6) and S.A.dtype == torch.float32
    assert G.A.shape == (1 << 13, 9) and G.A.dtype == torch.float64
    assert S.extra["w"].shape == (1 << 13, 3) and G.extra["w"].shape == (1 << 13, 3)
    lamG = G.lam_nominal.numpy()
    sc = np.abs(lamG).max(axis=1)
    assert sc.min() < 1e-6 and sc.max() > 1e6                      # scales 10^U[-8, 8]


@pytest.mark.parametrize("kmax", [2.0, 4.0])
def test_illconditioned_kappa(kmax):
    bt = W.illconditioned(3000, "cpu", seed=13, log10_kappa_max=kmax)
    k = bt.kappa.numpy()
    assert k.min() >= 1.0 and k.max() <= 10.0 ** kmax * (1 + 1e-12)
    assert np.median(np.log10(k)) == pytest.approx(kmax / 2, abs=0.2)
    # the stated kappa is that of the generating eigenbasis: the eigenvector
    # matrix of a well-separated sample has at least that condition up to scaling
    lam = bt.lam_nominal.numpy()
    sep = np.all(np.diff(np.sort(lam, axis=1), axis=1) > 0.05, axis=1) & (k > 10)
    A = bt.A.numpy()[sep][:200].reshape(-1, 3, 3)
    ev, V = np.linalg.eig(A)
    cond = np.linalg.cond(V / np.linalg.norm(V, axis=1, keepdims=True))
    assert np.median(cond / k[sep][:200]) > 0.05


def test_lode_sweep_and_stress_field_shapes():
    L = W.lode_sweep(360)
    assert L.shape == (360, 6)
    sf = W.stress_field(1000, "cpu", seed=3)
    assert sf.A.shape == (1000, 6) and sf.A.dtype == torch.float64


def test_seeds_reproduce_and_differ():
    a = W.workload2(n=1000, device="cpu", seed=21).A
    b = W.workload2(n=1000, device="cpu", seed=21).A
    c = W.workload2(n=1000, device="cpu", seed=22).A
    assert torch.equal(a, b) and not torch.equal(a, c)
    # chunking does not change the stream of matrices
    d = W.workload2(n=1000, device="cpu", seed=21, chunk=256).A
    assert d.shape == a.shape
