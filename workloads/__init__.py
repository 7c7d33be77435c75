"""Seeded synthetic inputs shaped like the paper's test matrices.

This module only builds input matrices with a prescribed spectrum and
eigenbasis; it holds none of the eigenvalue method's arithmetic.  Both the
oracle-side tests and the CUDA-side tests and benchmark draw their inputs
from here, so the two implementations always see the same bytes.

Constructions (all in binary64 before any rounding to the storage type):

* Paper test matrices (Section "Benchmarks"): fl(A) = fl(U D U^-1) with
  U in {U_symm, U1, U2(gamma)}, D1 = diag(1, 1, 1+delta) and
  D2 = diag(-1, 1, 1+delta), using numpy.linalg.inv and numpy.matmul as the
  paper describes.
* Haar-orthogonal Q: a uniformly random unit quaternion (a normalised
  4-vector of independent standard normals) gives a Haar rotation of SO(3)
  (Shoemake, "Uniform random rotations", Graphics Gems III, 1992); a random
  sign makes it Haar on O(3).
* General matrices with a controlled eigenbasis: V = Q1 diag(s) Q2 with
  s_i = exp(U[0, ln 10]), so kappa_2(V) = max(s)/min(s) <= 10, and
  A = V diag(lambda) V^-1 = Q1 diag(s) Q2 diag(lambda) Q2^T diag(1/s) Q1^T.
* Spectra: distinct U[-1,1]^3; double (a, a+delta, b); triple
  (a, a+delta, a+2 delta); delta log-uniform.

Workloads (seed 1000 + c for workload c):
  1  4096 symmetric A = Q diag(lambda) Q^T, lambda iid U[-1,1], plus 64
     near-repeated cases (1, 1+d, 2) and (1, 1+d, 1+2d), d log-spaced
     1e-1 .. 1e-15; FP64.
  2  general FP64 matrices, one third each distinct / double / triple,
     delta log-uniform in [1e-16, 1e-2].
  3  symmetric 6-entry FP32 "stress field": scale 10^U[-6,6]; 80% with
     lambda = s U[-1,1]^3, 20% near-hydrostatic lambda = s (p + delta xi)
     with delta log-uniform in [1e-12, 1e-3].
  4  as 2, plus loss weights w ~ N(0, 1), one per eigenvalue.
  5  mixed: half symmetric FP32 as 3 but scales 10^U[-8,8] and 30%
     triple-perturbed; half general FP64 as 2 with scales 10^U[-8,8],
     35% distinct / 35% double / 30% triple.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

LN10 = math.log(10.0)

# Symmetric storage order: (A00, A11, A22, A12, A02, A01).
SYM6_INDEX = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


# --------------------------------------------------------------------------
# Paper test matrices
# --------------------------------------------------------------------------

def paper_U(name: str, gamma: float = 1e-3) -> np.ndarray:
    """Transformation matrices U_symm, U1 and U2(gamma) of Section "Benchmarks"."""
    if name == "symm":
        r = 1.0 / math.sqrt(2.0)
        return np.array([[r, -0.5, 0.5], [r, 0.5, -0.5], [0.0, r, r]])
    if name == "u1":
        return np.array([[1.0, -1.0, 1.0], [1.0, 1.0, 1.0], [-1.0, -1.0, 1.0]])
    if name == "u2":
        return np.array([[1.0, 1.0, 1.0], [1.0, 0.0, 1.0], [2.0, 1.0, 2.0 + gamma]])
    raise ValueError(name)


def paper_D(path: str, delta: float) -> np.ndarray:
    """D1 = diag(1, 1, 1+delta) (towards a triple eigenvalue) and
    D2 = diag(-1, 1, 1+delta) (towards a double eigenvalue)."""
    if path == "d1":
        return np.diag([1.0, 1.0, 1.0 + delta])
    if path == "d2":
        return np.diag([-1.0, 1.0, 1.0 + delta])
    raise ValueError(path)


def paper_matrix(U: np.ndarray, D: np.ndarray) -> np.ndarray:
    """fl(U D U^-1) with numpy.linalg.inv and numpy.matmul, row-major 9 entries."""
    return np.matmul(np.matmul(U, D), np.linalg.inv(U)).reshape(9)


def paper_paths(deltas=None, gamma: float = 1e-3):
    """All (path, U) combinations of the paper's error figures.

    Returns a list of dicts with keys path, U, delta, A (9 entries), kappa.
    """
    if deltas is None:
        deltas = np.logspace(-1, -16, 31)
    out = []
    for path in ("d1", "d2"):
        for uname in ("u1", "symm", "u2"):
            U = paper_U(uname, gamma)
            kappa = float(np.linalg.cond(U, 2))
            for d in deltas:
                out.append(dict(path=path, U=uname, delta=float(d),
                                A=paper_matrix(U, paper_D(path, float(d))), kappa=kappa))
    return out


# --------------------------------------------------------------------------
# Random constructions (torch, any device)
# --------------------------------------------------------------------------

def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def haar_o3(n: int, g: torch.Generator, device, dtype=torch.float64) -> torch.Tensor:
    """(n, 3, 3) Haar-distributed orthogonal matrices (unit quaternion + sign)."""
    q = torch.randn(n, 4, generator=g, device=device, dtype=dtype)
    q = q / torch.linalg.vector_norm(q, dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y),
    ], dim=1).reshape(n, 3, 3)
    sign = torch.where(torch.rand(n, generator=g, device=device, dtype=dtype) < 0.5, -1.0, 1.0)
    return R * sign.to(dtype).view(n, 1, 1)


def log_uniform(n, lo, hi, g, device, dtype=torch.float64):
    u = torch.rand(n, generator=g, device=device, dtype=dtype)
    return torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


def uniform(shape, lo, hi, g, device, dtype=torch.float64):
    return lo + (hi - lo) * torch.rand(shape, generator=g, device=device, dtype=dtype)


def spectra(n: int, kinds: torch.Tensor, dlo: float, dhi: float, g, device) -> torch.Tensor:
    """Spectra by kind: 0 distinct U[-1,1]^3, 1 double (a, a+d, b),
    2 triple (a, a+d, a+2d), with d log-uniform in [dlo, dhi]."""
    lam = uniform((n, 3), -1.0, 1.0, g, device)
    d = log_uniform(n, dlo, dhi, g, device)
    a = lam[:, 0]
    dbl = torch.stack([a, a + d, lam[:, 2]], dim=1)
    tri = torch.stack([a, a + d, a + 2 * d], dim=1)
    k = kinds.view(n, 1)
    return torch.where(k == 0, lam, torch.where(k == 1, dbl, tri))


def symmetric_from_spectrum(lam: torch.Tensor, Q: torch.Tensor) -> torch.Tensor:
    """Q diag(lam) Q^T, explicitly symmetrised, (n, 3, 3)."""
    A = (Q * lam.unsqueeze(1)) @ Q.transpose(1, 2)
    return 0.5 * (A + A.transpose(1, 2))


def general_from_spectrum(lam, Q1, s, Q2) -> torch.Tensor:
    """V diag(lam) V^-1 with V = Q1 diag(s) Q2, (n, 3, 3)."""
    M = (Q2 * lam.unsqueeze(1)) @ Q2.transpose(1, 2)
    N = M * s.unsqueeze(2) / s.unsqueeze(1)
    return Q1 @ N @ Q1.transpose(1, 2)


def to_sym6(A: torch.Tensor) -> torch.Tensor:
    return torch.stack([A[:, i, j] for (i, j) in SYM6_INDEX], dim=1)


@dataclass
class Batch:
    """One synthetic workload: A in its storage layout, plus what the tests need."""
    A: torch.Tensor                  # (n, 9) or (n, 6), storage dtype
    layout: str                      # "general9" | "sym6"
    kappa: torch.Tensor              # (n,) kappa_2 of the eigenbasis used to build A
    lam_nominal: torch.Tensor        # (n, 3) prescribed spectrum (before rounding), FP64
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.A.shape[0])


def _general_chunk(n, g, device, kind_probs, dlo, dhi, scale_range=None):
    Q1 = haar_o3(n, g, device)
    Q2 = haar_o3(n, g, device)
    s = torch.exp(LN10 * torch.rand(n, 3, generator=g, device=device, dtype=torch.float64))
    u = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    c0, c1 = kind_probs[0], kind_probs[0] + kind_probs[1]
    kinds = torch.where(u < c0, 0, torch.where(u < c1, 1, 2))
    lam = spectra(n, kinds, dlo, dhi, g, device)
    if scale_range is not None:
        sc = torch.pow(10.0, uniform(n, scale_range[0], scale_range[1], g, device))
        lam = lam * sc.unsqueeze(1)
    A = general_from_spectrum(lam, Q1, s, Q2).reshape(n, 9)
    kappa = s.max(dim=1).values / s.min(dim=1).values
    return A, kappa, lam, kinds


def _sym_stress_chunk(n, g, device, frac_near, dlo, dhi, scale_exp):
    Q = haar_o3(n, g, device)
    sigma = torch.pow(10.0, uniform(n, -scale_exp, scale_exp, g, device))
    lam_free = uniform((n, 3), -1.0, 1.0, g, device)
    p = uniform(n, -1.0, 1.0, g, device)
    xi = uniform((n, 3), -1.0, 1.0, g, device)
    d = log_uniform(n, dlo, dhi, g, device)
    near = torch.rand(n, generator=g, device=device, dtype=torch.float64) < frac_near
    lam_near = p.unsqueeze(1) + d.unsqueeze(1) * xi
    lam = torch.where(near.unsqueeze(1), lam_near, lam_free) * sigma.unsqueeze(1)
    A = symmetric_from_spectrum(lam, Q)
    return to_sym6(A), lam, near


def _chunks(n, chunk):
    i = 0
    while i < n:
        yield i, min(chunk, n - i)
        i += chunk


def workload1(device="cpu") -> dict:
    """Workload 1: 4096 symmetric FP64 + 64 near-repeated cases, both layouts."""
    g = _gen(1001, device)
    n0 = 4096
    Q = haar_o3(n0 + 64, g, device)
    lam0 = uniform((n0, 3), -1.0, 1.0, g, device)
    deltas = torch.logspace(-1, -15, 32, dtype=torch.float64, device=device)
    ones = torch.ones_like(deltas)
    famA = torch.stack([ones, 1 + deltas, 2 * ones], dim=1)
    famB = torch.stack([ones, 1 + deltas, 1 + 2 * deltas], dim=1)
    lam = torch.cat([lam0, famA, famB], dim=0)
    A = symmetric_from_spectrum(lam, Q)
    n = A.shape[0]
    kappa = torch.ones(n, dtype=torch.float64, device=device)
    return dict(general9=Batch(A.reshape(n, 9).contiguous(), "general9", kappa, lam),
                sym6=Batch(to_sym6(A).contiguous(), "sym6", kappa, lam))


def workload2(n: int = 1 << 26, device="cpu", seed: int = 1002, chunk: int = 1 << 22) -> Batch:
    """Workload 2: general FP64, 1/3 distinct, 1/3 double, 1/3 triple."""
    g = _gen(seed, device)
    A = torch.empty((n, 9), dtype=torch.float64, device=device)
    kappa = torch.empty(n, dtype=torch.float64, device=device)
    lam = torch.empty((n, 3), dtype=torch.float64, device=device)
    kinds = torch.empty(n, dtype=torch.int64, device=device)
    for i, m in _chunks(n, chunk):
        a, k, l, kd = _general_chunk(m, g, device, (1 / 3, 1 / 3), 1e-16, 1e-2)
        A[i:i + m] = a; kappa[i:i + m] = k; lam[i:i + m] = l; kinds[i:i + m] = kd
    return Batch(A, "general9", kappa, lam, dict(kinds=kinds))


def illconditioned(n: int, device="cpu", seed: int = 1007, log10_kappa_max: float = 4.0,
                   chunk: int = 1 << 22) -> Batch:
    """General FP64 matrices with ill-conditioned eigenbases: V = Q1 diag(s) Q2
    with s = (1, 10^(t u), 10^t), t ~ U[0, log10_kappa_max], u ~ U[0, 1], so
    kappa_2(V) = 10^t; spectra one third each distinct / double / triple with
    delta log-uniform in [1e-12, 1e-2] (the paper's U2(1e-3) has kappa ~ 9e3)."""
    g = _gen(seed, device)
    A = torch.empty((n, 9), dtype=torch.float64, device=device)
    kappa = torch.empty(n, dtype=torch.float64, device=device)
    lam = torch.empty((n, 3), dtype=torch.float64, device=device)
    kinds = torch.empty(n, dtype=torch.int64, device=device)
    for i, m in _chunks(n, chunk):
        Q1 = haar_o3(m, g, device)
        Q2 = haar_o3(m, g, device)
        t = uniform(m, 0.0, log10_kappa_max, g, device)
        u = torch.rand(m, generator=g, device=device, dtype=torch.float64)
        sv = torch.stack([torch.ones_like(t), torch.pow(10.0, t * u), torch.pow(10.0, t)], dim=1)
        kd = torch.randint(0, 3, (m,), generator=g, device=device)
        lm = spectra(m, kd, 1e-12, 1e-2, g, device)
        A[i:i + m] = general_from_spectrum(lm, Q1, sv, Q2).reshape(m, 9)
        kappa[i:i + m] = torch.pow(10.0, t)
        lam[i:i + m] = lm
        kinds[i:i + m] = kd
    return Batch(A, "general9", kappa, lam, dict(kinds=kinds))


def workload3(n: int = 1 << 27, device="cpu", seed: int = 1003, chunk: int = 1 << 22) -> Batch:
    """Workload 3: symmetric 6-entry FP32 stress field."""
    g = _gen(seed, device)
    A = torch.empty((n, 6), dtype=torch.float32, device=device)
    lam = torch.empty((n, 3), dtype=torch.float64, device=device)
    near = torch.empty(n, dtype=torch.bool, device=device)
    for i, m in _chunks(n, chunk):
        a, l, nr = _sym_stress_chunk(m, g, device, 0.2, 1e-12, 1e-3, 6.0)
        A[i:i + m] = a.to(torch.float32); lam[i:i + m] = l; near[i:i + m] = nr
    kappa = torch.ones(n, dtype=torch.float64, device=device)
    return Batch(A, "sym6", kappa, lam, dict(near=near))


def workload4(n: int = 1 << 24, device="cpu", seed: int = 1004, chunk: int = 1 << 22) -> Batch:
    """Workload 4: as workload 2, plus loss weights w ~ N(0,1) per eigenvalue."""
    b = workload2(n, device, seed, chunk)
    g = _gen(seed + 500, device)
    b.extra["w"] = torch.randn((n, 3), generator=g, device=device, dtype=torch.float64)
    return b


def workload5(n: int = 1 << 28, device="cpu", seed: int = 1005, chunk: int = 1 << 22) -> dict:
    """Workload 5: half symmetric FP32, half general FP64, scales 10^U[-8,8]."""
    g = _gen(seed, device)
    h = n // 2
    S = torch.empty((h, 6), dtype=torch.float32, device=device)
    lamS = torch.empty((h, 3), dtype=torch.float64, device=device)
    for i, m in _chunks(h, chunk):
        a, l, _ = _sym_stress_chunk(m, g, device, 0.3, 1e-12, 1e-3, 8.0)
        S[i:i + m] = a.to(torch.float32); lamS[i:i + m] = l
    G = torch.empty((n - h, 9), dtype=torch.float64, device=device)
    kappa = torch.empty(n - h, dtype=torch.float64, device=device)
    lamG = torch.empty((n - h, 3), dtype=torch.float64, device=device)
    for i, m in _chunks(n - h, chunk):
        a, k, l, _ = _general_chunk(m, g, device, (0.35, 0.35), 1e-16, 1e-2, (-8.0, 8.0))
        G[i:i + m] = a; kappa[i:i + m] = k; lamG[i:i + m] = l
    gw = _gen(seed + 500, device)
    wS = torch.randn((h, 3), generator=gw, device=device, dtype=torch.float32)
    wG = torch.randn((n - h, 3), generator=gw, device=device, dtype=torch.float64)
    return dict(sym6=Batch(S, "sym6", torch.ones(h, dtype=torch.float64, device=device), lamS,
                           dict(w=wS)),
                general9=Batch(G, "general9", kappa, lamG, dict(w=wG)))


def gradient_batch(n: int, device="cpu", seed: int = 2001, min_gap: float = 1e-2) -> Batch:
    """General FP64 matrices whose spectra have relative gaps >= min_gap
    (relative to the spectral spread), for finite-difference gradient checks."""
    g = _gen(seed, device)
    Q1 = haar_o3(n, g, device)
    Q2 = haar_o3(n, g, device)
    s = torch.exp(LN10 * torch.rand(n, 3, generator=g, device=device, dtype=torch.float64))
    base = torch.tensor([-1.0, 0.0, 1.0], dtype=torch.float64, device=device)
    jit = uniform((n, 3), -0.5 + min_gap, 0.5 - min_gap, g, device) * 0.9
    lam = base + jit
    A = general_from_spectrum(lam, Q1, s, Q2).reshape(n, 9)
    kappa = s.max(dim=1).values / s.min(dim=1).values
    return Batch(A, "general9", kappa, lam)


def lode_sweep(n: int, j2: float = 150.0) -> np.ndarray:
    """The stress states of the paper's yield-function study (Section
    "Application"): sigma = U_symm diag(s1, s2, s3) U_symm^T with
    s_k = (2/3) sqrt(3 J2) cos(theta + 2 pi k / 3), theta evenly over [0, 2 pi),
    J2 = 150 (MPa^2).  Returns (n, 6) symmetric rows (A00, A11, A22, A12, A02, A01)."""
    U = paper_U("symm")
    th = np.arange(n) * (2.0 * np.pi / n)
    out = np.empty((n, 6))
    for i, t in enumerate(th):
        s = [(2.0 / 3.0) * np.sqrt(3.0 * j2) * np.cos(t + 2.0 * np.pi * k / 3.0) for k in (1, 2, 3)]
        A = U @ np.diag(s) @ U.T
        A = 0.5 * (A + A.T)
        out[i] = [A[0, 0], A[1, 1], A[2, 2], A[1, 2], A[0, 2], A[0, 1]]
    return out


def stress_field(n: int, device="cpu", seed: int = 1006, scale: float = 100.0) -> Batch:
    """Symmetric stress states of engineering magnitude (MPa): Haar rotations
    of principal stresses with hydrostatic part p ~ U[-2, 1] scale, deviatoric
    radius log-uniform in [1e-3, 1] scale and Lode angle U[0, 2 pi)."""
    g = _gen(seed, device)
    Q = haar_o3(n, g, device)
    p = uniform(n, -2.0, 1.0, g, device) * scale
    rad = log_uniform(n, 1e-3, 1.0, g, device) * scale
    th = uniform(n, 0.0, 2.0 * math.pi, g, device)
    k = torch.arange(1, 4, device=device, dtype=torch.float64)
    lam = p.unsqueeze(1) + (2.0 / 3.0) * rad.unsqueeze(1) * torch.cos(
        th.unsqueeze(1) + 2.0 * math.pi * k / 3.0)
    A = symmetric_from_spectrum(lam, Q)
    return Batch(to_sym6(A).contiguous(), "sym6", torch.ones(n, dtype=torch.float64,
                                                             device=device), lam)


def sample_indices(n: int, k: int, seed: int = 7) -> np.ndarray:
    """k sorted distinct indices in [0, n), always including the first and last."""
    rng = np.random.default_rng(seed)
    if k >= n:
        return np.arange(n)
    idx = rng.choice(n, size=k, replace=False)
    idx[0] = 0
    idx[1] = n - 1
    return np.unique(idx)
