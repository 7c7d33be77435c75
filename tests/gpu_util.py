"""Shared helpers of the GPU parity tests: tolerances and comparisons.

Tolerances (all per matrix, on the same seeded inputs as the oracle):

* binary64 eigenvalues: |lambda_gpu - lambda_oracle| <= 2 b + 4 ulp64(max|lambda|),
  with b = C kappa ||A||_F u64 the paper's per-matrix eigenvalue stability bound
  (Lemma of Section "Eigenvalues") and its moderate constant taken as C = 8: the
  smallest power of two that the oracle itself meets against exact eigenvalues
  on its pinned cases (measured up to 7.4; the literal evaluation of
  cos((phi + 2 pi k)/3) dominates).  Two evaluations each within b of the
  exact eigenvalues differ by at most 2 b.
* binary64 path on binary32 storage: the binary64 result rounded once to
  binary32, so add 0.5 ulp32 of the larger of the two values compared.
* compensated binary32 eigenvalues: the paper's bound at binary32 unit
  roundoff plus the final rounding to binary32,
  |lambda_gpu - lambda_oracle| <= C32 kappa ||A||_F u32 + 2 ulp32(max|lambda|),
  C32 = 8; the ulp term also covers matrices whose eigenvalues fall in the
  binary32 subnormal range, where the output spacing is 2^-149.  Measured
  maxima are printed.
* invariants: C_inv times the paper's first-order bound of each invariant
  (I1: ||A|| u, J2: ||dev A||^2 u, J3: ||dev cof dev A|| ||dev A|| u,
  Delta: ||dev(12 J2^2 A^T - 54 J3 cof dev A)|| ||dev A|| u), kappa^2-scaled
  for J3 and Delta which the paper shows to be only conditionally stable.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

U64 = 2.0 ** -53
U32 = 2.0 ** -24
EIG_C = 8.0


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().double().numpy()


def oracle_eigs(A: np.ndarray, layout: int):
    lam = np.sort(oracle.eigvals(A, layout=layout), axis=1)
    return lam


def eig_tol_f64(A: np.ndarray, kappa, layout: int, lam_ref: np.ndarray) -> np.ndarray:
    b = EIG_C * oracle.bounds(A, kappa, layout=layout)[:, 4]
    return 2.0 * b + 4.0 * np.spacing(np.abs(lam_ref).max(axis=1))


def check_eig_f64(lam_gpu: np.ndarray, A: np.ndarray, kappa, layout: int, f32_storage=False):
    ref = oracle_eigs(A, layout)
    tol = eig_tol_f64(A, kappa, layout, ref)[:, None] * np.ones((1, 3))
    if f32_storage:
        big = np.maximum(np.abs(ref), np.abs(lam_gpu)).astype(np.float32)
        tol = tol + 0.5 * np.spacing(big).astype(np.float64) * (1 + 1e-6)
    err = np.abs(lam_gpu - ref)
    bad = ~(err <= tol)
    return err, tol, bad


def check_eig_f32c(lam_gpu: np.ndarray, A: np.ndarray, kappa, layout: int, c32: float = 8.0):
    ref = oracle_eigs(A, layout)
    nA = np.linalg.norm(A if layout == 0 else oracle.sym6_to_general9(A), axis=1)
    ulp = np.spacing(np.abs(ref).max(axis=1).astype(np.float32)).astype(np.float64)
    tol = c32 * np.asarray(kappa) * nA * U32 + 2.0 * ulp
    err = np.abs(lam_gpu - ref).max(axis=1)
    return err, tol, err / np.where(ulp > 0, ulp, 1.0)


def check_invariants(inv_gpu: np.ndarray, A: np.ndarray, kappa, layout: int, u: float,
                     c_inv: float = 16.0):
    ref = oracle.invariants(A, layout=layout)
    b = oracle.bounds(A, kappa, layout=layout, u=u)[:, :4]
    k2 = np.asarray(kappa, dtype=np.float64).reshape(-1) ** 2 * np.ones(A.shape[0])
    scale = np.stack([np.ones_like(k2), np.ones_like(k2), k2, k2], axis=1)
    # both sides carry their own rounding errors: the oracle's at u64
    b64 = oracle.bounds(A, kappa, layout=layout, u=U64)[:, :4]
    tol = c_inv * scale * (b + b64)
    err = np.abs(inv_gpu - ref)
    return err, tol
