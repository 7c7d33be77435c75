"""Batched, numerically stable closed-form eigenvalues of real 3x3 matrices on
GB300 (sm_103a), after Habera & Zilian, arXiv 2511.00292.

Every step of the computation runs in the CUDA library ``libeig3.so``
(include/eig3.h); this module only allocates outputs with torch and passes
pointers and the current CUDA stream.  There is no CPU path: inputs must be
CUDA tensors, or page-locked (pinned) host tensors that the kernels read and
write directly over the host link (zero copy), and the library must be built.

Layouts: ``"general9"`` (n, 9) row-major, or (n, 3, 3); ``"sym6"`` (n, 6) in
the order (A00, A11, A22, A12, A02, A01).
Precisions: ``"f64"`` (binary64 arithmetic; storage float64 or float32),
``"f32c"`` (compensated binary32 arithmetic; storage float32), ``"f32c64"``
(the same with the final combination of Delta and the triple angle in binary64;
eigenvalues and adjoint only) and ``"f64g"`` (binary64 with the guard for
ill-conditioned eigenbases: a strongly non-normal matrix gets its eigenvalues
from the shifted QR algorithm instead of the closed form; eigenvalues and
adjoint only).

Entry points: :func:`eigvals`, :func:`eigvals_backward`, :func:`eigvals_ad`
(autograd), :func:`eigvals_vjp` (eigenvalues and the gradient of a loss linear
in them, fused), :func:`invariants`, :func:`eigprojectors`, :func:`mohr_coulomb`,
:func:`eigvals_variant` (the paper's comparison variants), :class:`Stats`;
host-resident batches stream through :class:`host.HostPipeline`.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import (F32, F64, GENERAL9, PREC_F32_COMP, PREC_F64, SYM6, Eig3Error, Eig3Stats,
                   check, load)

__all__ = ["eigvals", "invariants", "eigvals_backward", "eigvals_ad", "eigvals_vjp",
           "eigprojectors",
           "mohr_coulomb", "eigvals_variant", "Stats", "Eig3Error", "layout_of", "GENERAL9",
           "SYM6"]

_LAYOUTS = {"general9": GENERAL9, "sym6": SYM6, GENERAL9: GENERAL9, SYM6: SYM6}
_PRECS = {"f64": PREC_F64, "f32c": PREC_F32_COMP, "f64g": _lib.PREC_F64_GUARDED,
          "f32c64": _lib.PREC_F32_COMP_A64,
          PREC_F64: PREC_F64, PREC_F32_COMP: PREC_F32_COMP,
          _lib.PREC_F64_GUARDED: _lib.PREC_F64_GUARDED,
          _lib.PREC_F32_COMP_A64: _lib.PREC_F32_COMP_A64}


def layout_of(A: torch.Tensor, layout=None) -> int:
    if layout is not None:
        return _LAYOUTS[layout]
    if A.dim() >= 2 and A.shape[-2:] == (3, 3):
        return GENERAL9
    if A.shape[-1] == 9:
        return GENERAL9
    if A.shape[-1] == 6:
        return SYM6
    raise ValueError(f"cannot infer the layout of a tensor of shape {tuple(A.shape)}")


def _rows(A: torch.Tensor, layout: int) -> torch.Tensor:
    w = 9 if layout == GENERAL9 else 6
    if not A.is_cuda and not A.is_pinned():
        raise ValueError("eig3 runs on the GPU: pass a CUDA tensor, or a page-locked (pinned) "
                         "host tensor that the kernels read directly; there is no CPU path")
    if A.dtype not in (torch.float64, torch.float32):
        raise TypeError(f"unsupported dtype {A.dtype}; use float64 or float32")
    if not A.is_contiguous():
        raise ValueError("A must be contiguous")
    if A.numel() % w != 0:
        raise ValueError(f"A has {A.numel()} elements, not a multiple of {w}")
    return A.reshape(-1, w)


def _dtype_code(t: torch.Tensor) -> int:
    return F64 if t.dtype == torch.float64 else F32


def _stream(dev: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _device(X: torch.Tensor, device=None) -> torch.device:
    """The GPU that runs the kernels: the tensor's own, or for pinned host
    tensors `device` (default: the current CUDA device)."""
    if X.is_cuda:
        return X.device
    if device is not None:
        return torch.device(device)
    return torch.device("cuda", torch.cuda.current_device())


def _alloc(shape, dtype, like: torch.Tensor, dev: torch.device) -> torch.Tensor:
    """Outputs live where the input lives: on the GPU, or in pinned host memory
    (written by the kernels over the host link) for pinned host inputs."""
    if like.is_cuda:
        return torch.empty(shape, dtype=dtype, device=dev)
    return torch.empty(shape, dtype=dtype, pin_memory=True)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _out(t, numel: int, dtype, name: str):
    """A caller-supplied output: the kernels write numel elements of dtype
    through its pointer, so it must hold exactly that, contiguously, where the
    GPU can write it (device or pinned host memory)."""
    if t.dtype != dtype or t.numel() != numel or not t.is_contiguous() or not (
            t.is_cuda or t.is_pinned()):
        raise ValueError(f"{name} must be a contiguous CUDA or pinned tensor of {numel} "
                         f"{dtype} elements (got {tuple(t.shape)} {t.dtype})")
    return t


class Stats:
    """Device-resident eig3_stats accumulated by :func:`eigvals` (see eig3.h)."""

    def __init__(self, device=None):
        self.buf = torch.empty(6, dtype=torch.float64,
                               device=device if device is not None else torch.device("cuda"))
        self.reset()

    def reset(self):
        with torch.cuda.device(self.buf.device):
            check(load().eig3_stats_reset(_ptr(self.buf), _stream(self.buf.device)),
                  "eig3_stats_reset")

    def read(self) -> dict:
        raw = self.buf.cpu().numpy().tobytes()
        s = Eig3Stats.from_buffer_copy(raw)
        return {f: getattr(s, f) for f, _ in Eig3Stats._fields_}


def invariants(A: torch.Tensor, layout=None, precision="f64", device=None) -> torch.Tensor:
    """(n, 4) float64 tensor of (I1, J2, J3, Delta) (Algorithms 1, 2, 4, 5)."""
    lay = layout_of(A, layout)
    X = _rows(A, lay)
    dev = _device(X, device)
    out = _alloc((X.shape[0], 4), torch.float64, X, dev)
    with torch.cuda.device(dev):
        st = load().eig3_invariants(_ptr(X), lay, _dtype_code(X), _PRECS[precision], X.shape[0],
                                    _ptr(out), _stream(dev))
    check(st, "eig3_invariants")
    return out


def eigvals(A: torch.Tensor, layout=None, precision="f64", return_aux=False, stats=None,
            out=None, aux_out=None, device=None):
    """Ascending eigenvalues, (n, 3) in the storage dtype (Algorithm 6).

    With ``return_aux`` also returns the (n, 4) adjoint inputs
    (r, sin(phi/3), sin((pi-phi)/3), I1) for :func:`eigvals_backward`.
    ``out`` / ``aux_out`` may supply preallocated outputs (CUDA-graph use).
    A pinned host ``A`` is read by the kernels directly (zero copy); the
    eigenvalues then go to pinned host memory and ``aux`` to the GPU.
    """
    lay = layout_of(A, layout)
    X = _rows(A, lay)
    n = X.shape[0]
    dev = _device(X, device)
    lam = _out(out, 3 * n, X.dtype, "out") if out is not None else _alloc((n, 3), X.dtype, X, dev)
    aux = None
    if return_aux:
        aux = (_out(aux_out, 4 * n, X.dtype, "aux_out") if aux_out is not None
               else torch.empty((n, 4), dtype=X.dtype, device=dev))
    if stats is not None and not (stats.buf.is_cuda and stats.buf.numel() == 6):
        raise ValueError("stats must be a Stats object")
    sp = _ptr(stats.buf) if stats is not None else None
    with torch.cuda.device(dev):
        st = load().eig3_eigvals(_ptr(X), lay, _dtype_code(X), _PRECS[precision], n, _ptr(lam),
                                 _ptr(aux), sp, _stream(dev))
    check(st, "eig3_eigvals")
    return (lam, aux) if return_aux else lam


def eigvals_backward(A: torch.Tensor, grad_lam: torch.Tensor, aux=None, layout=None,
                     precision="f64", out=None, device=None) -> torch.Tensor:
    """dL/dA (same shape and dtype as the stored rows) given dL/dlambda (n, 3).
    Pinned host ``A`` / ``grad_lam`` are read directly by the kernels."""
    lay = layout_of(A, layout)
    X = _rows(A, lay)
    g = grad_lam if grad_lam.is_contiguous() else grad_lam.contiguous()
    if g.dtype != X.dtype or g.numel() != 3 * X.shape[0] or not (g.is_cuda or g.is_pinned()):
        raise ValueError("grad_lam must be a CUDA or pinned (n, 3) tensor of the storage dtype")
    if aux is not None and (aux.dtype != X.dtype or aux.numel() != 4 * X.shape[0]):
        raise ValueError("aux must be the (n, 4) tensor returned by eigvals(return_aux=True)")
    dev = _device(X, device)
    gA = (_out(out, X.numel(), X.dtype, "out") if out is not None
          else _alloc(tuple(X.shape), X.dtype, X, dev))
    with torch.cuda.device(dev):
        st = load().eig3_eigvals_backward(_ptr(X), lay, _dtype_code(X), _PRECS[precision],
                                          X.shape[0], _ptr(g), _ptr(aux), _ptr(gA),
                                          _stream(dev))
    check(st, "eig3_eigvals_backward")
    return gA


def eigvals_vjp(A: torch.Tensor, w: torch.Tensor, layout=None, precision="f64",
                return_eigvals=True, stats=None, out=None, grad_out=None, device=None):
    """Eigenvalues (n, 3) and dL/dA for L = sum_k w_k lambda_k in one fused
    pass (eig3_eigvals_vjp): returns (lam, grad_A), or grad_A alone with
    ``return_eigvals=False``.  ``w`` is (n, 3) in the storage dtype."""
    lay = layout_of(A, layout)
    X = _rows(A, lay)
    n = X.shape[0]
    wc = w if w.is_contiguous() else w.contiguous()
    if wc.dtype != X.dtype or wc.numel() != 3 * n or not (wc.is_cuda or wc.is_pinned()):
        raise ValueError("w must be a CUDA or pinned (n, 3) tensor of the storage dtype")
    dev = _device(X, device)
    lam = None
    if return_eigvals:
        lam = _out(out, 3 * n, X.dtype, "out") if out is not None else _alloc((n, 3), X.dtype,
                                                                             X, dev)
    gA = (_out(grad_out, X.numel(), X.dtype, "grad_out") if grad_out is not None
          else _alloc(tuple(X.shape), X.dtype, X, dev))
    if stats is not None and not (stats.buf.is_cuda and stats.buf.numel() == 6):
        raise ValueError("stats must be a Stats object")
    sp = _ptr(stats.buf) if stats is not None else None
    with torch.cuda.device(dev):
        st = load().eig3_eigvals_vjp(_ptr(X), lay, _dtype_code(X), _PRECS[precision], n,
                                     _ptr(wc), _ptr(lam), _ptr(gA), sp, _stream(dev))
    check(st, "eig3_eigvals_vjp")
    return (lam, gA) if return_eigvals else gA


def eigprojectors(A: torch.Tensor, layout=None, precision="f64", return_eigvals=False,
                  out=None, lam_out=None, device=None):
    """Eigenprojectors E_1, E_2, E_3 (n, 3, 3, 3) with E_k^T = d lambda_k / dA
    (ascending order); optionally also the eigenvalues (n, 3)."""
    lay = layout_of(A, layout)
    X = _rows(A, lay)
    n = X.shape[0]
    dev = _device(X, device)
    P = _out(out, 27 * n, X.dtype, "out") if out is not None else _alloc((n, 3, 3, 3), X.dtype,
                                                                         X, dev)
    lam = None
    if return_eigvals:
        lam = (_out(lam_out, 3 * n, X.dtype, "lam_out") if lam_out is not None
               else _alloc((n, 3), X.dtype, X, dev))
    with torch.cuda.device(dev):
        st = load().eig3_eigprojectors(_ptr(X), lay, _dtype_code(X), _PRECS[precision], n,
                                       _ptr(lam), _ptr(P), _stream(dev))
    check(st, "eig3_eigprojectors")
    return (P, lam) if return_eigvals else P


def mohr_coulomb(sigma: torch.Tensor, s_yc: float = 100.0, m: float = 10.0, layout=None,
                 precision="f64", grad=False, out=None, grad_out=None, device=None):
    """Mohr-Coulomb yield value f(sigma) per stress tensor (n,), and with
    grad=True also df/dsigma in sigma's storage layout (n, 9) or (n, 6)."""
    lay = layout_of(sigma, layout)
    X = _rows(sigma, lay)
    n = X.shape[0]
    dev = _device(X, device)
    f = _out(out, n, X.dtype, "out") if out is not None else _alloc((n,), X.dtype, X, dev)
    g = None
    if grad:
        g = (_out(grad_out, X.numel(), X.dtype, "grad_out") if grad_out is not None
             else _alloc(tuple(X.shape), X.dtype, X, dev))
    with torch.cuda.device(dev):
        st = load().eig3_mohr_coulomb(_ptr(X), lay, _dtype_code(X), _PRECS[precision], n,
                                      float(s_yc), float(m), _ptr(f), _ptr(g), _stream(dev))
    check(st, "eig3_mohr_coulomb")
    return (f, g) if grad else f


_VARIANTS = {"present": _lib.VARIANT_PRESENT, "naive": _lib.VARIANT_NAIVE,
             "naive_tensor": _lib.VARIANT_NAIVE_TENSOR}


def eigvals_variant(A: torch.Tensor, variant: str, layout=None, invariants=True, eigvals=True,
                    inv_out=None, lam_out=None, device=None):
    """The paper's comparison variants ("naive", "naive_tensor") or the method
    itself ("present"), binary64 arithmetic: returns (inv (n, 4) or None,
    lam (n, 3) or None).  For stability measurements, not for results."""
    lay = layout_of(A, layout)
    X = _rows(A, lay)
    n = X.shape[0]
    dev = _device(X, device)
    inv = None
    if invariants:
        inv = (_out(inv_out, 4 * n, torch.float64, "inv_out") if inv_out is not None
               else _alloc((n, 4), torch.float64, X, dev))
    lam = None
    if eigvals:
        lam = (_out(lam_out, 3 * n, X.dtype, "lam_out") if lam_out is not None
               else _alloc((n, 3), X.dtype, X, dev))
    with torch.cuda.device(dev):
        st = load().eig3_eigvals_variant(_ptr(X), lay, _dtype_code(X), _VARIANTS[variant], n,
                                         _ptr(inv), _ptr(lam), _stream(dev))
    check(st, "eig3_eigvals_variant")
    return inv, lam


class _Eig3Fn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, layout, precision):
        lam, aux = eigvals(A, layout=layout, precision=precision, return_aux=True)
        ctx.save_for_backward(A, aux)
        ctx.layout = layout
        ctx.precision = precision
        return lam

    @staticmethod
    def backward(ctx, grad_lam):
        A, aux = ctx.saved_tensors
        gA = eigvals_backward(A, grad_lam.contiguous(), aux=aux, layout=ctx.layout,
                              precision=ctx.precision)
        return gA.reshape(A.shape), None, None


def eigvals_ad(A: torch.Tensor, layout=None, precision="f64") -> torch.Tensor:
    """Differentiable eigenvalues: the backward pass is the library's adjoint kernel."""
    lay = layout_of(A, layout)
    lam = _Eig3Fn.apply(A.contiguous(), lay, precision)
    return lam
