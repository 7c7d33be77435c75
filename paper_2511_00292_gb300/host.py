"""Host-resident batches: stream chunks through the GPU.

For a batch that lives in page-locked host memory, `HostPipeline` runs the
library's forward and adjoint on fixed-size chunks with three CUDA streams:
host-to-device copies of chunk i+1, the kernels on chunk i and the
device-to-host copies of chunk i-1 overlap, so the step costs about the
slowest of the three instead of their sum.  The three stages touch three
different device slots, so the default depth is 3 (with 2, the copy of chunk
i+1 would wait for the copy-back of chunk i-1 from the same slot and the two
copy directions would not overlap).  The device slots are allocated
once per pipeline with torch (plumbing; the kernels only see their inputs and
outputs).  Every computation is a call of the C ABI.

`pinned_empty` / `pinned_copy` allocate the host side: page-locked memory
backed by transparent huge pages, which the copy engines read and write at the
link rate throughout (see `pinned_empty`).
"""
from __future__ import annotations

import ctypes
import math
import mmap

import torch

from . import eigvals, eigvals_backward, eigvals_vjp, layout_of


def _huge_backed_bytes(lo: int, hi: int) -> int:
    """Bytes of [lo, hi) that /proc/self/smaps reports as backed by anonymous
    huge pages (summed over the mappings overlapping the range)."""
    total = 0
    inside = False
    try:
        with open("/proc/self/smaps") as f:
            for line in f:
                head = line.split(None, 1)[0]
                if "-" in head and not head.endswith(":"):
                    a, b = head.split("-")
                    inside = int(a, 16) < hi and int(b, 16) > lo
                elif inside and head == "AnonHugePages:":
                    total += int(line.split()[1]) * 1024
    except OSError:
        return 0
    return total


class _PinnedMap(mmap.mmap):
    """Page-locked host memory behind `pinned_empty`: an anonymous private
    mapping advised for transparent huge pages (MADV_HUGEPAGE) and registered
    with cudaHostRegister.  torch.frombuffer keeps a reference to the mapping
    itself, so it stays registered and mapped while any tensor views it; the
    finalizer unregisters it before the mapping is unmapped."""

    @classmethod
    def create(cls, nbytes: int) -> "_PinnedMap":
        m = cls(-1, int(nbytes), flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        m.ptr = None
        if hasattr(mmap, "MADV_HUGEPAGE"):
            m.madvise(mmap.MADV_HUGEPAGE)
        probe = (ctypes.c_char * int(nbytes)).from_buffer(m)
        ptr = ctypes.addressof(probe)
        del probe
        err = torch.cuda.cudart().cudaHostRegister(ptr, int(nbytes), 0)
        if int(getattr(err, "value", err)) != 0:
            m.close()
            raise RuntimeError(f"cudaHostRegister of {nbytes} bytes failed: {err}")
        m.ptr = ptr
        return m

    def __del__(self):
        ptr = self.__dict__.get("ptr")
        if ptr is not None:
            self.ptr = None
            try:
                torch.cuda.cudart().cudaHostUnregister(ptr)
            except Exception:  # interpreter shutdown
                pass


def pinned_empty(shape, dtype=torch.float64) -> torch.Tensor:
    """An uninitialised page-locked host tensor, for HostPipeline and for the
    kernels' zero-copy path.

    The memory is an anonymous mapping backed by transparent huge pages and
    registered with cudaHostRegister.  On GB300 (64 KiB base pages, 512 MiB huge
    pages) buffers from torch's pinned allocator at times copied to the device at
    11-13 GB/s over whole GiB ranges while the rest of the buffer ran at 211 GB/s,
    so the same streamed step took 107 to 199 ms from one repetition to the next;
    with buffers from this function it took 106.5 ms every time, the rate of the
    two copy directions at once."""
    shape = tuple(int(d) for d in (shape if isinstance(shape, (tuple, list, torch.Size))
                                   else (shape,)))
    nbytes = math.prod(shape) * torch.empty((), dtype=dtype).element_size()
    if nbytes == 0:
        return torch.empty(shape, dtype=dtype, pin_memory=True)
    region = _PinnedMap.create(nbytes)
    return torch.frombuffer(region, dtype=torch.uint8, count=nbytes).view(dtype).view(shape)


def huge_page_fraction(t: torch.Tensor) -> float:
    """The fraction of the host tensor t's bytes backed by transparent huge
    pages (0 where the kernel does not report it)."""
    nbytes = t.numel() * t.element_size()
    if nbytes == 0:
        return 1.0
    return min(1.0, _huge_backed_bytes(t.data_ptr(), t.data_ptr() + nbytes) / nbytes)


def pinned_copy(t: torch.Tensor) -> torch.Tensor:
    """A `pinned_empty` host tensor holding a copy of t (host or device)."""
    out = pinned_empty(t.shape, t.dtype)
    out.copy_(t)
    return out


class HostPipeline:
    def __init__(self, device=None, chunk: int = 1 << 24, depth: int = 3):
        self.dev = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.chunk = int(chunk)
        self.depth = int(depth)
        self.s_in = torch.cuda.Stream(self.dev)
        self.s_run = torch.cuda.Stream(self.dev)
        self.s_out = torch.cuda.Stream(self.dev)
        self._slots = {}

    # The device slots of a slot set are one fresh allocation, cut at 2 MiB
    # boundaries.  Cached allocator blocks that earlier kernels had written
    # took host-to-device copies at 20-100 GB/s instead of 200 GB/s, so the
    # allocator's cache is released first and the slots come from new device
    # memory (a one-time cost per slot set).
    _ALIGN = 1 << 21

    def _get_slots(self, key, width, dtype):
        if key not in self._slots:
            c, d, al = self.chunk, self.depth, self._ALIGN
            esize = torch.empty((), dtype=dtype).element_size()
            widths = {"A": width, "w": 3, "lam": 3, "aux": 4, "g": width}
            span = lambda w: (c * w * esize + al - 1) // al * al
            total = d * sum(span(w) for w in widths.values())
            torch.cuda.synchronize(self.dev)
            torch.cuda.empty_cache()
            raw = torch.empty(total + al, dtype=torch.uint8, device=self.dev)
            off = (-raw.data_ptr()) % al
            slots = {}
            for name, w in widths.items():
                views = []
                for _ in range(d):
                    views.append(raw[off:off + c * w * esize].view(dtype).view(c, w))
                    off += span(w)
                slots[name] = views
            slots.update(raw=raw, free=[torch.cuda.Event() for _ in range(d)],
                         loaded=[torch.cuda.Event() for _ in range(d)],
                         done=[torch.cuda.Event() for _ in range(d)])
            self._slots[key] = slots
        return self._slots[key]

    def forward_backward(self, A: torch.Tensor, w: torch.Tensor, lam_out: torch.Tensor,
                         grad_out: torch.Tensor, layout=None, precision="f64"):
        """Eigenvalues of every row of the pinned host tensor A into lam_out and the
        gradient of sum(w * lambda) into grad_out (both pinned host tensors).
        Asynchronous with respect to the host; ordered after the current stream's
        pending work, and the current stream waits for the last copy."""
        self.run([(A, w, lam_out, grad_out, layout, precision)])

    def run(self, jobs):
        """Several forward_backward jobs, (A, w, lam_out, grad_out, layout,
        precision) each, streamed back to back: the chunks of the next job enter
        the pipeline while the last ones of the previous job are still in it."""
        for A, w, lam_out, grad_out, layout, _ in jobs:
            for t in (A, w, lam_out, grad_out):
                if t.is_cuda or not t.is_pinned() or not t.is_contiguous():
                    raise ValueError("HostPipeline works on contiguous pinned host tensors")
            n = A.numel() // (9 if layout_of(A, layout) == 0 else 6)
            if any(t.dtype != A.dtype for t in (w, lam_out, grad_out)) or w.numel() != 3 * n \
                    or lam_out.numel() != 3 * n or grad_out.numel() != A.numel():
                raise ValueError("w and lam_out must hold (n, 3) and grad_out A's shape, all in "
                                 "A's dtype")
        main = torch.cuda.current_stream(self.dev)
        for s in (self.s_in, self.s_run, self.s_out):
            s.wait_stream(main)
        used = {}  # chunks issued per slot set in this run
        for A, w, lam_out, grad_out, layout, precision in jobs:
            lay = layout_of(A, layout)
            width = 9 if lay == 0 else 6
            X = A.reshape(-1, width)
            n = X.shape[0]
            key = (width, A.dtype)
            slots = self._get_slots(key, width, A.dtype)
            for lo in range(0, n, self.chunk):
                i = used.get(key, 0)
                used[key] = i + 1
                hi = min(n, lo + self.chunk)
                m = hi - lo
                k = i % self.depth
                dA, dw = slots["A"][k][:m], slots["w"][k][:m]
                dl, da, dg = slots["lam"][k][:m], slots["aux"][k][:m], slots["g"][k][:m]
                with torch.cuda.stream(self.s_in):
                    if i >= self.depth:
                        self.s_in.wait_event(slots["free"][k])
                    dA.copy_(X[lo:hi], non_blocking=True)
                    dw.copy_(w[lo:hi], non_blocking=True)
                    slots["loaded"][k].record(self.s_in)
                with torch.cuda.stream(self.s_run):
                    self.s_run.wait_event(slots["loaded"][k])
                    if precision in ("f64", "f32c"):  # fused forward + vector-Jacobian product
                        eigvals_vjp(dA, dw, layout=lay, precision=precision, out=dl,
                                    grad_out=dg)
                    else:
                        eigvals(dA, layout=lay, precision=precision, return_aux=True, out=dl,
                                aux_out=da)
                        eigvals_backward(dA, dw, aux=da, layout=lay, precision=precision,
                                         out=dg)
                    slots["done"][k].record(self.s_run)
                with torch.cuda.stream(self.s_out):
                    self.s_out.wait_event(slots["done"][k])
                    lam_out[lo:hi].copy_(dl, non_blocking=True)
                    grad_out.reshape(-1, width)[lo:hi].copy_(dg, non_blocking=True)
                    slots["free"][k].record(self.s_out)
        main.wait_stream(self.s_out)

    def capture(self, jobs) -> torch.cuda.CUDAGraph:
        """run(jobs) captured once into a CUDA graph (copies, kernels and the
        cross-stream dependencies); each replay() repeats the whole run on the
        same host and device buffers with a single launch from the host."""
        self.run(jobs)  # allocates the device slots and loads the library
        torch.cuda.synchronize(self.dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(jobs)
        return g

