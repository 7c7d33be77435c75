"""Host-side logic of the huge-page pinned allocator (`host.pinned_empty`),
with a fake CUDA runtime recording cudaHostRegister / cudaHostUnregister: the
region is registered once, stays registered while any tensor views it, and is
unregistered exactly once after the last view is gone; a failed registration
raises.  (The copy rates themselves are measured on the GPU.)"""
import gc
import mmap

import pytest
import torch

from paper_2511_00292_gb300 import host


class FakeCudart:
    def __init__(self, fail=False):
        self.calls = []
        self.fail = fail

    def cudaHostRegister(self, ptr, nbytes, flags):
        self.calls.append(("register", ptr, nbytes, flags))
        return 2 if self.fail else 0

    def cudaHostUnregister(self, ptr):
        self.calls.append(("unregister", ptr))
        return 0


@pytest.fixture
def fake(monkeypatch):
    f = FakeCudart()
    monkeypatch.setattr(torch.cuda, "cudart", lambda: f)
    return f


def test_region_lives_while_any_view_does(fake):
    t = host.pinned_empty((1000, 9), torch.float64)
    assert t.shape == (1000, 9) and t.dtype == torch.float64 and t.is_contiguous()
    assert t.data_ptr() % mmap.PAGESIZE == 0
    assert fake.calls == [("register", t.data_ptr(), 72000, 0)]
    ptr = t.data_ptr()
    v = t[10:20]
    del t
    gc.collect()
    assert len(fake.calls) == 1                 # the view keeps the region registered
    v.fill_(1.5)
    assert float(v.sum()) == 1.5 * 90
    del v
    gc.collect()
    assert fake.calls[1:] == [("unregister", ptr)]


def test_shapes_dtypes_and_copy(fake):
    x = torch.arange(6 * 7, dtype=torch.float32).reshape(7, 6)
    y = host.pinned_copy(x)
    assert y.dtype == torch.float32 and y.shape == (7, 6) and torch.equal(x, y)
    z = host.pinned_empty(5, torch.float64)
    assert z.shape == (5,)
    w = host.pinned_empty(torch.Size([3, 4]), torch.int64)
    assert w.shape == (3, 4) and w.element_size() == 8
    regs = [c for c in fake.calls if c[0] == "register"]
    assert [c[2] for c in regs] == [168, 40, 96]
    del y, z, w
    gc.collect()
    assert sum(c[0] == "unregister" for c in fake.calls) == 3


def test_failed_registration_raises(monkeypatch):
    f = FakeCudart(fail=True)
    monkeypatch.setattr(torch.cuda, "cudart", lambda: f)
    with pytest.raises(RuntimeError, match="cudaHostRegister"):
        host.pinned_empty((64, 6), torch.float32)
    gc.collect()
    assert [c[0] for c in f.calls] == ["register"]  # nothing to unregister


def test_huge_page_fraction_reads_smaps():
    """The smaps reader finds the anonymous huge pages (or none) of a live
    mapping without error; a range outside every mapping counts 0; an empty
    tensor counts as fully backed."""
    m = mmap.mmap(-1, 1 << 20, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    import ctypes
    buf = (ctypes.c_char * (1 << 20)).from_buffer(m)
    a = ctypes.addressof(buf)
    buf[0] = b"x"
    assert host._huge_backed_bytes(a, a + (1 << 20)) >= 0
    assert host._huge_backed_bytes(8, 16) == 0
    del buf
    m.close()
    t = torch.zeros(1000)
    assert 0.0 <= host.huge_page_fraction(t) <= 1.0
    assert host.huge_page_fraction(torch.zeros(0)) == 1.0
