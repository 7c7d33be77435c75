"""On the GPU, the integer-pipe binary64 multiplication (the kernels' dmul)
gives the hardware product bit for bit: the multiplication-chain loop of
libeig3_peaks.so run with dmul (kind 8) and with the FP64 pipe's DMUL (kind 1)
from the same starting values, over every chain count, must leave identical
results.  (The host build of the same header is checked against the host's
IEEE multiplication, special cases included, in tests/test_dmul.py.)"""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chains", [2, 4, 8, 16])
def test_integer_pipe_products_equal_the_fp64_pipe(chains):
    from paper_2511_00292_gb300 import build as _b
    _b.build()
    lib = ctypes.CDLL(_b.PEAKS_LIB)
    lib.eig3_peak_loop.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p, ctypes.c_void_p]
    lib.eig3_peak_loop.restype = ctypes.c_int
    dev = torch.device("cuda", 0)
    blocks, threads, iters = 2 * torch.cuda.get_device_properties(dev).multi_processor_count, \
        256, 1000
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    out = {}
    for kind in (1, 8):
        o = torch.full((blocks * threads,), float("nan"), dtype=torch.float64, device=dev)
        st = lib.eig3_peak_loop(kind, chains, blocks, threads, iters,
                                ctypes.c_void_p(o.data_ptr()), stream)
        assert st == 0
        torch.cuda.synchronize(dev)
        out[kind] = o
    assert torch.isfinite(out[1]).all()
    assert torch.equal(out[1], out[8])
