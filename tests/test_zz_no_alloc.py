"""The allocation-free resampling entry point against the context-based one.

pcsir_resample_noalloc serves callers that cannot allocate device memory (a
fixed device-memory budget owned by the host application, another framework's
caching allocator holding the free memory, or a real-time loop that cannot
afford the synchronisation an allocation may cause).  Its scratch lives in a
fixed array inside the library, so it must give exactly the ancestors that
pcsir_resample computes with a context's workspace, call after call.  This
file is collected last, so a run that stops at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


def _noalloc(pc, logw, u0):
    fn = ctypes.CDLL(pc.LIB_PATH).pcsir_resample_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    out = torch.full((logw.numel(),), -1, dtype=torch.int32, device="cuda")
    st = fn(ctypes.c_void_p(logw.data_ptr()), logw.numel(), float(u0), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_noalloc_resample_matches_context_resample_on_consecutive_calls(pc):
    rng = np.random.default_rng(20261203)
    N = 1_000_003
    ctx = pc.Context(N, torch.float32)
    for call in range(2):
        lw = torch.from_numpy(rng.normal(size=N) * (1.0 + call)).cuda()
        u0 = float(rng.random())
        st, anc = _noalloc(pc, lw, u0)
        assert st == pc.OK
        ref = pc.pcsir_resample(ctx, lw, u0)
        torch.cuda.synchronize()
        assert torch.equal(anc, ref), "call %d: %d ancestors differ" % (call, int((anc != ref).sum()))
    ctx.close()


def test_noalloc_resample_rejects_sizes_beyond_its_limit(pc):
    lw = torch.zeros(16, dtype=torch.float64, device="cuda")
    fn = ctypes.CDLL(pc.LIB_PATH).pcsir_resample_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    assert fn(ctypes.c_void_p(lw.data_ptr()), (1 << 22) + 1, 0.5, ctypes.c_void_p(lw.data_ptr()), None) == pc.ERANGE
