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


@pytest.mark.parametrize("N", [1, 4097, 1 << 22])
def test_noalloc_resample_at_the_edges_of_its_range(pc, N):
    """N = 1, a ragged tile, and exactly the limit 2^22 (every entry of the scratch's tile table in
    use): the same ancestors as the context-based entry point, on two consecutive calls."""
    rng = np.random.default_rng(N)
    ctx = pc.Context(N, torch.float32)
    for call in range(2):
        lw = torch.from_numpy(rng.normal(size=N) * 3.0).cuda()
        u0 = float(rng.random())
        st, anc = _noalloc(pc, lw, u0)
        assert st == pc.OK
        ref = pc.pcsir_resample(ctx, lw, u0)
        torch.cuda.synchronize()
        assert torch.equal(anc, ref), "N=%d call %d: %d ancestors differ" % (N, call, int((anc != ref).sum()))
    ctx.close()


def test_noalloc_resample_without_positive_weight_keeps_every_particle(pc):
    """Every log-weight -inf (or NaN): nothing to sample; both entry points return the identity."""
    N = 10_000
    ctx = pc.Context(N, torch.float32)
    for fill in (-np.inf, np.nan):
        lw = torch.full((N,), fill, dtype=torch.float64, device="cuda")
        st, anc = _noalloc(pc, lw, 0.25)
        assert st == pc.OK
        ref = pc.pcsir_resample(ctx, lw, 0.25)
        torch.cuda.synchronize()
        ident = torch.arange(N, dtype=torch.int32, device="cuda")
        assert torch.equal(anc, ident) and torch.equal(ref, ident)
    # and a normal call afterwards is unaffected by the scratch the zero-sum call left behind
    lw = torch.from_numpy(np.random.default_rng(5).normal(size=N)).cuda()
    st, anc = _noalloc(pc, lw, 0.5)
    assert st == pc.OK and torch.equal(anc, pc.pcsir_resample(ctx, lw, 0.5))
    ctx.close()


def test_noalloc_resample_rejects_sizes_beyond_its_limit(pc):
    lw = torch.zeros(16, dtype=torch.float64, device="cuda")
    fn = ctypes.CDLL(pc.LIB_PATH).pcsir_resample_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    assert fn(ctypes.c_void_p(lw.data_ptr()), (1 << 22) + 1, 0.5, ctypes.c_void_p(lw.data_ptr()), None) == pc.ERANGE
