"""Systematic resampling when the weight sits in a few particles of one tile.

The resampling kernel gives each tile of 4096 particles the outputs whose U_i fall inside the
tile's share of the cumulative weight (Sec. 2, the resampling step of Algorithms 1 and 2).  When
one particle carries all the weight, one tile owns all N outputs; those past its first chunk are
written by extra blocks.  These cases check that every output is still the systematic resample of
the weights, exactly: the ancestors are compared with the plain definition s(i) = the first j with
C_j > (i + u0) T / N over integer weights in the same ratios as the GPU's.
"""
import numpy as np
import pytest
import torch

import resample_checks as RC

pytestmark = pytest.mark.gpu

N_CASES = [4096 * 5 + 17, (1 << 20) + 123, 1 << 22]


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


@pytest.mark.parametrize("N", N_CASES)
def test_one_particle_carries_all_the_weight(pc, N):
    rng = np.random.default_rng(N)
    ctx = pc.Context(N, torch.float32)
    for k in (0, N // 2 + 5, N - 1):
        lw = torch.full((N,), -np.inf, dtype=torch.float64, device="cuda")
        lw[k] = float(rng.normal() * 50.0)
        for entry in ("context", "noalloc"):
            if entry == "context":
                anc = pc.pcsir_resample(ctx, lw, float(rng.random()))
            else:
                anc = pc.pcsir_resample_noalloc(lw, float(rng.random()))
            torch.cuda.synchronize()
            assert torch.all(anc == k), (entry, k, int((anc != k).sum()))
    ctx.close()


@pytest.mark.parametrize("N", N_CASES)
def test_weight_in_a_few_particles_of_one_tile(pc, N):
    """Weights 1 : 2 : 1 on three particles of one tile (log-weights log 1/2, 0, log 1/2; the
    kernel's integer weights keep those ratios within its 2^-32 log-weight quantum, far inside the
    check's band), then the same with a fourth particle in the next tile; the ancestors are the
    systematic resample of those ratios."""
    rng = np.random.default_rng(N + 1)
    ctx = pc.Context(N, torch.float32)
    base = (N // 2) // 4096 * 4096
    sets = [{base + 3: 1, base + 10: 2, base + 4000: 1}]
    if base + 4096 + 7 < N:
        sets.append({base + 3: 1, base + 10: 2, base + 4000: 1, base + 4096 + 7: 4})
    for ratios in sets:
        top = max(ratios.values())
        lw = torch.full((N,), -np.inf, dtype=torch.float64, device="cuda")
        q = np.zeros(N, np.int64)
        for j, r in ratios.items():
            lw[j] = float(np.log(r / top))
            q[j] = r << 40
        for call in range(2):
            u0 = float(rng.random())
            anc = pc.pcsir_resample(ctx, lw, u0).cpu().numpy()
            RC.exact_systematic(anc, q, u0)
            counts = np.bincount(anc, minlength=N)
            for j, r in ratios.items():
                share = N * r / sum(ratios.values())
                assert abs(counts[j] - share) < 1.0
    ctx.close()


def test_no_weight_at_all_keeps_every_particle_at_full_size(pc):
    """Every log-weight -inf over a million particles: the last tile owns all outputs, which the
    extra blocks write as the identity."""
    N = (1 << 20) + 123
    ctx = pc.Context(N, torch.float32)
    lw = torch.full((N,), -np.inf, dtype=torch.float64, device="cuda")
    ident = torch.arange(N, dtype=torch.int32, device="cuda")
    assert torch.equal(pc.pcsir_resample(ctx, lw, 0.3), ident)
    assert torch.equal(pc.pcsir_resample_noalloc(lw, 0.3), ident)
    ctx.close()
