"""GPU parity of the steps whose process noise is drawn in the propagation kernel (pcsir_step_philox,
pcsir_deferred_step_philox) against the oracle fed with the noise oracle's increments.

The noise oracle (oracle/noise_oracle.py) implements the same counter-based generator and transform
from their definitions with correctly rounded single-precision operations, so the propagated states
must equal the oracle's bit for bit; the rest of the step is the plain pcSIR step's parity
(cells and counts exact, dummies, log-likelihoods, weights and results within the tolerances of
tests/test_gpu_parity.py), and a drawn-noise step equals pcsir_step given the oracle's noise array.
"""
import numpy as np
import pytest
import torch

import resample_checks as RC
from oracle import noise_oracle as NO
from oracle import pcsir_oracle as O
from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = 1310551900
Q = (0.5, 0.5, 0.1, 0.1, 1.0)
KEEP = 1 | 2 | 16


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


@pytest.mark.parametrize("N,h", [(4096 * 3 + 77, 0.5), (1 << 18, 0.25), (1, 0.5)])
def test_drawn_noise_step_matches_oracle(pc, N, h):
    model = synth.Model(patch=21)
    seq = synth.make_sequence(128, 128, 3, model, SEED + N)
    st0 = synth.initial_state(seq.gt[0], N, np.float32)
    ctx = pc.Context(N, torch.float32, patch=21, psf_sigma=model.sigma_psf, bg=model.bg, keep=KEEP)
    st = torch.from_numpy(st0).cuda()
    seed, frame, u0 = 0x1234_5678_9ABC_DEF0 + N, 7, 0.4375
    pc.pcsir_step_philox(ctx, st, torch.from_numpy(seq.images[0]).cuda(), h, Q, seed, frame, u0)
    torch.cuda.synchronize()
    out = ctx.outputs()
    noise = NO.process_noise(N, Q, seed, frame)
    ref = O.pcsir_step(st0, seq.images[0], noise, u0, h, model)
    np.testing.assert_array_equal(out["prop_state"].cpu().numpy(), ref["prop"])
    B = out["n_bins"]
    xy = out["bin_xy"].cpu().numpy()
    order = np.lexsort((xy[0], xy[1]))
    np.testing.assert_array_equal(xy[:, order].T, ref["bin_keys"])
    np.testing.assert_array_equal(out["bin_count"].cpu().numpy()[order], ref["bin_counts"])
    ll = out["bin_loglik"].cpu().numpy()[order]
    assert np.all(np.abs(ll - ref["ll_bins"]) <= 1e-4 + 4e-7 * np.abs(ref["ll_bins"]))
    q = out["qweight"].cpu().numpy()
    anc = out["ancestor"].cpu().numpy()
    RC.exact_systematic(anc, q, u0)
    open_band, _ = RC.oracle_band(anc, ref["w"], u0, RC.weight_tolerance(ref["w"]))
    assert int(np.sum(anc != ref["ancestors"])) <= open_band
    np.testing.assert_array_equal(st.cpu().numpy(), ref["prop"][:, anc])
    r = ctx.last_result()
    assert r["device_error"] == 0 and r["n_bins"] == B
    np.testing.assert_allclose(r["estimate"], ref["estimate"], rtol=1e-5, atol=1e-6)
    ctx.close()


def test_drawn_noise_equals_the_array_step_and_the_deferred_run(pc):
    """Five frames three ways on the same context size: pcsir_step with the oracle's noise arrays,
    pcsir_step_philox, and a deferred run with drawn noise: identical states, weights and ancestors."""
    N = (1 << 20) + 4
    model = synth.Model(patch=21)
    seq = synth.make_sequence(256, 256, 5, model, SEED + 3)
    st0 = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).cuda()
    ctxs = [pc.Context(N, torch.float32, patch=21, psf_sigma=model.sigma_psf, bg=model.bg, keep=KEEP)
            for _ in range(3)]
    sa, sb = st0.clone(), st0.clone()
    pc.pcsir_deferred_begin(ctxs[2], st0)
    out = torch.empty_like(st0)
    seed = 987654321
    for k in range(5):
        img = torch.from_numpy(seq.images[k]).cuda()
        u0 = synth.make_u0(SEED, k)
        pc.pcsir_step(ctxs[0], sa, img, 0.5, torch.from_numpy(NO.process_noise(N, Q, seed, k)).cuda(), u0)
        pc.pcsir_step_philox(ctxs[1], sb, img, 0.5, Q, seed, k, u0)
        pc.pcsir_deferred_step_philox(ctxs[2], img, 0.5, Q, seed, k, u0)
        pc.pcsir_deferred_state(ctxs[2], out)
        torch.cuda.synchronize()
        o = [c.outputs() for c in ctxs]
        for x in o[1:]:
            assert torch.equal(x["prop_state"], o[0]["prop_state"]), k
            assert torch.equal(x["qweight"], o[0]["qweight"]), k
            assert torch.equal(x["ancestor"], o[0]["ancestor"]), k
        assert torch.equal(sa, sb) and torch.equal(sa, out), k
    for c in ctxs:
        c.close()


def test_drawn_noise_arguments_are_checked(pc):
    ctx = pc.Context(100, torch.float32)
    st = torch.zeros((5, 100), dtype=torch.float32, device="cuda")
    img = torch.ones((16, 16), dtype=torch.float32, device="cuda")
    for q, frame in (((0.5, 0.5, 0.1, 0.1, -1.0), 0), ((0.5, 0.5, 0.1, 0.1, float("nan")), 0), (Q, 1 << 32)):
        with pytest.raises(pc.PcsirError) as e:
            pc.pcsir_step_philox(ctx, st, img, 0.5, q, 1, frame, 0.5)
        assert e.value.status == pc.EINVAL
    ctx.close()
    ctx64 = pc.Context(100, torch.float64)
    with pytest.raises(pc.PcsirError) as e:
        pc.pcsir_step_philox(ctx64, st.double(), img, 0.5, Q, 1, 0, 0.5)
    assert e.value.status == pc.ENOTSUP
    ctx64.close()
