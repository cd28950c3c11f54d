"""Deferred resampling against the plain pcSIR step.

A deferred run (pcsir_deferred_begin / _step / _state) keeps the particle set in the context and
records each resampling as ancestors only; the next step's propagation reads x~_k^{a(i)} itself
(Algorithm 2: the resampled particle i is the propagated particle a(i)).  On the same inputs every
step must give what pcsir_step gives: propagated states, integer weights, ancestors and the resampled
states bit for bit, cells and dummies equal up to the order of the cells, and the normalised weights
and the step's results within the rounding of an FP64 sum taken in another order.
"""
import numpy as np
import pytest
import torch

from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = 1310550700
KEEP = 1 | 2 | 16  # ancestors, weights, integer weights


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


def _cells(o):
    B = o["n_bins"]
    xy = o["bin_xy"].cpu().numpy()
    order = np.lexsort((xy[0], xy[1]))
    return (xy[:, order], o["bin_count"].cpu().numpy()[order], o["dummy"].cpu().numpy()[:, order],
            o["bin_loglik"].cpu().numpy()[order], B)


@pytest.mark.parametrize("N,h,dtype", [(4096 * 5 + 123, 0.5, torch.float32), (1 << 20, 0.5, torch.float32),
                                       (1 << 20, 0.1, torch.float32), (30001, 0.3, torch.float64)])
def test_deferred_run_equals_plain_steps(pc, N, h, dtype):
    model = synth.Model()
    seq = synth.make_sequence(256, 256, 6, model, SEED + N)
    npdt = np.float32 if dtype == torch.float32 else np.float64
    st0 = torch.from_numpy(synth.initial_state(seq.gt[0], N, npdt)).cuda()
    imgs = [torch.from_numpy(seq.images[k]).cuda() for k in range(6)]
    noise = [torch.from_numpy(synth.make_noise(N, model.q, SEED, k, npdt)).cuda() for k in range(6)]
    u0s = [synth.make_u0(SEED + 1, k) for k in range(6)]
    plain = pc.Context(N, dtype, patch=21, psf_sigma=model.sigma_psf, bg=model.bg, keep=KEEP)
    defer = pc.Context(N, dtype, patch=21, psf_sigma=model.sigma_psf, bg=model.bg, keep=KEEP)
    st = st0.clone()
    pc.pcsir_deferred_begin(defer, st0)
    out = torch.empty_like(st0)
    for k in range(6):
        pc.pcsir_step(plain, st, imgs[k], h, noise[k], u0s[k])
        pc.pcsir_deferred_step(defer, imgs[k], h, noise[k], u0s[k])
        pc.pcsir_deferred_state(defer, out)
        torch.cuda.synchronize()
        a, b = plain.outputs(), defer.outputs()
        assert torch.equal(a["prop_state"], b["prop_state"]), k
        assert torch.equal(a["qweight"], b["qweight"]), k
        # normalised by the step's total weight, an FP64 sum whose order the atomics decide
        assert torch.allclose(a["weight"], b["weight"], rtol=1e-13, atol=0.0), k
        assert torch.equal(a["ancestor"], b["ancestor"]), k
        assert torch.equal(st, out), k
        ca, cb = _cells(a), _cells(b)
        assert ca[4] == cb[4]
        for x, y in zip(ca[:4], cb[:4]):
            np.testing.assert_array_equal(x, y)
        ra, rb = plain.last_result(), defer.last_result()
        np.testing.assert_allclose(rb["estimate"], ra["estimate"], rtol=1e-12, atol=1e-12)
        assert abs(rb["ess"] - ra["ess"]) <= 1e-12 * ra["ess"]
        assert rb["device_error"] == 0 and rb["n_bins"] == ra["n_bins"]
    plain.close()
    defer.close()


def test_a_plain_step_ends_the_run(pc):
    N = 5000
    model = synth.Model()
    seq = synth.make_sequence(128, 128, 2, model, SEED)
    ctx = pc.Context(N, torch.float32, patch=21, psf_sigma=model.sigma_psf, bg=model.bg)
    st = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).cuda()
    img = torch.from_numpy(seq.images[0]).cuda()
    nz = torch.from_numpy(synth.make_noise(N, model.q, SEED, 0, np.float32)).cuda()
    with pytest.raises(pc.PcsirError) as e:
        pc.pcsir_deferred_step(ctx, img, 0.5, nz, 0.5)
    assert e.value.status == pc.ESTATE
    pc.pcsir_deferred_begin(ctx, st)
    pc.pcsir_deferred_step(ctx, img, 0.5, nz, 0.5)
    pc.pcsir_step(ctx, st, img, 0.5, nz, 0.5)
    with pytest.raises(pc.PcsirError) as e:
        pc.pcsir_deferred_step(ctx, img, 0.5, nz, 0.5)
    assert e.value.status == pc.ESTATE
    with pytest.raises(pc.PcsirError) as e:
        pc.pcsir_deferred_state(ctx, st)
    assert e.value.status == pc.ESTATE
    ctx.close()
