"""GPU parity of 3D pcSIR / SIR against the 3D oracle (7-D state, 3D cells, anisotropic PSF).

Same tolerances as the 2D parity tests: propagated states, cells, counts and the member -> cell map
bit-exact; dummy positions 1e-9 voxel, other components 2.5e-7; log-likelihoods 1e-4 + 4e-7 |ll|;
significant weights relative 1e-5; estimates relative 1e-5; every resampled particle is its reported
ancestor's propagated state, the ancestors are exactly the systematic resample of the step's own
integer weights (which meet the weight tolerance against the oracle's), and every ancestor lies in
the range the oracle's weights allow under that tolerance; ancestors that differ from the oracle's
are counted and can only be where that range holds more than one particle.
"""
import numpy as np
import pytest
import torch

import resample_checks as RC
from oracle import pcsir3_oracle as O3
from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = 1310554700
KEEP_ALL = 1 | 2 | 4 | 8 | 16


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


@pytest.fixture(scope="module")
def case():
    seq = synth.make_sequence3(64, 56, 24, 3, seed=SEED)
    m = O3.Model3()
    N = 40_000 + 77
    st = synth.initial_state3(seq.gt[0], N, np.float32)
    for k in range(2):  # a realistic cloud: two oracle steps
        nz = synth.make_noise(N, synth.Q3, SEED + 1, k, np.float32)
        st = O3.pcsir_step(st, seq.images[k], nz, synth.make_u0(SEED + 1, k), (0.5, 0.5, 1.0), m)["new_state"]
    return seq, m, N, st


def _check_weights(w, ref):
    sig = ref >= 1e-3 * ref.max()
    assert (np.abs(w[sig] - ref[sig]) / ref[sig]).max() <= 1e-5
    assert np.abs(w[~sig] - ref[~sig]).max(initial=0.0) <= 1e-5 * ref.max()


def _check_scalars(res, ref):
    est = np.array(res["estimate"])
    assert np.all(np.abs(est - ref["estimate"]) <= 1e-5 * np.abs(ref["estimate"]) + 1e-6), (est, ref["estimate"])
    assert abs(res["ess"] - ref["ess"]) <= 1e-5 * ref["ess"]


def _check_resampled(new, prop, anc, q, u0, ref_w, ref_anc):
    np.testing.assert_array_equal(new, prop[:, anc])
    RC.exact_systematic(anc, q, u0)
    _check_weights(q.astype(np.float64) / float(q.sum()), ref_w)
    open_band, _ = RC.oracle_band(anc, ref_w, u0, RC.weight_tolerance(ref_w))
    mism = int(np.sum(anc != ref_anc))
    assert mism <= open_band
    return mism


@pytest.mark.parametrize("h", [(0.5, 0.5, 1.0), (1.0, 1.0, 2.0), (0.25, 0.25, 0.5)])
def test_pcsir3_matches_oracle(pc, case, h):
    seq, m, N, st = case
    nz = synth.make_noise(N, synth.Q3, SEED + 2, 2, np.float32)
    u0 = synth.make_u0(SEED + 2, 2)
    ref = O3.pcsir_step(st, seq.images[2], nz, u0, h, m)
    ctx = pc.Context3(N, keep=KEEP_ALL)
    d = torch.from_numpy(np.ascontiguousarray(st)).cuda()
    ctx.step(d, torch.from_numpy(seq.images[2]).cuda(), h, torch.from_numpy(nz).cuda(), u0)
    torch.cuda.synchronize()
    res = ctx.last_result()
    out = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in ctx.outputs().items()}
    assert res["device_error"] == 0 and res["kind"] == 1
    np.testing.assert_array_equal(out["prop_state"], ref["prop"])
    B = res["n_bins"]
    assert B == ref["bin_keys"].shape[0]
    xyz = out["bin_xyz"]
    order = np.lexsort((xyz[0], xyz[1], xyz[2]))
    np.testing.assert_array_equal(xyz[:, order].T, ref["bin_keys"])
    np.testing.assert_array_equal(out["bin_count"][order], ref["bin_counts"])
    rank = np.empty(B, np.int64)
    rank[order] = np.arange(B)
    np.testing.assert_array_equal(rank[out["particle_bin"]], ref["member_bin"])
    dum = out["dummy"][:, order]
    np.testing.assert_allclose(dum[:3], ref["dummies"][:3], rtol=0, atol=1e-9)
    np.testing.assert_allclose(dum[3:], ref["dummies"][3:], rtol=0, atol=2.5e-7)
    ll = out["bin_loglik"][order]
    assert np.all(np.abs(ll - ref["ll_bins"]) <= 1e-4 + 4e-7 * np.abs(ref["ll_bins"]))
    _check_weights(out["weight"], ref["w"])
    _check_scalars(res, ref)
    mism = _check_resampled(d.cpu().numpy(), out["prop_state"], out["ancestor"], out["qweight"], u0, ref["w"],
                            ref["ancestors"])
    print("3D pcSIR h=%s: B=%d, ancestors differing %d of %d" % (h, B, mism, N))
    ctx.close()


def test_sir3_matches_oracle(pc, case):
    seq, m, N, st = case
    n = 5000 + 3
    st = np.ascontiguousarray(st[:, :n])
    nz = synth.make_noise(n, synth.Q3, SEED + 3, 2, np.float32)
    u0 = synth.make_u0(SEED + 3, 2)
    ref = O3.sir_step(st, seq.images[2], nz, u0, m)
    ctx = pc.Context3(n, keep=1 | 2 | 8 | 16)
    d = torch.from_numpy(st).cuda()
    ctx.sir_step(d, torch.from_numpy(seq.images[2]).cuda(), torch.from_numpy(nz).cuda(), u0)
    torch.cuda.synchronize()
    res = ctx.last_result()
    out = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in ctx.outputs().items()}
    assert res["device_error"] == 0 and res["kind"] == 0
    np.testing.assert_array_equal(out["prop_state"], ref["prop"])
    assert np.all(np.abs(out["loglik"] - ref["ll"]) <= 1e-4 + 4e-7 * np.abs(ref["ll"]))
    _check_weights(out["weight"], ref["w"])
    _check_scalars(res, ref)
    mism = _check_resampled(d.cpu().numpy(), out["prop_state"], out["ancestor"], out["qweight"], u0, ref["w"],
                            ref["ancestors"])
    print("3D SIR: ancestors differing %d of %d" % (mism, n))
    ctx.close()


def test_one_particle_per_cell_is_sir_on_gpu(pc, case):
    """Section 4.2 in 3D on the GPU: with tiny cells the dummies are the particles and the
    log-likelihoods equal SIR's bit for bit."""
    seq, m, N, st = case
    n = 3000
    st = np.ascontiguousarray(st[:, :n]) + np.random.default_rng(4).normal(size=(7, n)).astype(np.float32) * 0.01
    nz = torch.from_numpy(synth.make_noise(n, synth.Q3, SEED + 4, 2, np.float32)).cuda()
    vol = torch.from_numpy(seq.images[2]).cuda()
    a = pc.Context3(n, keep=1 | 2 | 8)
    b = pc.Context3(n, keep=1 | 2 | 4)
    da = torch.from_numpy(st).cuda()
    db = torch.from_numpy(st).cuda()
    a.sir_step(da, vol, nz, 0.4)
    # cell indices are limited to |b| < 2^20 per axis: 1e-4 voxel cells still hold one particle each here
    b.step(db, vol, (1e-4, 1e-4, 1e-4), nz, 0.4)
    torch.cuda.synchronize()
    ra, rb = a.last_result(), b.last_result()
    assert ra["device_error"] == 0 and rb["device_error"] == 0
    oa, ob = a.outputs(), b.outputs()
    assert rb["n_bins"] == n and np.all(ob["bin_count"].cpu().numpy() == 1)
    ll_p = ob["bin_loglik"].cpu().numpy()[ob["particle_bin"].cpu().numpy()]
    np.testing.assert_array_equal(ll_p, oa["loglik"].cpu().numpy())
    wp = ob["weight"].cpu().numpy()
    np.testing.assert_allclose(wp, oa["weight"].cpu().numpy(), rtol=1e-6, atol=1e-12 * wp.max())
    np.testing.assert_allclose(rb["estimate"], ra["estimate"], rtol=1e-6)
    a.close()
    b.close()


def test_cell_index_range_is_flagged(pc, case):
    """Cells finer than the 21-bit key allows raise the range flag instead of aliasing."""
    seq, m, N, st = case
    n = 1000
    st = np.ascontiguousarray(st[:, :n])
    nz = torch.from_numpy(np.zeros((7, n), np.float32)).cuda()
    ctx = pc.Context3(n)
    d = torch.from_numpy(st).cuda()
    ctx.step(d, torch.from_numpy(seq.images[2]).cuda(), (1e-6, 1e-6, 1e-6), nz, 0.4)
    torch.cuda.synchronize()
    assert ctx.last_result()["device_error"] & pc.DERR_RANGE
    # the context stays usable
    ctx.step(d, torch.from_numpy(seq.images[2]).cuda(), (0.5, 0.5, 1.0), nz, 0.4)
    torch.cuda.synchronize()
    assert ctx.last_result()["device_error"] == 0
    ctx.close()


@pytest.mark.parametrize("comp,value", [(6, np.nan), (5, np.inf), (3, -2.0e9), (4, -5000.0)])
def test_out_of_range_component_is_flagged(pc, case, comp, value):
    """A 3D state component that is not finite, of magnitude 10^9 or more, or (velocities and
    intensity) 2^12 or more below particle 0's value raises the range flag; the context stays
    usable."""
    seq, m, N, st = case
    n = 3000
    st = np.ascontiguousarray(st[:, :n]).copy()
    st[comp, 2000] = np.float32(value)
    nz = torch.from_numpy(np.zeros((7, n), np.float32)).cuda()
    ctx = pc.Context3(n)
    d = torch.from_numpy(st).cuda()
    ctx.step(d, torch.from_numpy(seq.images[2]).cuda(), (0.5, 0.5, 1.0), nz, 0.4)
    torch.cuda.synchronize()
    assert ctx.last_result()["device_error"] & pc.DERR_RANGE, (comp, value)
    st[comp, 2000] = st[comp, 1999]
    d = torch.from_numpy(st).cuda()
    ctx.step(d, torch.from_numpy(seq.images[2]).cuda(), (0.5, 0.5, 1.0), nz, 0.4)
    torch.cuda.synchronize()
    assert ctx.last_result()["device_error"] == 0
    ctx.close()
