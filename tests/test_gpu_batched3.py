"""GPU parity of the batched 3D multi-target step against the 3D oracle run per target.

Each target is an independent 3D pcSIR filter (Algorithm 2 over (x, y, z, vx, vy, vz, I0)) with its
own particle count, cell edges, PSF and patch; the oracle runs ``pcsir3_oracle.pcsir_step`` on each
target's slice of the state and noise with that target's model.  Tolerances are the single-target
3D ones: propagated states, cells, counts bit-exact; dummy positions 1e-9 voxel, other components
2.5e-7; dummy log-likelihoods 1e-4 + 4e-7 |ll|; posterior mean and ESS relative 1e-5; every output
its ancestor's propagated state, the ancestors exactly the systematic resample of the target's own
integer weights (which meet the weight tolerance against the oracle's), and every ancestor in the
range the oracle's weights allow under that tolerance.
"""
import numpy as np
import pytest
import torch

import resample_checks as RC
from oracle import pcsir3_oracle as O3
from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = 1310555300
KEEP = 1 | 16  # ancestors, integer weights


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


def _model(batch, t):
    return O3.Model3(sigma_xy=float(batch.sigma_xy[t]), sigma_z=float(batch.sigma_z[t]), bg=float(batch.bg[t]),
                     patch_xy=int(batch.patch_xy[t]), patch_z=int(batch.patch_z[t]))


def _decode(keys):
    k = keys.astype(np.uint64)
    t = (k >> np.uint64(54)).astype(np.int64)
    ax = [((k >> np.uint64(18 * a)) & np.uint64(0x3FFFF)).astype(np.int64) - (1 << 17) for a in range(3)]
    return t, ax[0], ax[1], ax[2]


def _warm(batch, frames):
    st = synth.batch3_initial_state(batch)
    offs = np.concatenate([[0], np.cumsum(batch.n)])
    for k in range(frames):
        nz = synth.make_noise(int(batch.n.sum()), synth.Q3, SEED + 1, k, np.float32)
        u0 = synth.batch_u0(len(batch.n), SEED + 1, k)
        for t in range(len(batch.n)):
            sl = slice(offs[t], offs[t + 1])
            st[:, sl] = O3.pcsir_step(np.ascontiguousarray(st[:, sl]), batch.images[k], np.ascontiguousarray(nz[:, sl]),
                                      u0[t], tuple(batch.h[t]), _model(batch, t))["new_state"]
    return st


def _check_target(t, sl, st, nz, u0, vol, batch, prop, new, res, tk, bx, by, bz, cnt, dum, bll, anc, q):
    ref = O3.pcsir_step(np.ascontiguousarray(st[:, sl]), vol, np.ascontiguousarray(nz[:, sl]), u0, tuple(batch.h[t]),
                        _model(batch, t))
    np.testing.assert_array_equal(prop[:, sl], ref["prop"])
    sel = tk == t
    order = np.lexsort((bx[sel], by[sel], bz[sel]))
    np.testing.assert_array_equal(np.stack([bx[sel][order], by[sel][order], bz[sel][order]], 1), ref["bin_keys"])
    np.testing.assert_array_equal(cnt[sel][order], ref["bin_counts"])
    assert res[t]["n_bins"] == ref["bin_keys"].shape[0]
    d = dum[:, sel][:, order]
    np.testing.assert_allclose(d[:3], ref["dummies"][:3], rtol=0, atol=1e-9)
    np.testing.assert_allclose(d[3:], ref["dummies"][3:], rtol=0, atol=2.5e-7)
    ll = bll[sel][order]
    assert np.all(np.abs(ll - ref["ll_bins"]) <= 1e-4 + 4e-7 * np.abs(ref["ll_bins"]))
    est = np.array(res[t]["estimate"])
    assert np.all(np.abs(est - ref["estimate"]) <= 1e-5 * np.abs(ref["estimate"]) + 1e-6), (t, est, ref["estimate"])
    assert abs(res[t]["ess"] - ref["ess"]) <= 1e-5 * ref["ess"]
    a, qt = anc[sl], q[sl]
    np.testing.assert_array_equal(new[:, sl], prop[:, sl][:, a])
    RC.exact_systematic(a, qt, u0)
    w = qt.astype(np.float64) / float(qt.sum())
    sig = ref["w"] >= 1e-3 * ref["w"].max()
    assert (np.abs(w[sig] - ref["w"][sig]) / ref["w"][sig]).max() <= 1e-5
    assert np.abs(w[~sig] - ref["w"][~sig]).max(initial=0.0) <= 1e-5 * ref["w"].max()
    open_band, _ = RC.oracle_band(a, ref["w"], u0, RC.weight_tolerance(ref["w"]))
    mism = int(np.sum(a != ref["ancestors"]))
    assert mism <= open_band
    return mism


def _run(pc, batch, st, frame, seed, targets=None):
    T = len(batch.n)
    offs = np.concatenate([[0], np.cumsum(batch.n)])
    nz = synth.make_noise(int(batch.n.sum()), synth.Q3, seed, frame, np.float32)
    u0 = synth.batch_u0(T, seed, frame)
    bt = pc.Batch3(batch.n, batch.h, batch.sigma_xy, batch.sigma_z, batch.bg, batch.patch_xy, batch.patch_z, keep=KEEP)
    d_st = torch.from_numpy(np.ascontiguousarray(st)).cuda()
    vol = torch.from_numpy(batch.images[frame]).cuda()
    bt.step(d_st, vol, torch.from_numpy(nz).cuda(), torch.from_numpy(u0).cuda())
    torch.cuda.synchronize()
    res, derr = bt.results()
    assert derr == 0, derr
    o = bt.outputs()
    h = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in o.items()}
    bt.close()
    new = d_st.cpu().numpy()
    tk, bx, by, bz = _decode(h["bin_key"])
    mism = 0
    for t in (range(T) if targets is None else targets):
        sl = slice(offs[t], offs[t + 1])
        mism += _check_target(t, sl, st, nz, u0[t], batch.images[frame], batch, h["prop_state"], new, res, tk, bx, by,
                              bz, h["bin_count"], h["dummy"], h["bin_loglik"], h["ancestor"], h["qweight"])
    return mism, h, new, nz, u0, offs


def test_batched3_matches_per_target_oracle(pc):
    n = [1, 4095, 4097, 20000, 777]
    batch = synth.make_batch3(len(n), 96, 80, 32, 3, SEED, n_values=n, min_sep=14.0)
    batch.h[:] = [(0.5, 0.5, 1.0), (0.25, 0.25, 0.5), (1.0, 1.0, 2.0), (0.5, 0.5, 1.0), (2.0, 2.0, 2.0)]
    batch.patch_xy[:] = [11, 9, 11, 13, 7]
    batch.patch_z[:] = [7, 5, 7, 9, 3]
    batch.sigma_xy[:] = [1.5, 1.2, 1.8, 1.5, 1.5]
    batch.sigma_z[:] = [3.0, 2.5, 3.0, 3.5, 3.0]
    st = _warm(batch, 2)
    mism, *_ = _run(pc, batch, st, 2, SEED + 2)
    print("batched 3D: ancestors differing from the oracle's: %d of %d" % (mism, int(batch.n.sum())))


def test_batched3_full_size_workload_sampled(pc):
    """The 3D multi-target workload at its full size: 200 targets x 200,000 particles in 256 x 256 x 64
    volumes, 11 x 11 x 7 patches, 0.5 x 0.5 x 1 voxel cells.  Propagated states of every particle
    bit-exact; eight sampled targets against the oracle on their own slices; every target's
    resampling exactly systematic over its own integer weights."""
    batch = synth.make_batch3(200, 256, 256, 64, 1, SEED + 10)
    st = synth.batch3_initial_state(batch)
    sample = sorted(set(np.random.default_rng(SEED + 11).choice(200, 8, replace=False).tolist()) | {0, 199})
    mism, h, new, nz, u0, offs = _run(pc, batch, st, 0, SEED + 12, targets=sample)
    np.testing.assert_array_equal(h["prop_state"], O3.propagate(st, nz))
    for t in range(len(batch.n)):
        sl = slice(offs[t], offs[t + 1])
        np.testing.assert_array_equal(new[:, sl], h["prop_state"][:, sl][:, h["ancestor"][sl]])
        RC.exact_systematic(h["ancestor"][sl], h["qweight"][sl], u0[t])
    print("batched 3D full size: %d particles, %d sampled targets, ancestors differing %d" %
          (int(batch.n.sum()), len(sample), mism))


def test_batched3_graph_replay_equals_direct_step(pc):
    n = [5000, 3000, 123]
    batch = synth.make_batch3(len(n), 64, 64, 24, 1, SEED + 20, n_values=n, min_sep=12.0, margin_xy=8.0)
    st0 = torch.from_numpy(synth.batch3_initial_state(batch)).cuda()
    nz = torch.from_numpy(synth.make_noise(int(sum(n)), synth.Q3, SEED, 0, np.float32)).cuda()
    u0 = torch.from_numpy(synth.batch_u0(3, SEED, 0)).cuda()
    vol = torch.from_numpy(batch.images[0]).cuda()
    bt = pc.Batch3(batch.n, batch.h, batch.sigma_xy, batch.sigma_z, batch.bg, batch.patch_xy, batch.patch_z)
    s = torch.cuda.Stream()
    st = st0.clone()
    with torch.cuda.stream(s):
        bt.step(st, vol, nz, u0, stream=s)
    torch.cuda.synchronize()
    ref = st.clone()
    st.copy_(st0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bt.step(st, vol, nz, u0, stream=s)
    st.copy_(st0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(st, ref)
    bt.close()
