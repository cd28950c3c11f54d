"""GPU parity of the batched multi-target step against the oracle run per target.

Each target is an independent pcSIR filter (Algorithm 2) with its own particle
count, PSF, patch and cell edge; the oracle runs ``pcsir_step`` on each
target's slice of the state and noise with that target's model.  Tolerances
are those of the single-target parity tests: propagated states and cells
(with member counts) bit-exact, posterior means and ESS relative 1e-5, every
resampled particle its reported ancestor's propagated state within its own
target, the ancestors exactly the systematic resample of the target's own
integer weights (which meet the weight tolerance against the oracle's), and
every ancestor in the range the oracle's weights allow under that tolerance.
The number of outputs that differ from the oracle's is reported; they can
only be where that range holds more than one particle.
"""
import numpy as np
import pytest
import torch

import resample_checks as RC
from oracle import pcsir_oracle as O
from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = 1310554300


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


def _model(batch, t):
    return synth.Model(sigma_psf=float(batch.sigma[t]), I0=float(batch.i0[t]), bg=batch.bg,
                       patch=int(batch.patch[t]))


def _warm(batch, frames):
    """Per-target oracle runs for a few frames: realistic clouds for every target."""
    st = synth.batch_initial_state(batch, np.float32)
    offs = np.concatenate([[0], np.cumsum(batch.n)])
    for k in range(frames):
        nz = synth.batch_noise(batch, (0.5, 0.5, 0.1, 0.1, 1.0), SEED + 1, k)
        u0 = synth.batch_u0(len(batch.n), SEED + 1, k)
        for t in range(len(batch.n)):
            sl = slice(offs[t], offs[t + 1])
            r = O.pcsir_step(np.ascontiguousarray(st[:, sl]), batch.images[k], np.ascontiguousarray(nz[:, sl]),
                             u0[t], batch.h[t], _model(batch, t))
            st[:, sl] = r["new_state"]
    return st


def _decode(keys):
    k = keys.astype(np.uint64)
    t = (k >> np.uint64(52)).astype(np.int64)
    by = ((k >> np.uint64(26)) & np.uint64(0x3FFFFFF)).astype(np.int64) - (1 << 25)
    bx = (k & np.uint64(0x3FFFFFF)).astype(np.int64) - (1 << 25)
    return t, bx, by


def _check_weights(w, ref):
    sig = ref >= 1e-3 * ref.max()
    assert (np.abs(w[sig] - ref[sig]) / ref[sig]).max() <= 1e-5
    assert np.abs(w[~sig] - ref[~sig]).max(initial=0.0) <= 1e-5 * ref.max()


def _check_target_resampling(new_t, prop_t, anc_t, q_t, u0, ref):
    """One target's resampling: outputs are their ancestors' propagated states, the ancestors are the
    exact systematic resample of the target's integer weights, which meet the weight tolerance, and
    lie in the oracle's allowed range.  Returns the ancestors that differ from the oracle's."""
    np.testing.assert_array_equal(new_t, prop_t[:, anc_t])
    RC.exact_systematic(anc_t, q_t, u0)
    _check_weights(q_t.astype(np.float64) / float(q_t.sum()), ref["w"])
    open_band, _ = RC.oracle_band(anc_t, ref["w"], u0, RC.weight_tolerance(ref["w"]))
    mism = int(np.sum(anc_t != ref["ancestors"]))
    assert mism <= open_band
    return mism


def _compare(pc, batch, st, frame, noise_seed, bt=None):
    T = len(batch.n)
    offs = np.concatenate([[0], np.cumsum(batch.n)])
    nz = synth.batch_noise(batch, (0.5, 0.5, 0.1, 0.1, 1.0), noise_seed, frame)
    u0 = synth.batch_u0(T, noise_seed, frame)
    own = bt is None
    if own:
        bt = pc.Batch(batch.n, batch.h, batch.sigma, batch.bg, batch.patch)
    bt.keep(pc.KEEP_ANCESTORS | pc.KEEP_QWEIGHTS)
    d_st = torch.from_numpy(np.ascontiguousarray(st)).cuda()
    bt.step(d_st, torch.from_numpy(batch.images[frame]).cuda(), torch.from_numpy(nz).cuda(),
            torch.from_numpy(u0).cuda())
    torch.cuda.synchronize()
    res, derr = bt.results()
    assert derr == 0
    out = bt.outputs()
    prop = out["prop_state"].cpu().numpy()
    new = d_st.cpu().numpy()
    tk, bx, by = _decode(out["bin_key"].cpu().numpy())
    cnt = out["bin_count"].cpu().numpy()
    kept = bt.kept()
    anc = kept["ancestor"].cpu().numpy()
    q = kept["qweight"].cpu().numpy()
    mism_total = 0
    for t in range(T):
        sl = slice(offs[t], offs[t + 1])
        ref = O.pcsir_step(np.ascontiguousarray(st[:, sl]), batch.images[frame], np.ascontiguousarray(nz[:, sl]),
                           u0[t], batch.h[t], _model(batch, t))
        np.testing.assert_array_equal(prop[:, sl], ref["prop"])
        sel = tk == t
        order = np.lexsort((bx[sel], by[sel]))
        np.testing.assert_array_equal(np.stack([bx[sel][order], by[sel][order]], 1), ref["bin_keys"])
        np.testing.assert_array_equal(cnt[sel][order], ref["bin_counts"])
        assert res[t]["n_bins"] == ref["bin_keys"].shape[0]
        est = np.array(res[t]["estimate"])
        assert np.all(np.abs(est - ref["estimate"]) <= 1e-5 * np.abs(ref["estimate"]) + 1e-6), (t, est)
        assert abs(res[t]["ess"] - ref["ess"]) <= 1e-5 * ref["ess"]
        mism_total += _check_target_resampling(new[:, sl], prop[:, sl], anc[sl], q[sl], u0[t], ref)
    if own:
        bt.close()
    return mism_total


def test_batched_step_matches_per_target_oracle(pc):
    n = [1, 3000, 4096, 4097, 9000, 777, 20000]
    batch = synth.make_batch(len(n), 192, 160, 3, seed=SEED, n_values=n, min_sep=30.0,
                             h_of_sigma=None)
    batch.h[:] = [0.25, 0.5, 1.0, 0.5, 2.0, 0.5, 0.25]
    st = _warm(batch, 2)
    mism = _compare(pc, batch, st, 2, SEED + 2)
    print("batched: ancestors differing from the oracle's:", mism, "of", int(batch.n.sum()))


@pytest.mark.parametrize("patches", [[21, 9, 17, 25, 11, 13, 19], [41, 9, 21, 15, 33, 11, 13]])
def test_batched_likelihood_lane_groups(pc, patches):
    """Patches up to 15 pixels take 8 lanes per cell in the likelihood phase, up to 31 take 16, larger
    ones a warp: the same per-target parity with 16 lanes (largest 25) and with a warp (largest 41)."""
    n = [3000, 4096, 777, 9000, 2500, 20000, 1]
    batch = synth.make_batch(len(n), 224, 192, 3, seed=SEED + 40, n_values=n, min_sep=44.0, h_of_sigma=None)
    batch.patch[:] = patches
    batch.h[:] = [0.5, 0.25, 1.0, 0.5, 0.5, 0.25, 1.0]
    st = _warm(batch, 2)
    _compare(pc, batch, st, 2, SEED + 42)


def test_batched_many_small_targets(pc):
    rng = np.random.default_rng(4)
    n = list(rng.integers(50, 3000, 40))
    batch = synth.make_batch(len(n), 320, 320, 2, seed=SEED + 10, n_values=n, min_sep=24.0)
    st = synth.batch_initial_state(batch, np.float32)
    _compare(pc, batch, st, 0, SEED + 11)


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_batched_rows_at_every_alignment(pc, r):
    # sum n_t = 8000 + r: state and noise rows start r, 2r, 3r, 4r floats (mod 4) off a
    # 16-byte boundary, which the vector loads of the propagation phase shift back into place
    n = [4000, 3990 + r, 10]
    batch = synth.make_batch(len(n), 160, 160, 1, seed=SEED + 30 + r, n_values=n, min_sep=30.0)
    st = synth.batch_initial_state(batch, np.float32)
    _compare(pc, batch, st, 0, SEED + 31 + r)


def test_batched_full_size_workload_sampled(pc):
    """The multi-target workload at its full size, in the launch configuration whose throughput is
    measured (1000 targets with log-uniform particle counts in [10^3, 10^5], about 2.2e7 particles,
    1024 x 1024 frames, cell edge = PSF width, two blocks per SM): propagated states of every
    particle bit-exact, and 40 sampled targets (with the largest and the smallest) against the
    oracle run on their own slices, one by one."""
    Q = (0.5, 0.5, 0.1, 0.1, 1.0)
    batch = synth.make_batch(1000, 1024, 1024, 1, seed=SEED + 60)
    batch.h[:] = batch.sigma * 1.0
    T = len(batch.n)
    offs = np.concatenate([[0], np.cumsum(batch.n)])
    st = synth.batch_initial_state(batch, np.float32)
    nz = synth.batch_noise(batch, Q, SEED + 61, 0)
    u0 = synth.batch_u0(T, SEED + 61, 0)
    bt = pc.Batch(batch.n, batch.h, batch.sigma, batch.bg, batch.patch)
    bt.set_grid(2)
    bt.keep(pc.KEEP_ANCESTORS | pc.KEEP_QWEIGHTS)
    d_st = torch.from_numpy(st).cuda()
    bt.step(d_st, torch.from_numpy(batch.images[0]).cuda(), torch.from_numpy(nz).cuda(), torch.from_numpy(u0).cuda())
    torch.cuda.synchronize()
    res, derr = bt.results()
    assert derr == 0
    out = bt.outputs()
    prop = out["prop_state"].cpu().numpy()
    new = d_st.cpu().numpy()
    np.testing.assert_array_equal(prop, O.propagate(st, nz))
    tk, bx, by = _decode(out["bin_key"].cpu().numpy())
    cnt = out["bin_count"].cpu().numpy()
    kept = bt.kept()
    anc = kept["ancestor"].cpu().numpy()
    q = kept["qweight"].cpu().numpy()
    bt.close()
    rng = np.random.default_rng(SEED + 62)
    sample = set(rng.choice(T, 40, replace=False).tolist()) | {int(np.argmax(batch.n)), int(np.argmin(batch.n))}
    mism = 0
    for t in sorted(sample):
        sl = slice(offs[t], offs[t + 1])
        ref = O.pcsir_step(np.ascontiguousarray(st[:, sl]), batch.images[0], np.ascontiguousarray(nz[:, sl]),
                           u0[t], batch.h[t], _model(batch, t))
        sel = tk == t
        order = np.lexsort((bx[sel], by[sel]))
        np.testing.assert_array_equal(np.stack([bx[sel][order], by[sel][order]], 1), ref["bin_keys"])
        np.testing.assert_array_equal(cnt[sel][order], ref["bin_counts"])
        assert res[t]["n_bins"] == ref["bin_keys"].shape[0]
        est = np.array(res[t]["estimate"])
        assert np.all(np.abs(est - ref["estimate"]) <= 1e-5 * np.abs(ref["estimate"]) + 1e-6), (t, est)
        assert abs(res[t]["ess"] - ref["ess"]) <= 1e-5 * ref["ess"]
        mism += _check_target_resampling(new[:, sl], prop[:, sl], anc[sl], q[sl], u0[t], ref)
    # every target (not only the sampled ones): exactly systematic over its own integer weights
    for t in range(T):
        sl = slice(offs[t], offs[t + 1])
        np.testing.assert_array_equal(new[:, sl], prop[:, sl][:, anc[sl]])
        RC.exact_systematic(anc[sl], q[sl], u0[t])
    n_sampled = int(sum(batch.n[t] for t in sample))
    print("batched full size: %d particles, %d sampled targets, ancestors differing from the oracle's: %d of %d"
          % (int(batch.n.sum()), len(sample), mism, n_sampled))


def test_batched_step_graph_capture_replays(pc):
    n = [5000, 7000, 123]
    batch = synth.make_batch(len(n), 128, 128, 1, seed=SEED + 20, n_values=n, min_sep=30.0)
    st0 = torch.from_numpy(synth.batch_initial_state(batch, np.float32)).cuda()
    nz = torch.from_numpy(synth.batch_noise(batch, (0.5, 0.5, 0.1, 0.1, 1.0), SEED, 0)).cuda()
    img = torch.from_numpy(batch.images[0]).cuda()
    u0 = torch.from_numpy(synth.batch_u0(3, SEED, 0)).cuda()
    bt = pc.Batch(batch.n, batch.h, batch.sigma, batch.bg, batch.patch)
    s = torch.cuda.Stream()
    st = st0.clone()
    with torch.cuda.stream(s):
        bt.step(st, img, nz, u0, stream=s)
    torch.cuda.synchronize()
    ref = st.clone()
    g = torch.cuda.CUDAGraph()
    st.copy_(st0)
    with torch.cuda.graph(g, stream=s):
        bt.step(st, img, nz, u0, stream=s)
    st.copy_(st0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(st, ref)
    bt.close()


def test_autotuner_picks_a_candidate_and_caches(pc, tmp_path, monkeypatch):
    from paper_1310_5541_gb300 import autotune

    monkeypatch.setenv("PCSIR_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    table = autotune.tune(n_targets=4, frames=4, n_particles=4000)
    assert table["c"] in autotune.CANDIDATES and table["blocks_per_sm"] in (1, 2)
    assert autotune.load()["c"] == table["c"]
    h = autotune.cell_edges(np.array([1.2, 2.0]))
    np.testing.assert_allclose(h, np.array([1.2, 2.0]) * table["c"])


@pytest.mark.parametrize("barrier", [0, 2, 6])
def test_batched_barrier_wait_runs_out_and_the_batch_recovers(pc, barrier):
    """Failure detection without a fault: one grid barrier is made to wait for a block that does not
    exist (a release nothing gives) under a short poll limit.  The wait runs out, the step reports
    PCSIR_DERR_TIMEOUT (pcsir_batch_results returns PCSIR_ETIMEDOUT) and every block leaves the
    kernel; a barrier after the propagation (2, 6) leaves cells in the table.  The next step with
    the normal waits clears the table first and matches the oracle like any other step."""
    n = [3000, 4097, 500]
    batch = synth.make_batch(len(n), 160, 160, 2, seed=SEED + 40, n_values=n, min_sep=30.0)
    st = synth.batch_initial_state(batch, np.float32)
    bt = pc.Batch(batch.n, batch.h, batch.sigma, batch.bg, batch.patch)
    bt.set_wait(max_polls=2000, unreachable_barrier=barrier)
    d_st = torch.from_numpy(st.copy()).cuda()
    nz = torch.from_numpy(synth.batch_noise(batch, (0.5, 0.5, 0.1, 0.1, 1.0), SEED + 41, 0)).cuda()
    u0 = torch.from_numpy(synth.batch_u0(len(n), SEED + 41, 0)).cuda()
    bt.step(d_st, torch.from_numpy(batch.images[0]).cuda(), nz, u0)
    torch.cuda.synchronize()
    _, derr = bt.results()
    assert derr & pc.DERR_TIMEOUT, derr
    bt.set_wait()
    mism = _compare(pc, batch, st, 1, SEED + 42, bt=bt)
    print("after a timed-out step at barrier %d: ancestors differing from the oracle's %d" % (barrier, mism))
    bt.close()


def test_batched_cell_table_size_does_not_change_the_step(pc):
    """The autotuner's cell-table sizes (2^9, 2^10, 2^11 slots per block) and grids give the same step:
    new states and cell counts identical, posterior means equal up to the FP64 atomics' order."""
    n = [3000, 9000, 4097, 600, 15000]
    batch = synth.make_batch(len(n), 256, 256, 1, seed=SEED + 50, n_values=n, min_sep=30.0)
    batch.h[:] = [0.25, 0.5, 1.0, 0.1, 0.2]
    st = synth.batch_initial_state(batch, np.float32)
    nz = torch.from_numpy(synth.batch_noise(batch, (0.5, 0.5, 0.1, 0.1, 1.0), SEED + 51, 0)).cuda()
    u0 = torch.from_numpy(synth.batch_u0(len(n), SEED + 51, 0)).cuda()
    img = torch.from_numpy(batch.images[0]).cuda()
    outs = []
    for bits, bps in ((10, 2), (9, 2), (11, 1), (9, 1)):
        bt = pc.Batch(batch.n, batch.h, batch.sigma, batch.bg, batch.patch)
        bt.set_table(bits)
        bt.set_grid(bps)
        d = torch.from_numpy(st.copy()).cuda()
        bt.step(d, img, nz, u0)
        torch.cuda.synchronize()
        res, derr = bt.results()
        assert derr == 0
        o = bt.outputs()
        keys = o["bin_key"].cpu().numpy()
        order = np.argsort(keys)
        outs.append((d.cpu().numpy(), keys[order], o["bin_count"].cpu().numpy()[order],
                     np.array([r["estimate"] for r in res])))
        bt.close()
    for other in outs[1:]:
        np.testing.assert_array_equal(outs[0][0], other[0])
        np.testing.assert_array_equal(outs[0][1], other[1])
        np.testing.assert_array_equal(outs[0][2], other[2])
        np.testing.assert_allclose(outs[0][3], other[3], rtol=1e-12)


def test_batched_deferred_run_equals_plain_steps(pc):
    """Deferred resampling of a batch (pcsir_batch_deferred_begin, pcsir_batched_deferred_step,
    pcsir_batch_deferred_state) against plain batched steps on the same frames: at every frame the
    resampled states, propagated states, kept ancestors and integer weights are identical and the
    per-target results agree (cell counts exactly, means and ESS up to the order of FP64 atomics).
    The total particle count leaves every state row off a 16-byte boundary, the run includes a
    captured graph of two deferred steps replayed, and a plain step ends the run."""
    Q = (0.5, 0.5, 0.1, 0.1, 1.0)
    n = [4000, 3993, 10, 1500, 7]  # sum 9510: rows start 2, 0, 2, 0 floats (mod 4) past a 16-byte boundary
    F = 7
    batch = synth.make_batch(len(n), 192, 192, F, seed=SEED + 70, n_values=n, min_sep=30.0)
    T = len(n)
    st0 = torch.from_numpy(synth.batch_initial_state(batch, np.float32)).cuda()
    plain = pc.Batch(batch.n, batch.h, batch.sigma, batch.bg, batch.patch)
    dfr = pc.Batch(batch.n, batch.h, batch.sigma, batch.bg, batch.patch)
    for x in (plain, dfr):
        x.keep(pc.KEEP_ANCESTORS | pc.KEEP_QWEIGHTS)
    with pytest.raises(pc.PcsirError) as e:
        dfr.deferred_step(torch.from_numpy(batch.images[0]).cuda(),
                          torch.from_numpy(synth.batch_noise(batch, Q, SEED + 71, 0)).cuda(),
                          torch.from_numpy(synth.batch_u0(T, SEED + 71, 0)).cuda())
    assert e.value.status == pc.ESTATE
    sa = st0.clone()
    dfr.deferred_begin(st0)
    out = torch.empty_like(st0)
    frames = [(torch.from_numpy(batch.images[k]).cuda(), torch.from_numpy(synth.batch_noise(batch, Q, SEED + 71, k)).cuda(),
               torch.from_numpy(synth.batch_u0(T, SEED + 71, k)).cuda()) for k in range(F)]
    s = torch.cuda.Stream()
    k = 0
    while k < F:
        if k == 3:
            # frames 3 and 4 from one captured graph of two deferred steps (the state buffers alternate)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                dfr.deferred_step(*frames[3], stream=s)
                dfr.deferred_step(*frames[4], stream=s)
            graph.replay()
            torch.cuda.synchronize()
            plain.step(sa, *frames[3])
            plain.step(sa, *frames[4])
            k = 4
        else:
            plain.step(sa, *frames[k])
            dfr.deferred_step(*frames[k])
        dfr.deferred_state(out)
        torch.cuda.synchronize()
        assert torch.equal(out, sa), k
        pa, pd = plain.outputs(), dfr.outputs()
        assert torch.equal(pa["prop_state"], pd["prop_state"]), k
        ka, kd = plain.kept(), dfr.kept()
        assert torch.equal(ka["ancestor"], kd["ancestor"]), k
        assert torch.equal(ka["qweight"], kd["qweight"]), k
        ra, ea = plain.results()
        rd, ed = dfr.results()
        assert ea == 0 and ed == 0
        for t in range(T):
            assert ra[t]["n_bins"] == rd[t]["n_bins"], (k, t)
            np.testing.assert_allclose(rd[t]["estimate"], ra[t]["estimate"], rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(rd[t]["ess"], ra[t]["ess"], rtol=1e-12)
        k += 1
    # a plain step ends the run
    dfr.step(out, *frames[0])
    with pytest.raises(pc.PcsirError) as e:
        dfr.deferred_state(out)
    assert e.value.status == pc.ESTATE
    plain.close()
    dfr.close()
