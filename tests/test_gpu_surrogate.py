"""GPU checks of the likelihood surrogate against its FP64 oracle.

* inference (fused tcgen05 kernel) equals the oracle network on the oracle's
  inputs within a bound derived from bf16 rounding: each bf16 value (inputs,
  layer-1 activations) carries a relative error of at most 2^-9, propagated
  through |W| with the SiLU slope bound 1.1; W1 and W2 are chosen
  bf16-representable so that the weights carry no rounding;
* dataset rows equal the oracle's inputs to one bf16 unit, in state order;
* gradients of the training pass equal the oracle's backpropagation within
  2e-2 relative (Frobenius) per parameter group: the backward pass rounds four
  operands to bf16 (inputs, activations, two back-propagated gradients), each
  within 2^-9, i.e. 8e-3 summed, doubled for the FP32 accumulation order;
* one Adam update equals the oracle's;
* training on pairs the method generates lowers the error, and the trained
  surrogate inside the pcSIR step tracks as well as the exact likelihood
  while evaluating the exact likelihood for a small fraction of the dummies;
* a rejected surrogate (held-out error above the threshold) gives the plain
  step's result bit for bit.
"""
import math

import numpy as np
import pytest
import torch

from oracle import pcsir_oracle as O
from oracle import surrogate_oracle as S
from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = 1310554400
U = 2.0 ** -9  # unit roundoff of bf16


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


def bf16_round(a):
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits_to_f64(t):
    u = t.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def rand_params(rng, scale=1.0):
    p = {}
    for k, s in S.PARAM_SHAPES:
        fan_in = s[1] if len(s) == 2 else S.HIDDEN
        p[k] = rng.uniform(-1, 1, s) * math.sqrt(3.0 / fan_in) * scale
    p["b1"] = rng.uniform(-0.2, 0.2, 256)
    p["b2"] = rng.uniform(-0.2, 0.2, 256)
    p["b3"] = np.array([0.3])
    p["W1"] = bf16_round(p["W1"])
    p["W2"] = bf16_round(p["W2"])
    for k in ("b1", "b2", "w3", "b3"):
        p[k] = np.asarray(p[k], np.float32).astype(np.float64)
    return p


def spot_image(W, H, x0, y0, seed, i0=100.0, bg=10.0, sigma=1.5):
    lam = synth.render(W, H, x0, y0, i0, bg, sigma)
    return np.random.default_rng(seed).poisson(lam).astype(np.float32)


def states_near(rng, n, x0, y0, spread, W, H, n_edge=0):
    st = np.zeros((5, n))
    st[0] = x0 + rng.uniform(-spread, spread, n)
    st[1] = y0 + rng.uniform(-spread, spread, n)
    st[2] = rng.normal(0, 0.3, n)
    st[3] = rng.normal(0, 0.3, n)
    st[4] = rng.uniform(50, 150, n)
    if n_edge:
        st[0, :n_edge] = rng.uniform(0, 9.4, n_edge)  # patches leaving the image
    return st


def window_bound(img, x, y):
    """Bound on |T_gpu - T|: a few roundings of size 2^-24 per FP32 per-pixel term, and the final
    rounding of the (double-float) sum to FP32."""
    z = img.astype(np.float64)
    mag = z + np.where(z > 0, z * np.abs(np.log(np.where(z > 0, z, 1.0))), 0.0) + np.log(10.0) * z
    cx = np.floor(np.asarray(x) + 0.5).astype(int)
    cy = np.floor(np.asarray(y) + 0.5).astype(int)
    T = np.abs(S.window_term(img, x, y, 10.0))
    return np.array([16 * 2.0 ** -24 * mag[b - 10:b + 11, a - 10:a + 11].sum() for a, b in zip(cx, cy)]) \
        + 2.0 ** -23 * T + 1e-9


def forward_bound(p, X):
    """Worst-case |GPU - oracle| of the network output from bf16 rounding (see module docstring)."""
    z1 = X @ p["W1"].T + p["b1"]
    a1 = S.silu(z1)
    e1 = U * (np.abs(X) @ np.abs(p["W1"]).T) * 1.0001 + 1e-6 * (np.abs(X) @ np.abs(p["W1"]).T + np.abs(p["b1"]))
    ea1 = 1.1 * e1 + U * np.abs(a1) * 1.0001 + 1e-6 * np.abs(a1)
    z2 = a1 @ p["W2"].T + p["b2"]
    e2 = ea1 @ np.abs(p["W2"]).T + 1e-6 * (np.abs(a1) @ np.abs(p["W2"]).T + np.abs(p["b2"]))
    eo = 1.1 * e2 @ np.abs(p["w3"]) + 1e-6 * (np.abs(S.silu(z2)) @ np.abs(p["w3"]) + abs(p["b3"][0]))
    return eo


def test_inference_matches_oracle(pc):
    rng = np.random.default_rng(SEED)
    W, H = 96, 80
    img = spot_image(W, H, 47.3, 38.8, SEED)
    n = 1000  # seven full tiles of 128 and a ragged tail
    st = states_near(rng, n, 47.3, 38.8, 4.0, W, H, n_edge=20)
    p = rand_params(rng)
    mean, scale = -150.0, 40.0
    sur = pc.Surrogate(capacity=1, batch=128, i0_ref=100.0, sigma_ref=1.5, max_pixels=W * H)
    sur.set_params(S.pack(p), mean, scale)
    d_st = torch.from_numpy(st).cuda()
    pred = sur.predict(d_st, torch.from_numpy(img).cuda(), 10.0, 1.5).cpu().numpy()
    X, clipped = S.features(img, st[0], st[1], st[4], 1.5, 10.0, 100.0, 1.5)
    assert clipped[:20].all() and not clipped[20:].any()
    assert np.isnan(pred[clipped]).all()
    T = S.window_term(img, st[0, ~clipped], st[1, ~clipped], 10.0)
    ref = S.predict_ll(p, mean, scale, X[~clipped], T)
    bound = scale * forward_bound(p, X[~clipped]) + window_bound(img, st[0, ~clipped], st[1, ~clipped])
    err = np.abs(pred[~clipped] - ref)
    print("inference: max err %.3e, max bound %.3e, max err/bound %.3f" % (err.max(), bound.max(),
                                                                         (err / bound).max()))
    assert np.all(err <= bound)
    # the parameters round-trip
    flat, m2, s2 = sur.get_params()
    assert m2 == mean and s2 == scale
    np.testing.assert_array_equal(flat, S.pack(p).astype(np.float32))
    sur.close()


def test_dataset_rows_follow_state_order(pc):
    rng = np.random.default_rng(SEED + 1)
    W, H = 64, 64
    img = spot_image(W, H, 31.0, 30.2, SEED + 1)
    d_img = torch.from_numpy(img).cuda()
    sur = pc.Surrogate(capacity=5000, batch=128)
    all_X, all_y, all_st, all_c, all_cens, all_tb = [], [], [], [], [], []
    for call, n in enumerate((700, 1, 333)):
        st = states_near(rng, n, 31.0, 30.2, 3.0, W, H, n_edge=min(n, 40) if call != 1 else 0)
        all_st.append(st)
        ll = rng.normal(-100, 30, n)
        floor = -120.0 if call == 2 else -np.inf
        # a strided view, as the step's dummy outputs are
        buf = torch.zeros((5, n + 17), dtype=torch.float64, device="cuda")
        buf[:, :n] = torch.from_numpy(st).cuda()
        sur.add(buf[:, :n], torch.from_numpy(ll).cuda(), d_img, 10.0, 1.5, label_floor=floor)
        X, clipped = S.features(img, st[0], st[1], st[4], 1.5, 10.0, 128.0, 1.5)
        all_X.append(X[~clipped])
        T = S.window_term(img, st[0, ~clipped], st[1, ~clipped], 10.0)
        all_y.append(np.maximum(ll[~clipped], floor) - T)
        all_tb.append(window_bound(img, st[0, ~clipped], st[1, ~clipped]))
        all_cens.append(ll[~clipped] < floor)
        all_c.append(clipped)
    X = np.concatenate(all_X)
    y = np.concatenate(all_y)
    assert sur.rows() == X.shape[0]
    dx, dy, dc = sur.dataset()
    g = bf16_bits_to_f64(dx)
    assert np.all(g[:, 445:] == 0)
    want = bf16_round(X.astype(np.float32))
    diff = np.abs(g[:, :445] - want)
    assert np.all(diff <= 2.0 * U * np.abs(want) + 1e-30)
    assert np.mean(diff == 0) > 0.999
    tb = np.concatenate(all_tb)
    lab = dy.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(lab - y) <= tb + 2.0 ** -24 * np.abs(y) * 1.01)
    cens = np.concatenate(all_cens)
    assert cens.any() and not cens.all()
    np.testing.assert_array_equal(dc.cpu().numpy(), cens.astype(np.uint8))
    # predictions from stored rows (label units) and from the image differ by the window term
    rng2 = np.random.default_rng(9)
    sur.set_params(S.pack(rand_params(rng2)), -100.0, 30.0)
    pr = sur.predict_rows(0, sur.rows()).cpu().numpy()
    sts = np.concatenate(all_st, axis=1)[:, ~np.concatenate(all_c)]
    ps = sur.predict(torch.from_numpy(np.ascontiguousarray(sts)).cuda(), d_img, 10.0, 1.5).cpu().numpy()
    T = S.window_term(img, sts[0], sts[1], 10.0)
    assert np.all(np.abs((ps - pr) - T) <= tb + 1e-9 * np.abs(ps))
    sur.clear()
    assert sur.rows() == 0
    sur.close()


def _dataset_for_grads(pc, n_rows=512):
    """The GPU's training rows from synthetic states, and the oracle's own rows from the same
    states: inputs, residual labels and censoring flags (no oracle input read back from the GPU)."""
    rng = np.random.default_rng(SEED + 2)
    W, H = 64, 64
    img = spot_image(W, H, 32.4, 31.7, SEED + 2)
    st = states_near(rng, n_rows, 32.4, 31.7, 3.0, W, H)
    m = synth.Model(patch=21)
    ll = O.loglik(img, st[0], st[1], st[4], m)
    sur = pc.Surrogate(capacity=n_rows, batch=256)
    floor = float(np.median(ll))  # half the rows censored
    sur.add(torch.from_numpy(st).cuda(), torch.from_numpy(ll).cuda(), torch.from_numpy(img).cuda(), 10.0, 1.5,
            label_floor=floor)
    assert sur.rows() == n_rows
    X, clipped = S.features(img, st[0], st[1], st[4], 1.5, 10.0, 128.0, 1.5)
    assert not clipped.any()
    y = np.maximum(ll, floor) - S.window_term(img, st[0], st[1], 10.0)
    return sur, X, y, ll < floor


def test_gradients_match_oracle_backprop(pc):
    sur, X, y, cens = _dataset_for_grads(pc)
    p = rand_params(np.random.default_rng(11))
    mean, scale = float(y.mean()), float(y.std())
    sur.set_params(S.pack(p), mean, scale)
    for begin, n in ((0, 256), (128, 128)):
        g, loss = sur.grads(begin, n)
        t = (y[begin:begin + n] - mean) / scale
        lo, go = S.loss_and_grads(p, X[begin:begin + n], t, cens[begin:begin + n])
        assert abs(loss - lo) <= 1e-2 * lo
        gg = S.unpack(g.astype(np.float64))
        for k, _ in S.PARAM_SHAPES:
            rel = np.linalg.norm(gg[k] - go[k]) / np.linalg.norm(go[k])
            print("grad %s: rel err %.2e" % (k, rel))
            assert rel <= 2e-2, k
    sur.close()


def test_adam_update_matches_oracle(pc):
    sur, X, y, cens = _dataset_for_grads(pc)
    p = rand_params(np.random.default_rng(12))
    mean, scale = float(y.mean()), float(y.std())
    sur.set_params(S.pack(p), mean, scale)
    lr = 1e-3
    sur.train(0, 256, 1, lr, 0)  # seed 0: rows 0..255 in order, one update
    after, _, _ = sur.get_params()
    t = (y[:256] - mean) / scale
    _, go = S.loss_and_grads(p, X[:256], t, cens[:256])
    q = {k: v.copy() for k, v in p.items()}
    S.adam_step(q, go, {}, lr)
    a = S.unpack(after.astype(np.float64))
    for k, _ in S.PARAM_SHAPES:
        sig = np.abs(go[k]) > 0.05 * np.abs(go[k]).max()
        d_gpu = a[k] - p[k]
        d_or = q[k] - p[k]
        # first bias-corrected step: -lr g / (|g| + eps) = -lr sign(g) for significant g
        assert np.all(np.abs(d_gpu[sig] - d_or[sig]) <= 1e-3 * lr + 2e-7), k
        assert np.all(np.abs(d_gpu) <= lr * 1.0001 + 2e-7), k
    sur.close()


# ----------------------------------------------------------------------------
# Training on pairs the method generates, and the surrogate inside the step
# ----------------------------------------------------------------------------
MODEL = synth.Model(patch=21)
W_IMG = H_IMG = 128


def _frames(seq, N, seed):
    for k in range(seq.images.shape[0]):
        yield (torch.from_numpy(seq.images[k]).cuda(),
               torch.from_numpy(synth.make_noise(N, MODEL.q, seed, k, np.float32)).cuda(),
               synth.make_u0(seed, k))


@pytest.fixture(scope="module")
def trained(pc):
    from paper_1310_5541_gb300 import surrogate

    N = 1 << 15
    ctx = pc.Context(N, torch.float32, patch=21, psf_sigma=MODEL.sigma_psf, bg=MODEL.bg)
    sur = pc.Surrogate(capacity=1 << 23, batch=4096, i0_ref=128.0, sigma_ref=1.5, max_pixels=W_IMG * H_IMG)
    hs = (0.03, 0.05, 0.1, 0.2, 0.5)
    # training rows from 100 sequences, then validation rows from 10 further ones
    n_train = None
    for part, (n_seq, frames) in enumerate(((100, 20), (10, 6))):
        for i in range(n_seq):
            seed = SEED + 100 + 1000 * part + i
            seq = synth.make_sequence(W_IMG, H_IMG, frames, MODEL, seed)
            st = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).cuda()
            surrogate.collect(ctx, sur, st, _frames(seq, N, seed), hs[i % len(hs)], MODEL.bg, MODEL.sigma_psf)
        if part == 0:
            n_train = sur.rows()
    rows = sur.rows()
    sur.init(7)
    res = surrogate.fit(sur, steps=40000, lr=2e-3, seed=3, n_train=n_train, chunk=2000)
    print("surrogate: %d rows (%d train), label std %.1f nats, validation rmse %.3f max %.3f nats, "
          "loss %.4f -> %.5f" % (rows, n_train, res["val_label_std"], res["val_rmse"], res["val_max"],
                                 res["loss"][:50].mean(), res["loss"][-200:].mean()))
    ctx.close()
    return sur, res


def test_training_lowers_the_error(pc, trained):
    sur, res = trained
    loss = res["loss"]
    assert loss[-200:].mean() < 0.05 * loss[:50].mean()
    # on rows of sequences it never saw, the error is a small fraction of the spread of the labels
    assert res["val_rmse"] < 0.1 * res["val_label_std"]


def _track(pc, sur, seq, N, h, seed, **attach):
    ctx = pc.Context(N, torch.float32, patch=21, psf_sigma=MODEL.sigma_psf, bg=MODEL.bg)
    if sur is not None:
        pc.attach_surrogate(ctx, sur, **attach)
    st = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).cuda()
    est, checks = [], []
    for k, (img, nz, u0) in enumerate(_frames(seq, N, seed)):
        pc.pcsir_step(ctx, st, img, h, nz, u0)
        torch.cuda.synchronize()
        r = ctx.last_result()
        assert r["device_error"] == 0
        est.append(r["estimate"][:2])
        if sur is not None:
            checks.append(pc.surrogate_last_check(ctx))
    ctx.close()
    est = np.array(est)
    rmse = float(np.sqrt(np.mean(np.sum((est - seq.gt[1:, :2]) ** 2, axis=1))))
    return rmse, checks


def test_trained_surrogate_tracks_like_exact_likelihood(pc, trained):
    sur, _ = trained
    N, h = 1 << 17, 0.05
    rm_ex, rm_su, exact_frac, fallbacks = [], [], [], 0
    for r in range(3):
        seed = SEED + 500 + r
        seq = synth.make_sequence(W_IMG, H_IMG, 20, MODEL, seed)
        a, _ = _track(pc, None, seq, N, h, seed)
        b, checks = _track(pc, sur, seq, N, h, seed, holdout_frac=0.02, min_holdout=32, window=20.0, max_err=3.0)
        rm_ex.append(a)
        rm_su.append(b)
        fallbacks += sum(c["fallback"] for c in checks)
        exact_frac.append(sum(c["n_exact"] for c in checks) / max(1, sum(c["n_dummies"] for c in checks)))
    print("tracking rmse exact %s, surrogate %s; exact evaluations %s; fallbacks %d" % (
        np.round(rm_ex, 4), np.round(rm_su, 4), np.round(exact_frac, 3), fallbacks))
    assert np.mean(rm_su) <= 1.05 * np.mean(rm_ex) + 0.005
    assert np.mean(exact_frac) < 0.25


def test_rejected_surrogate_gives_the_plain_step(pc):
    N, h = 20000, 0.1
    seq = synth.make_sequence(W_IMG, H_IMG, 3, MODEL, SEED + 900)
    sur = pc.Surrogate(capacity=1, batch=128)
    sur.init(5)  # untrained: its predictions are far off
    outs = []
    for use in (False, True):
        ctx = pc.Context(N, torch.float32, patch=21, psf_sigma=MODEL.sigma_psf, bg=MODEL.bg)
        if use:
            pc.attach_surrogate(ctx, sur, holdout_frac=0.05, min_holdout=16, window=1e9, max_err=0.0)
        st = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).cuda()
        res = []
        for k, (img, nz, u0) in enumerate(_frames(seq, N, SEED + 900)):
            pc.pcsir_step(ctx, st, img, h, nz, u0)
            torch.cuda.synchronize()
            res.append(ctx.last_result())
            if use:
                c = pc.surrogate_last_check(ctx)
                assert c["fallback"] == 1 and c["n_exact"] == c["n_dummies"] and c["n_holdout"] >= 16
        outs.append((st.cpu().numpy(), res))
        ctx.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    # the estimate's sums are accumulated with atomics: equal up to their order
    for a, b in zip(outs[0][1], outs[1][1]):
        np.testing.assert_allclose(a["estimate"], b["estimate"], rtol=1e-12)
        np.testing.assert_allclose(a["ess"], b["ess"], rtol=1e-12)
    sur.close()


def test_surrogate_step_uses_predictions_and_checks_like_oracle(pc):
    """Wiring of the surrogate-assisted step against the oracle on the same input: cells and dummies
    as the oracle forms them, the oracle's network prediction for unclipped dummies and its exact
    likelihood for clipped ones (within the inference and likelihood bounds), the held-out set the
    oracle's hash selects, the check statistics the oracle computes, and the estimate of the oracle's
    step with those log-likelihoods (within what the bounds allow).  The step's predictions also equal
    the stand-alone inference entry point's at the step's own dummies, bit for bit."""
    N, h = 60000, 0.1
    W, H = 64, 48
    m = synth.Model(patch=21)
    seq = synth.make_sequence(W, H, 1, m, SEED + 950, start=(12.0, 20.0), vmax=0.1, margin=0)
    rng = np.random.default_rng(3)
    sur = pc.Surrogate(capacity=1, batch=128)
    p = rand_params(rng, scale=0.5)
    mean, scale = -60.0, 15.0
    sur.set_params(S.pack(p), mean, scale)
    ctx = pc.Context(N, torch.float32, patch=21, psf_sigma=m.sigma_psf, bg=m.bg, keep=pc.KEEP_ANCESTORS | pc.KEEP_WEIGHTS | pc.KEEP_PARTICLE_BIN | pc.KEEP_LOGLIK)
    frac, min_ho, window, max_err = 0.03, 8, 25.0, 1e9
    pc.attach_surrogate(ctx, sur, holdout_frac=frac, min_holdout=min_ho, window=window, max_err=max_err)
    st0 = synth.initial_state(seq.gt[0], N, np.float32)
    st0[0] += np.random.default_rng(4).normal(0, 1.5, N).astype(np.float32)  # a wide cloud: some patches clipped
    nz = synth.make_noise(N, m.q, SEED, 0, np.float32)
    u0 = synth.make_u0(SEED, 0)
    img = seq.images[0]
    d_st = torch.from_numpy(st0).cuda()
    pc.pcsir_step(ctx, d_st, torch.from_numpy(img).cuda(), h, torch.from_numpy(nz).cuda(), u0)
    torch.cuda.synchronize()
    out = ctx.outputs()
    chk = pc.surrogate_last_check(ctx)
    B = out["n_bins"]
    bll = out["bin_loglik"].cpu().numpy()
    bxy = out["bin_xy"].cpu().numpy()
    order = np.lexsort((bxy[0], bxy[1]))
    # the oracle's cells and dummies (the plain mean of the members), against the step's
    prop = O.propagate(st0, nz)
    keys, member, _ = O.segment(*O.bin_coords(prop[0], prop[1], h))
    assert B == keys.shape[0]
    np.testing.assert_array_equal(bxy[:, order].T, keys)
    dum = O.dummies(prop, member, B)
    dg = out["dummy"].cpu().numpy()[:, order]
    np.testing.assert_allclose(dg[:2], dum[:2], rtol=0, atol=1e-9)
    np.testing.assert_allclose(dg[2:], dum[2:], rtol=0, atol=2.5e-7)
    bll = bll[order]
    X, clipped = S.features(img, dum[0], dum[1], dum[4], m.sigma_psf, m.bg, 100.0, 1.5)
    assert clipped.any() and not clipped.all()
    assert chk["n_clipped"] == int(clipped.sum())
    # the oracle's log-likelihood of every cell: exact where the patch is clipped, else the network's
    exact = O.loglik(img, dum[0], dum[1], dum[4], m)
    e = 1e-3  # slope of the exact likelihood, for the dummies' displacement (1e-9 px, 2.5e-7 in I0)
    gx = np.abs(O.loglik(img, dum[0] + e, dum[1], dum[4], m) - O.loglik(img, dum[0] - e, dum[1], dum[4], m)) / (2 * e)
    gy = np.abs(O.loglik(img, dum[0], dum[1] + e, dum[4], m) - O.loglik(img, dum[0], dum[1] - e, dum[4], m)) / (2 * e)
    ga = np.abs(O.loglik(img, dum[0], dum[1], dum[4] + e, m) - O.loglik(img, dum[0], dum[1], dum[4] - e, m)) / (2 * e)
    tol_exact = 1e-4 + 4e-7 * np.abs(exact) + 2.0 * (1e-9 * (gx + gy) + 2.5e-7 * ga)
    nc = ~clipped
    T = S.window_term(img, dum[0, nc], dum[1, nc], m.bg)
    pred = np.full(B, np.nan)
    pred[nc] = S.predict_ll(p, mean, scale, X[nc], T)
    tol_pred = np.zeros(B)
    tol_pred[nc] = scale * forward_bound(p, X[nc]) + window_bound(img, dum[0, nc], dum[1, nc]) + 1e-6 * scale
    ll_ref = np.where(clipped, exact, pred)
    tol = np.where(clipped, tol_exact, tol_pred)
    assert np.all(np.abs(bll - ll_ref) <= tol), ("cell loglik", (np.abs(bll - ll_ref) / tol).max())
    # the step's predictions are the stand-alone inference's at the step's own dummies
    pred_gpu = sur.predict(out["dummy"].contiguous(), torch.from_numpy(img).cuda(), m.bg, m.sigma_psf).cpu().numpy()
    np.testing.assert_array_equal(bll[nc], pred_gpu[order][nc])
    # held-out selection and statistics, as the oracle selects and computes them
    fe = max(frac, min_ho / B)
    held = S.holdout_mask(keys[:, 0], keys[:, 1], 0, fe) & nc
    assert chk["n_holdout"] == int(held.sum())
    ref = S.holdout_check(pred[held], exact[held], ll_ref.max(), window, max_err)
    # each statistic moves by at most the prediction and exact-likelihood bounds of its cells
    b = tol_pred[held] + tol_exact[held]
    tmax = float(tol.max())
    thr = ll_ref.max() - window
    if np.all(np.abs(np.maximum(pred[held], exact[held]) - thr) > b + tmax):
        assert chk["n_significant"] == ref["n_significant"]
    assert abs(chk["max_abs_err"] - ref["max_abs_err"]) <= b.max()
    assert abs(chk["rms_err"] - ref["rms_err"]) <= b.max()
    assert chk["fallback"] == 0 and chk["n_exact"] == int(held.sum()) + int(clipped.sum())
    # the oracle's step with the oracle's cell log-likelihoods: the estimate within what log-likelihood
    # differences of at most delta allow (each weight within a factor e^(2 delta))
    r = O.pcsir_step(st0, img, nz, u0, h, m, lik=lambda x, y, i0: ll_ref)
    est = np.array(ctx.last_result()["estimate"])
    rw = np.expm1(2.0 * tmax) + 1e-5
    spread = (r["w"][None, :] * np.abs(prop.astype(np.float64) - r["estimate"][:, None])).sum(axis=1)
    assert np.all(np.abs(est - r["estimate"]) <= rw * spread + 1e-5 * np.abs(r["estimate"]) + 1e-6)
    # and, a property of the step's own values, the estimate formed from its cells' log-likelihoods
    lw = bll[member]
    w = np.exp(lw - lw.max())
    w /= w.sum()
    est_g = (prop.astype(np.float64) * w[None, :]).sum(axis=1)
    assert np.all(np.abs(est - est_g) <= 1e-5 * np.abs(est_g) + 1e-6)
    ctx.close()
    sur.close()
