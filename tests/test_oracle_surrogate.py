"""Pins of the surrogate oracle against what its definitions fix (CPU only).

* network inputs: a pure-Python loop over a small hand-built image;
* backpropagation: central finite differences of the loss in FP64 at the
  network's real sizes (445 -> 256 -> 256 -> 1);
* silu and its derivative at closed-form points;
* Adam: the first bias-corrected step is -lr g / (|g| + eps) exactly, the
  second follows the recursion written out for one scalar;
* splitmix64: the published first outputs of the generator seeded with 0;
* held-out check: hand-made cases.
"""
import math

import numpy as np
import pytest

from oracle import surrogate_oracle as S


def _rand_params(rng, scale=0.3):
    p = {}
    for k, s in S.PARAM_SHAPES:
        fan_in = s[1] if len(s) == 2 else S.HIDDEN
        p[k] = rng.standard_normal(s) * scale / math.sqrt(fan_in) * (3.0 if k == "w3" else 1.0)
    return p


def test_features_match_pixel_loop():
    rng = np.random.default_rng(1)
    H, W = 40, 37
    img = rng.uniform(0, 50, (H, W)).astype(np.float32)
    xs = np.array([18.2, 10.49, 10.5, 25.0, 3.0, 35.9])
    ys = np.array([20.7, 10.51, 11.49, 29.2, 20.0, 1.0])
    i0 = np.array([90.0, 100.0, 110.0, 5.0, 70.0, 100.0])
    bg, i0_ref, s_ref = 10.0, 100.0, 2.0
    X, clipped = S.features(img, xs, ys, i0, 1.5, bg, i0_ref, s_ref)
    for n in range(len(xs)):
        cx = math.floor(xs[n] + 0.5)
        cy = math.floor(ys[n] + 0.5)
        clip = not (cx - 10 >= 0 and cx + 10 <= W - 1 and cy - 10 >= 0 and cy + 10 <= H - 1)
        assert clipped[n] == clip
        k = 0
        for r in range(cy - 10, cy + 11):
            for c in range(cx - 10, cx + 11):
                z = float(img[r, c]) if (0 <= r < H and 0 <= c < W) else bg
                assert X[n, k] == (z - bg) / i0_ref
                k += 1
        assert X[n, 441] == 2 * (xs[n] - cx) and X[n, 442] == 2 * (ys[n] - cy)
        assert X[n, 443] == i0[n] / i0_ref and X[n, 444] == 1.5 / s_ref
    # exact ties go up, as the exact likelihood's nearest pixel does
    assert X[2, 441] == -1.0 and X[1, 441] == 2 * (10.49 - 10)
    assert not clipped[0] and clipped[4] and clipped[5]


def test_window_term_splits_the_poisson_likelihood():
    # ll - T equals the spot-only sum  sum_j z_j log(1 + I0 g_j / bg) - I0 g_j  (closed form, pixel loop)
    from oracle import pcsir_oracle as O
    from paper_1310_5541_gb300 import synth

    rng = np.random.default_rng(5)
    H, W = 40, 44
    img = rng.poisson(synth.render(W, H, 21.3, 19.6, 100.0, 10.0, 1.5)).astype(np.float32)
    img[5, 7] = 0.0  # a zero count inside some windows
    xs = np.array([21.3, 20.6, 14.2, 23.9])
    ys = np.array([19.6, 20.4, 15.1, 12.5])
    i0 = np.array([100.0, 90.0, 120.0, 0.0])
    m = synth.Model(patch=21)
    ll = O.loglik(img, xs, ys, i0, m)
    T = S.window_term(img, xs, ys, 10.0)
    for n in range(len(xs)):
        cx, cy = math.floor(xs[n] + 0.5), math.floor(ys[n] + 0.5)
        r = 0.0
        for py in range(cy - 10, cy + 11):
            for px in range(cx - 10, cx + 11):
                g = math.exp(-((px - xs[n]) ** 2 + (py - ys[n]) ** 2) / (2 * 1.5 ** 2))
                r += float(img[py, px]) * math.log1p(i0[n] * g / 10.0) - i0[n] * g
        assert ll[n] - T[n] == pytest.approx(r, rel=1e-9, abs=1e-8)
    # I0 = 0: the prediction lambda = bg everywhere, and ll is the window term itself
    assert ll[3] == pytest.approx(T[3], rel=1e-12)


def test_silu_closed_forms():
    assert S.silu(0.0) == 0.0 and S.silu_grad(0.0) == 0.5
    t = np.array([-3.0, -0.5, 0.7, 4.0])
    np.testing.assert_allclose(S.silu(t), t / (1 + np.exp(-t)), rtol=0)
    h = 1e-6
    np.testing.assert_allclose(S.silu_grad(t), (S.silu(t + h) - S.silu(t - h)) / (2 * h), rtol=1e-8)
    # maximum of the derivative, used by the error bounds of the GPU tests
    grid = np.linspace(-10, 10, 200001)
    assert S.silu_grad(grid).max() < 1.0999


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(7)
    p = _rand_params(rng)
    X = rng.standard_normal((16, S.N_IN)) * 0.5
    t = rng.standard_normal(16)
    loss, g = S.loss_and_grads(p, X, t)
    eps = 1e-6
    for k, shape in S.PARAM_SHAPES:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for j in idx:
            old = flat[j]
            flat[j] = old + eps
            lp = S.loss_and_grads(p, X, t)[0]
            flat[j] = old - eps
            lm = S.loss_and_grads(p, X, t)[0]
            flat[j] = old
            fd = (lp - lm) / (2 * eps)
            an = g[k].reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)) + 1e-9, (k, j, fd, an)
    assert loss > 0


def test_censored_rows_count_only_above_their_floor():
    rng = np.random.default_rng(9)
    p = _rand_params(rng)
    X = rng.standard_normal((16, S.N_IN)) * 0.5
    out, _ = S.forward(p, X)
    t = out + np.where(np.arange(16) % 2 == 0, 0.3, -0.3)  # even rows: output below the label
    cens = np.arange(16) % 4 < 2                           # rows 0, 1, 4, 5, ...
    loss, g = S.loss_and_grads(p, X, t, cens)
    # censored rows with out below the floor (rows 0, 4, 8, 12) contribute nothing
    keep = ~(cens & (np.arange(16) % 2 == 0))
    assert loss == pytest.approx(np.sum(keep * 0.09) / 16, rel=1e-12)
    # the same gradient as the plain loss over the counted rows, rescaled to the full batch
    l2, g2 = S.loss_and_grads(p, X[keep], t[keep])
    for k, _ in S.PARAM_SHAPES:
        np.testing.assert_allclose(g[k], g2[k] * keep.sum() / 16, rtol=1e-12, atol=1e-15)
    # and central differences agree with it
    eps = 1e-6
    flat = p["W2"].reshape(-1)
    for j in rng.choice(flat.size, 6, replace=False):
        old = flat[j]
        flat[j] = old + eps
        lp = S.loss_and_grads(p, X, t, cens)[0]
        flat[j] = old - eps
        lm = S.loss_and_grads(p, X, t, cens)[0]
        flat[j] = old
        assert abs((lp - lm) / (2 * eps) - g["W2"].reshape(-1)[j]) <= 1e-6 * max(1e-3, abs(g["W2"].reshape(-1)[j]))


def test_gradient_vanishes_at_a_perfect_fit():
    rng = np.random.default_rng(8)
    p = _rand_params(rng)
    X = rng.standard_normal((9, S.N_IN))
    out, _ = S.forward(p, X)
    loss, g = S.loss_and_grads(p, X, out)
    assert loss == 0.0
    for k, _ in S.PARAM_SHAPES:
        assert np.all(g[k] == 0.0)


def test_adam_first_and_second_step():
    p = {k: np.zeros(s) for k, s in S.PARAM_SHAPES}
    g = {k: np.full(s, 0.25) for k, s in S.PARAM_SHAPES}
    g["b3"] = np.array([-2.0])
    st = {}
    S.adam_step(p, g, st, lr=0.01)
    # bias-corrected first step: m^ = g, v^ = g^2
    np.testing.assert_allclose(p["W1"], -0.01 * 0.25 / (0.25 + 1e-8), rtol=1e-15)
    np.testing.assert_allclose(p["b3"], 0.01 * 2.0 / (2.0 + 1e-8), rtol=1e-15)
    g2 = {k: np.full(s, -1.0) for k, s in S.PARAM_SHAPES}
    S.adam_step(p, g2, st, lr=0.01)
    m = 0.9 * (0.1 * 0.25) + 0.1 * (-1.0)
    v = 0.999 * (0.001 * 0.0625) + 0.001 * 1.0
    want = -0.01 * 0.25 / (0.25 + 1e-8) - 0.01 * (m / (1 - 0.81)) / (math.sqrt(v / (1 - 0.999 ** 2)) + 1e-8)
    np.testing.assert_allclose(p["W2"], want, rtol=1e-13)


def test_splitmix64_published_outputs():
    # the generator seeded with 0: its first two outputs (Steele, Lea and Flood 2014)
    assert S.splitmix64(0) == 0xE220A8397B1DCDAF
    assert S.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_holdout_mask_fraction_and_determinism():
    rng = np.random.default_rng(3)
    bx = rng.integers(-5000, 5000, 40000)
    by = rng.integers(-5000, 5000, 40000)
    m = S.holdout_mask(bx, by, 17, 0.02)
    assert abs(m.mean() - 0.02) < 5 * math.sqrt(0.02 * 0.98 / 40000)
    assert np.array_equal(m, S.holdout_mask(bx, by, 17, 0.02))
    assert not np.array_equal(m, S.holdout_mask(bx, by, 18, 0.02))
    assert not S.holdout_mask(bx, by, 17, 0.0).any() and S.holdout_mask(bx, by, 17, 1.0).all()


def test_holdout_check_cases():
    r = S.holdout_check([-10.0, -50.0, -12.0], [-10.2, -80.0, -11.0], max_pred=-9.0, window=20.0, max_err=0.5)
    # the second dummy is far below the maximum on both sides: not significant
    assert r["n_significant"] == 2 and r["max_abs_err"] == pytest.approx(1.0) and r["fallback"]
    r = S.holdout_check([-10.0, -12.0], [-10.1, -12.2], max_pred=-10.0, window=20.0, max_err=0.5)
    assert not r["fallback"] and r["max_abs_err"] == pytest.approx(0.2)
    assert S.holdout_check([np.nan], [-1.0], -1.0, 20.0, 0.5)["fallback"]
    e = S.holdout_check([], [], -1.0, 20.0, 0.5)
    assert e["n_holdout"] == 0 and not e["fallback"]


def test_pack_roundtrip():
    rng = np.random.default_rng(2)
    p = _rand_params(rng)
    flat = S.pack(p)
    assert flat.size == S.N_PARAMS == 256 * 445 + 256 + 256 * 256 + 256 + 256 + 1
    q = S.unpack(flat)
    for k, _ in S.PARAM_SHAPES:
        assert np.array_equal(p[k], q[k])


# ----------------------------------------------------------------------------
# The 3D surrogate (11 x 11 x 7 voxel patch)
# ----------------------------------------------------------------------------
def _spot_volume(rng, W=30, H=26, D=18, x0=14.3, y0=12.6, z0=8.8):
    from paper_1310_5541_gb300 import synth

    return rng.poisson(synth.render3(W, H, D, x0, y0, z0, 100.0, 10.0, 1.5, 3.0)).astype(np.float32)


def test_features3_match_voxel_loop():
    """Inputs 0..846 are the window's voxels with x fastest, then y, then z; then the sub-voxel
    offsets, I0 and sigma; a window leaving the volume is clipped."""
    rng = np.random.default_rng(31)
    vol = _spot_volume(rng)
    xs, ys, zs = np.array([14.3, 13.51, 4.2]), np.array([12.6, 11.49, 12.0]), np.array([8.8, 9.5, 9.0])
    i0 = np.array([100.0, 80.0, 90.0])
    X, clipped = S.features3(vol, xs, ys, zs, i0, 1.5, 10.0, 128.0, 1.5)
    assert list(clipped) == [False, False, True]  # x = 4.2: cx - 5 < 0
    for n in range(2):
        cx, cy, cz = (math.floor(v + 0.5) for v in (xs[n], ys[n], zs[n]))
        f = 0
        for dz in range(-3, 4):
            for dy in range(-5, 6):
                for dx in range(-5, 6):
                    assert X[n, f] == (float(vol[cz + dz, cy + dy, cx + dx]) - 10.0) / 128.0
                    f += 1
        assert f == S.NPIX3 == 847
        assert X[n, 847:].tolist() == [2 * (xs[n] - cx), 2 * (ys[n] - cy), 2 * (zs[n] - cz), i0[n] / 128.0, 1.0]


def test_window_term3_splits_the_3d_poisson_likelihood():
    """ll - T equals the spot-only sum over the 11 x 11 x 7 window, by a voxel loop against the 3D
    oracle's likelihood (an independent code path); with I0 = 0, ll is the window term itself."""
    from oracle import pcsir3_oracle as O3

    rng = np.random.default_rng(32)
    vol = _spot_volume(rng)
    vol[6, 10, 12] = 0.0  # a zero count inside the windows
    xs, ys, zs = np.array([14.3, 13.6, 15.4]), np.array([12.6, 13.4, 11.8]), np.array([8.8, 8.2, 9.4])
    i0 = np.array([100.0, 70.0, 0.0])
    m = O3.Model3()
    ll = O3.loglik(vol, xs, ys, zs, i0, m)
    T = S.window_term3(vol, xs, ys, zs, 10.0)
    for n in range(len(xs)):
        cx, cy, cz = (math.floor(v + 0.5) for v in (xs[n], ys[n], zs[n]))
        r = 0.0
        for vz in range(cz - 3, cz + 4):
            for vy in range(cy - 5, cy + 6):
                for vx in range(cx - 5, cx + 6):
                    g = math.exp(-((vx - xs[n]) ** 2 + (vy - ys[n]) ** 2) / (2 * 1.5 ** 2)
                                 - (vz - zs[n]) ** 2 / (2 * 3.0 ** 2))
                    r += float(vol[vz, vy, vx]) * math.log1p(i0[n] * g / 10.0) - i0[n] * g
        assert ll[n] - T[n] == pytest.approx(r, rel=1e-9, abs=1e-8)
    assert ll[2] == pytest.approx(T[2], rel=1e-12)


def test_holdout_mask3_key_and_fraction():
    # the key packs (bx + 2^20, by + 2^20, bz + 2^20) in 21-bit fields; compare with a direct call
    bx, by, bz = np.array([3, -7, 0]), np.array([-2, 5, 0]), np.array([1, 0, -4])
    got = S.holdout_mask3(bx, by, bz, 11, 0.5)
    for i in range(3):
        key = (int(bx[i]) + 2 ** 20) + ((int(by[i]) + 2 ** 20) << 21) + ((int(bz[i]) + 2 ** 20) << 42)
        h = S.splitmix64((key + 11 * 0x9E3779B97F4A7C15) % 2 ** 64)
        assert got[i] == ((h >> 40) < (1 << 23))
    rng = np.random.default_rng(3)
    cells = rng.integers(-1000, 1000, size=(3, 20000))
    frac = S.holdout_mask3(cells[0], cells[1], cells[2], 5, 0.1).mean()
    assert 0.09 < frac < 0.11
    assert S.holdout_mask3(cells[0], cells[1], cells[2], 5, 1.0).all()


def test_backprop3_shapes_match_central_differences():
    """The forward and backward passes are shape-generic: a spot check with the 3D input width."""
    rng = np.random.default_rng(33)
    p = {k: rng.standard_normal(s) * (0.05 if k == "W1" else 0.1) for k, s in S.PARAM_SHAPES3}
    X = rng.standard_normal((8, S.N_IN3)) * 0.5
    t = rng.standard_normal(8)
    loss, g = S.loss_and_grads(p, X, t)
    assert g["W1"].shape == (256, 852)
    eps = 1e-6
    for k in ("W1", "b1", "w3"):
        flat = p[k].reshape(-1)
        for j in rng.choice(flat.size, size=6, replace=False):
            old = flat[j]
            flat[j] = old + eps
            lp = S.loss_and_grads(p, X, t)[0]
            flat[j] = old - eps
            lm = S.loss_and_grads(p, X, t)[0]
            flat[j] = old
            an = g[k].reshape(-1)[j]
            assert abs((lp - lm) / (2 * eps) - an) <= 1e-6 * max(1e-3, abs(an)) + 1e-9
    flat = S.pack(p, S.PARAM_SHAPES3)
    assert flat.size == S.N_PARAMS3
    back = S.unpack(flat, S.PARAM_SHAPES3)
    np.testing.assert_array_equal(back["W1"], p["W1"])
