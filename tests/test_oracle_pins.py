"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a closed
form, a library routine's special case, an invariant, the paper's error bound
or a brute-force loop on a tiny input, chosen so that a dropped term, a wrong
sign or index or a transposed operand in the oracle fails at least one test.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

from oracle import pcsir_oracle as O
from paper_1310_5541_gb300 import synth

MODEL9 = synth.Model(sigma_psf=1.5, I0=100.0, bg=10.0, patch=9)


# --------------------------------------------------------------------------
# Section 5.1 dynamics
# --------------------------------------------------------------------------
def test_propagate_closed_form_constant_velocity():
    """Zero process noise: after k steps x = x0 + k vx, v and I0 unchanged (NCV model)."""
    st = np.array([[10.0, 3.0], [20.0, -4.0], [0.5, -0.25], [-1.5, 2.0], [100.0, 7.0]])
    zero = np.zeros_like(st)
    s = st
    for _ in range(8):
        s = O.propagate(s, zero)
    np.testing.assert_array_equal(s[0], st[0] + 8 * st[2])
    np.testing.assert_array_equal(s[1], st[1] + 8 * st[3])
    np.testing.assert_array_equal(s[2:], st[2:])


def test_propagate_noise_enters_each_component_once():
    st = np.zeros((5, 1))
    noise = np.array([[1.0], [2.0], [4.0], [8.0], [16.0]])
    s = O.propagate(st, noise)
    # position picks up its own noise but not yet the new velocity's noise
    np.testing.assert_array_equal(s[:, 0], [1.0, 2.0, 4.0, 8.0, 16.0])
    s2 = O.propagate(s, np.zeros((5, 1)))
    np.testing.assert_array_equal(s2[:, 0], [5.0, 10.0, 4.0, 8.0, 16.0])


def test_propagate_float32_stays_float32_rounding():
    """The FP32 path rounds after each addition, as IEEE float32 does."""
    st = np.zeros((5, 1), np.float32)
    st[0, 0] = np.float32(16777216.0)  # 2^24: adding 1 is not representable
    st[2, 0] = np.float32(1.0)
    noise = np.zeros((5, 1), np.float32)
    noise[0, 0] = np.float32(1.0)
    s = O.propagate(st, noise)
    assert s.dtype == np.float32
    # (2^24 + 1) rounds to 2^24 (ties to even), then + 1 rounds again to 2^24
    assert s[0, 0] == np.float32(16777216.0)


# --------------------------------------------------------------------------
# Algorithm 2: equal-size bins over position, h = 1 cells are the pixels
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_bin_coords_hand_values(dtype):
    # h = 1: pixel n covers [n - 0.5, n + 0.5)
    x = np.array([0.0, 0.49, 0.5, -0.5, -0.51, 3.7, 511.5], dtype)
    bx, _ = O.bin_coords(x, x, 1.0)
    assert bx.tolist() == [0, 0, 1, 0, -1, 4, 512]
    # h = 0.5: cells [-0.5, 0) -> 0, [0, 0.5) -> 1, [0.5, 1) -> 2
    x = np.array([-0.5, -0.01, 0.0, 0.49, 0.5, 0.99, 1.0], dtype)
    bx, _ = O.bin_coords(x, x, 0.5)
    assert bx.tolist() == [0, 0, 1, 1, 2, 2, 3]
    # h = 2: cells [-0.5, 1.5) -> 0, [1.5, 3.5) -> 1
    x = np.array([-0.5, 1.49, 1.5, 3.49, 3.5], dtype)
    bx, _ = O.bin_coords(x, x, 2.0)
    assert bx.tolist() == [0, 0, 1, 1, 2]


def test_bin_coords_y_uses_y():
    x = np.array([0.0, 0.0])
    y = np.array([0.0, 5.2])
    bx, by = O.bin_coords(x, y, 1.0)
    assert bx.tolist() == [0, 0] and by.tolist() == [0, 5]


def _bruteforce_groups(bx, by, state):
    groups = {}
    for i in range(len(bx)):
        groups.setdefault((int(by[i]), int(bx[i])), []).append(i)
    keys = sorted(groups)
    means = []
    for k in keys:
        idx = groups[k]
        means.append([sum(float(state[d, i]) for i in idx) / len(idx) for d in range(5)])
    return keys, [len(groups[k]) for k in keys], np.array(means).T, groups


def test_segment_and_dummies_hand_and_bruteforce():
    # hand case: two particles in cell (1,1) of h = 0.5, one in cell (0,1)
    st = np.zeros((5, 3))
    st[0] = [0.1, 0.3, -0.2]
    st[1] = [0.1, 0.2, 0.1]
    st[4] = [90.0, 110.0, 50.0]
    bx, by = O.bin_coords(st[0], st[1], 0.5)
    keys, member, counts = O.segment(bx, by)
    assert keys.tolist() == [[0, 1], [1, 1]]
    assert counts.tolist() == [1, 2]
    d = O.dummies(st, member, 2)
    np.testing.assert_allclose(d[0], [-0.2, 0.2], rtol=0, atol=1e-15)
    np.testing.assert_allclose(d[1], [0.1, 0.15], rtol=0, atol=1e-15)
    np.testing.assert_allclose(d[4], [50.0, 100.0], rtol=0, atol=1e-13)
    # brute force on a random tiny cloud
    rng = np.random.default_rng(5)
    st = rng.normal(size=(5, 40)) * np.array([[1.3], [0.9], [0.2], [0.2], [5.0]]) + 3.0
    bx, by = O.bin_coords(st[0], st[1], 0.5)
    keys, member, counts = O.segment(bx, by)
    bk, bc, bm, groups = _bruteforce_groups(bx, by, st)
    assert [tuple(k[::-1]) for k in keys.tolist()] == bk
    assert counts.tolist() == bc
    np.testing.assert_allclose(O.dummies(st, member, len(bk)), bm, rtol=1e-14)
    for b, k in enumerate(bk):
        assert sorted(np.nonzero(member == b)[0].tolist()) == groups[k]


def test_weighted_dummy_is_centre_of_mass():
    """Section 4: the dummy is the weight-averaged state of its bin."""
    st = np.zeros((5, 2))
    st[0] = [0.0, 0.4]
    w = np.array([3.0, 1.0])
    d = O.dummies(st, np.array([0, 0]), 1, prior_w=w)
    assert d[0, 0] == pytest.approx(0.1)


# --------------------------------------------------------------------------
# Eq. (object) + Eq. (likelihood)
# --------------------------------------------------------------------------
def _patch_of(img, cx, cy, R):
    return img[cy - R:cy + R + 1, cx - R:cx + R + 1]


def test_poisson_loglik_matches_full_logpmf_up_to_constant():
    """Two positions with the same patch: differences equal those of sum log Poisson pmf."""
    W = H = 32
    lam_true = synth.render(W, H, 15.2, 16.1, 100.0, 10.0, 1.5)
    img = np.random.default_rng(3).poisson(lam_true).astype(np.float32)
    img[14, 12] = 0.0  # exercise the z = 0 branch inside the patch
    pts = [(15.1, 15.8, 98.0), (14.6, 16.3, 104.0), (15.4, 15.55, 80.0)]
    # all three round to the pixel (15, 16)
    ll = O.loglik(img, [p[0] for p in pts], [p[1] for p in pts], [p[2] for p in pts], MODEL9)
    full = []
    for (x, y, i0) in pts:
        lam = synth.render(W, H, x, y, i0, 10.0, 1.5)
        full.append(stats.poisson.logpmf(_patch_of(img, 15, 16, 4), _patch_of(lam, 15, 16, 4)).sum())
    np.testing.assert_allclose(np.diff(ll), np.diff(full), rtol=0, atol=1e-9)


def test_poisson_term_is_minus_half_deviance_and_zero_at_perfect_fit():
    """Per pixel the term is z log(lam/z) - (lam - z) = -D/2 with the Poisson deviance D."""
    img = np.zeros((9, 9), np.float32)
    lam = synth.render(9, 9, 4.0, 4.0, 100.0, 10.0, 1.5)
    # image equal to the prediction -> every term is 0
    ll = O.loglik(lam, [4.0], [4.0], [100.0], MODEL9)
    assert abs(ll[0]) < 1e-9
    # all-zero image -> sum of -lambda over the patch
    ll0 = O.loglik(img, [4.0], [4.0], [100.0], MODEL9)
    assert ll0[0] == pytest.approx(-lam.sum(), rel=1e-12)
    # a single bright pixel: deviance via scipy's rel_entr (a different formula)
    img2 = lam.copy()
    img2[3, 5] = 170.0
    ll2 = O.loglik(img2, [4.0], [4.0], [100.0], MODEL9)
    z, l = 170.0, lam[3, 5]
    dev = 2.0 * (special.rel_entr(z, l) - z + l)
    assert ll2[0] == pytest.approx(-0.5 * dev, rel=1e-10)


def test_sse_loglik_closed_forms():
    """Paper Eq. (likelihood): 0 on the noise-free image, -P^2 c^2 / 2 sigma_xi^2 with offset c."""
    m = synth.Model(sigma_psf=1.5, I0=100.0, bg=10.0, patch=9, lik="sse", sigma_xi=20.0)
    lam = synth.render(40, 40, 20.0, 21.0, 100.0, 10.0, 1.5)
    assert abs(O.loglik(lam, [20.0], [21.0], [100.0], m)[0]) < 1e-20
    ll = O.loglik(lam + 3.0, [20.0], [21.0], [100.0], m)[0]
    assert ll == pytest.approx(-81 * 9.0 / (2 * 400.0), rel=1e-12)


def test_loglik_patch_clipped_at_image_border_bruteforce():
    """Pixels of S_x outside the image contribute nothing (brute-force loop, 3x3 patch)."""
    rng = np.random.default_rng(11)
    img = rng.poisson(12.0, size=(5, 6)).astype(np.float32)
    m = synth.Model(sigma_psf=0.8, I0=30.0, bg=5.0, patch=3)
    for (x, y, i0) in [(0.2, 0.1, 30.0), (5.4, 4.49, 25.0), (-0.7, 2.0, 10.0), (2.5, 2.5, -3.0)]:
        tot = 0.0
        cx, cy = math.floor(x + 0.5), math.floor(y + 0.5)
        for py in range(cy - 1, cy + 2):
            for px in range(cx - 1, cx + 2):
                if 0 <= px < 6 and 0 <= py < 5:
                    lam = max(i0, 0.0) * math.exp(-((px - x) ** 2 + (py - y) ** 2) / (2 * 0.64)) + 5.0
                    z = float(img[py, px])
                    tot += (z * math.log(lam / z) if z > 0 else 0.0) - (lam - z)
        assert O.loglik(img, [x], [y], [i0], m)[0] == pytest.approx(tot, rel=1e-12, abs=1e-12)


# --------------------------------------------------------------------------
# Algorithm 1: normalisation, ESS, systematic resampling
# --------------------------------------------------------------------------
def test_normalise_and_ess_closed_forms():
    w, m, T = O.normalise(np.full(7, -3.0))
    np.testing.assert_allclose(w, 1 / 7)
    assert O.ess(w) == pytest.approx(7.0)
    w, _, _ = O.normalise(np.array([0.0, -1e4, -1e4]))
    assert O.ess(w) == pytest.approx(1.0)
    w, _, _ = O.normalise(np.log(np.array([1.0, 3.0])) + 500.0)  # no overflow
    np.testing.assert_allclose(w, [0.25, 0.75])


def test_systematic_resample_bruteforce_and_invariants():
    rng = np.random.default_rng(2)
    for N in [1, 2, 5, 17, 64]:
        for _ in range(20):
            w = rng.exponential(size=N) ** 3
            w /= w.sum()
            u0 = rng.random()
            s = O.systematic_resample(w, u0)
            # brute force: walk the cumulative sum with a scalar loop
            ref, c, l = [], 0.0, 0
            cum = []
            for v in w:
                c += v
                cum.append(c)
            for i in range(N):
                U = (i + u0) / N * cum[-1]
                l = 0
                while l < N - 1 and not (cum[l] > U):
                    l += 1
                ref.append(l)
            assert s.tolist() == ref
            copies = np.bincount(s, minlength=N)
            assert copies.sum() == N
            assert np.all(copies >= np.floor(N * w - 1e-9)) and np.all(copies <= np.ceil(N * w + 1e-9))
    # uniform weights reproduce the identity map
    for N in [1, 10, 1000]:
        assert O.systematic_resample(np.full(N, 1.0 / N), 0.5).tolist() == list(range(N))


def test_posterior_mean_closed_form():
    st = np.zeros((5, 3))
    st[0] = [1.0, 2.0, 4.0]
    st[1] = [0.0, 0.0, 6.0]
    w = np.array([0.5, 0.25, 0.25])
    est = O.posterior_mean(w, st)
    assert est[0] == pytest.approx(2.0) and est[1] == pytest.approx(1.5)


# --------------------------------------------------------------------------
# Section 4.2: one particle per bin recovers SIR exactly
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_one_particle_per_bin_is_sir(dtype):
    seq = synth.make_sequence(48, 48, 3, MODEL9, seed=7)
    N = 300
    st = synth.initial_state(seq.gt[0], N, dtype)
    for k in range(3):
        noise = synth.make_noise(N, MODEL9.q, 7, k, dtype)
        u0 = synth.make_u0(7, k)
        a = O.sir_step(st, seq.images[k], noise, u0, MODEL9)
        b = O.pcsir_step(st, seq.images[k], noise, u0, 1e-4, MODEL9)
        assert b["bin_counts"].max() == 1 and b["bin_counts"].size == N
        np.testing.assert_array_equal(a["w"], b["w"])
        np.testing.assert_array_equal(a["estimate"], b["estimate"])
        np.testing.assert_array_equal(a["ancestors"], b["ancestors"])
        st = a["new_state"]


def test_pcsir_converges_to_sir_as_h_shrinks():
    """Section 6: the pcSIR posterior mean approaches SIR's as the bin edge h -> 0."""
    seq = synth.make_sequence(48, 48, 1, MODEL9, seed=9)
    N = 4000
    st = synth.initial_state(seq.gt[0], N)
    noise = synth.make_noise(N, MODEL9.q, 9, 0)
    u0 = synth.make_u0(9, 0)
    sir = O.sir_step(st, seq.images[0], noise, u0, MODEL9)["estimate"]
    errs = []
    for h in [2.0, 1.0, 0.5, 0.25, 0.1, 0.03, 0.01]:
        e = O.pcsir_step(st, seq.images[0], noise, u0, h, MODEL9)["estimate"]
        errs.append(np.hypot(e[0] - sir[0], e[1] - sir[1]))
    assert errs[-1] < 0.02 * errs[0]
    assert errs[-1] < 1e-3
    # each factor-of-three-or-so refinement does not make it worse by much
    assert all(errs[i + 2] <= errs[i] * 1.05 for i in range(len(errs) - 2))


# --------------------------------------------------------------------------
# Appendix: mid-point Riemann-sum error bound of the piecewise-constant likelihood
# --------------------------------------------------------------------------
def _gauss2(x, y, a, b, s):
    return np.exp(-((x - a) ** 2 + (y - b) ** 2) / (2 * s * s))


def test_midpoint_riemann_bound_with_lattice_dummies():
    """Cells holding a regular lattice of particles put the dummy at the cell centre, so the
    piecewise-constant likelihood integrates by the mid-point rule; its error must stay within
    the Appendix bound (per cell: l_x l_y / 24 (l_x^2 max|f_xx| + l_y^2 max|f_yy|)) and shrink
    like h^2."""
    a, b, s = 0.13, -0.21, 0.7
    lo, hi = -1.5, 2.5  # domain covered exactly by cells at every h below
    exact = (s * math.sqrt(math.pi / 2) * (special.erf((hi - a) / (s * math.sqrt(2)))
                                           - special.erf((lo - a) / (s * math.sqrt(2))))) * \
            (s * math.sqrt(math.pi / 2) * (special.erf((hi - b) / (s * math.sqrt(2)))
                                           - special.erf((lo - b) / (s * math.sqrt(2)))))
    errs = []
    for h in [1.0, 0.5, 0.25, 0.125]:
        n = int(round((hi - lo) / h))
        m = 4  # m x m lattice per cell, symmetric about the cell centre
        u = (np.arange(m) + 0.5) / m * h
        xs = (lo + np.arange(n)[:, None] * h + u[None, :]).reshape(-1)
        X_, Y_ = np.meshgrid(xs, xs)
        st = np.zeros((5, X_.size))
        # lo = -1.5 lies on the cell grid -0.5 + k h for every h used here
        st[0] = X_.reshape(-1)
        st[1] = Y_.reshape(-1)
        bx, by = O.bin_coords(st[0], st[1], h)
        keys, member, counts = O.segment(bx, by)
        assert np.all(counts == m * m) and keys.shape[0] == n * n
        d = O.dummies(st, member, keys.shape[0])
        dx, dy = d[0], d[1]
        approx = float(np.sum(_gauss2(dx, dy, a, b, s)) * h * h)
        err = abs(approx - exact)
        # bound: sum over cells of the per-cell bound with cell-wise maxima of |f_xx|, |f_yy|
        bound = 0.0
        g = np.linspace(0, 1, 9)
        for cxv, cyv in zip(dx, dy):
            gx = cxv - h / 2 + g * h
            gy = cyv - h / 2 + g * h
            GX, GY = np.meshgrid(gx, gy)
            f = _gauss2(GX, GY, a, b, s)
            fxx = np.abs((((GX - a) ** 2) / s ** 4 - 1 / s ** 2) * f).max()
            fyy = np.abs((((GY - b) ** 2) / s ** 4 - 1 / s ** 2) * f).max()
            bound += h * h / 24.0 * (h * h * fxx + h * h * fyy)
        assert err <= bound
        errs.append(err)
    slopes = np.diff(np.log(errs)) / np.diff(np.log([1.0, 0.5, 0.25, 0.125]))
    assert np.all(np.abs(slopes - 2.0) < 0.35)


# --------------------------------------------------------------------------
# Linear-Gaussian case: the particle filters must agree with the Kalman filter
# --------------------------------------------------------------------------
def _lg_lik(z, r):
    return lambda x, y, i0: -((x - z[0]) ** 2 + (y - z[1]) ** 2) / (2 * r * r)


@pytest.mark.parametrize("kind", ["sir", "pcsir"])
def test_linear_gaussian_matches_kalman(kind):
    rng = np.random.default_rng(21)
    q = (0.5, 0.5, 0.1, 0.1, 1.0)
    r = 0.7
    x0 = np.array([10.0, 12.0, 0.8, -0.4, 100.0])
    truth = x0.copy()
    zs = []
    for _ in range(6):
        truth = truth + np.array([truth[2], truth[3], 0, 0, 0]) + rng.normal(size=5) * np.array(q)
        zs.append(truth[:2] + rng.normal(size=2) * r)
    means, covs = O.ncv_kalman(x0, q, r, zs)
    N = 40000
    st = synth.initial_state(x0, N)
    m = synth.Model(q=q)
    min_ess = float(N)
    for k, z in enumerate(zs):
        noise = synth.make_noise(N, q, 33, k)
        u0 = synth.make_u0(33, k)
        if kind == "sir":
            res = O.sir_step(st, None, noise, u0, m, lik=_lg_lik(z, r))
        else:
            res = O.pcsir_step(st, None, noise, u0, 0.02, m, lik=_lg_lik(z, r))
        # Monte-Carlo error carried by the population is set by the smallest ESS so far
        min_ess = min(min_ess, res["ess"])
        for d in range(4):
            sd = math.sqrt(covs[k][d, d] / min_ess)
            assert abs(res["estimate"][d] - means[k][d]) < 5.0 * sd
        # the weighted particle covariance matches the Kalman covariance
        cov = np.cov(res["prop"][:4].astype(np.float64), aweights=res["w"])
        np.testing.assert_allclose(np.diag(cov), np.diag(covs[k])[:4], rtol=0.1)
        st = res["new_state"]


# --------------------------------------------------------------------------
# Section 5.5 / Fig. 5: Monte-Carlo rate of the weighted estimate
# --------------------------------------------------------------------------
def test_monte_carlo_rate_is_inverse_sqrt_n():
    """Pseudo-tracking: prior uniform on a 3x3-pixel square, SSE likelihood (sigma_xi = 20);
    the RMSE of the importance-weighted mean falls like N^-1/2."""
    m = synth.Model(sigma_psf=1.16, I0=60.0, bg=10.0, patch=9, lik="sse", sigma_xi=20.0)
    img = synth.render(32, 32, 16.2, 15.9, 60.0, 10.0, 1.16)
    rng = np.random.default_rng(8)
    # reference posterior mean by fine quadrature over the prior square
    g = np.linspace(14.7, 17.7, 301)
    GX, GY = np.meshgrid(g, g)
    ll = O.loglik(img, GX.ravel(), GY.ravel(), np.full(GX.size, 60.0), m)
    w = np.exp(ll - ll.max())
    ref = np.array([np.sum(w * GX.ravel()), np.sum(w * GY.ravel())]) / w.sum()
    Ns = [200, 800, 3200]
    rmse = []
    for N in Ns:
        e2 = []
        for _ in range(150):
            x = rng.uniform(14.7, 17.7, N)
            y = rng.uniform(14.7, 17.7, N)
            wn, _, _ = O.normalise(O.loglik(img, x, y, np.full(N, 60.0), m))
            e2.append((np.sum(wn * x) - ref[0]) ** 2 + (np.sum(wn * y) - ref[1]) ** 2)
        rmse.append(math.sqrt(np.mean(e2)))
    slope = np.polyfit(np.log(Ns), np.log(rmse), 1)[0]
    assert -0.65 < slope < -0.35


def test_coc_dummies_sit_at_cell_centres():
    """pcSIR-CoC (Section 5.4): the binned components of each dummy are its cell's geometric
    centre, checked by a loop over the cells; the other components stay the members' mean, and
    with particles on a lattice centred in each cell CoC and CoM coincide."""
    rng = np.random.default_rng(21)
    m = synth.Model(patch=9)
    img = rng.poisson(synth.render(32, 32, 15.2, 14.7, 100.0, 10.0, 1.5)).astype(np.float32)
    N = 500
    st = np.zeros((5, N))
    st[0] = 15.0 + rng.normal(0, 1.0, N)
    st[1] = 15.0 + rng.normal(0, 1.0, N)
    st[4] = 100.0 + rng.normal(0, 3.0, N)
    nz = np.zeros_like(st)
    for h in (0.5, 1.0, 0.3):
        r = O.pcsir_step(st, img, nz, 0.4, h, m, dummy="coc")
        com = O.pcsir_step(st, img, nz, 0.4, h, m)
        for j, (bx, by) in enumerate(r["bin_keys"]):
            lo_x, lo_y = bx * h - 0.5, by * h - 0.5
            assert r["dummies"][0, j] == pytest.approx(lo_x + h / 2, abs=1e-12)
            assert r["dummies"][1, j] == pytest.approx(lo_y + h / 2, abs=1e-12)
        np.testing.assert_array_equal(r["dummies"][2:], com["dummies"][2:])
    # a 2 x 2 lattice centred in every cell: centre of mass = cell centre
    h = 1.0
    cx, cy = np.meshgrid(np.arange(10, 20), np.arange(12, 18))
    pts = []
    for dx in (-0.25, 0.25):
        for dy in (-0.25, 0.25):
            pts.append(np.stack([cx.ravel() + dx, cy.ravel() + dy]))
    P2 = np.concatenate(pts, axis=1)
    lat = np.zeros((5, P2.shape[1]))
    lat[:2] = P2
    lat[4] = 100.0
    a = O.pcsir_step(lat, img, np.zeros_like(lat), 0.4, h, m, dummy="coc")
    b = O.pcsir_step(lat, img, np.zeros_like(lat), 0.4, h, m)
    np.testing.assert_allclose(a["dummies"], b["dummies"], atol=1e-12)
    np.testing.assert_allclose(a["estimate"], b["estimate"], rtol=1e-12)
