"""Pins of the oracle's ESS-thresholded steps (Algorithm 1's test: resample only when N_eff
is below N_thr, the weights being carried to the next step otherwise; no GPU).

Each test checks ``sir_step_ess`` / ``pcsir_step_ess`` against something other
than themselves: the every-step filters in the limit that always resamples,
hand-summed closed-form log-likelihoods along unresampled trajectories, the
Kalman filter, brute-force weighted means, a closed-form ESS, and invariants.
"""
import math

import numpy as np
import pytest

from oracle import pcsir_oracle as O
from paper_1310_5541_gb300 import synth

MODEL9 = synth.Model(sigma_psf=1.5, I0=100.0, bg=10.0, patch=9)


def _lg_lik(z, r):
    return lambda x, y, i0: -((x - z[0]) ** 2 + (y - z[1]) ** 2) / (2 * r * r)


@pytest.mark.parametrize("kind", ["sir", "pcsir"])
def test_threshold_above_n_is_the_every_step_filter(kind):
    """ess_min > N: every step resamples, exactly as sir_step / pcsir_step, and the carried
    log-weights are uniform (zeros)."""
    seq = synth.make_sequence(48, 48, 3, MODEL9, seed=3)
    N = 500
    st_a = st_b = synth.initial_state(seq.gt[0], N)
    lw = None
    for k in range(3):
        noise = synth.make_noise(N, MODEL9.q, 3, k)
        u0 = synth.make_u0(3, k)
        if kind == "sir":
            a = O.sir_step(st_a, seq.images[k], noise, u0, MODEL9)
            b = O.sir_step_ess(st_b, lw, seq.images[k], noise, u0, N + 1.0, MODEL9)
        else:
            a = O.pcsir_step(st_a, seq.images[k], noise, u0, 0.5, MODEL9)
            b = O.pcsir_step_ess(st_b, lw, seq.images[k], noise, u0, 0.5, N + 1.0, MODEL9)
        assert b["resampled"]
        np.testing.assert_array_equal(a["ancestors"], b["ancestors"])
        np.testing.assert_array_equal(a["new_state"], b["new_state"])
        np.testing.assert_array_equal(b["logw_out"], np.zeros(N))
        st_a, st_b, lw = a["new_state"], b["new_state"], b["logw_out"]


def test_never_resampling_carries_the_sum_of_log_likelihoods():
    """ess_min = 0: no step resamples, particle i keeps its index, and its carried log-weight
    is the sum over steps of the closed-form Gaussian log-likelihood at its own propagated
    positions, minus the maximum over particles."""
    rng = np.random.default_rng(4)
    q = (0.5, 0.5, 0.1, 0.1, 1.0)
    r = 0.8
    zs = [np.array([10.3, 11.8]), np.array([11.0, 11.5]), np.array([11.9, 11.0])]
    N = 64
    st = synth.initial_state(np.array([10.0, 12.0, 0.8, -0.4, 100.0]), N)
    m = synth.Model(q=q)
    lw = None
    total = np.zeros(N)
    for k, z in enumerate(zs):
        noise = rng.normal(size=(5, N)) * np.array(q)[:, None]
        res = O.sir_step_ess(st, lw, None, noise, 0.5, 0.0, m, lik=_lg_lik(z, r))
        assert not res["resampled"]
        np.testing.assert_array_equal(res["ancestors"], np.arange(N))
        np.testing.assert_array_equal(res["new_state"], res["prop"])
        for i in range(N):  # brute force, one particle at a time
            dx, dy = res["prop"][0, i] - z[0], res["prop"][1, i] - z[1]
            total[i] += -(dx * dx + dy * dy) / (2 * r * r)
        np.testing.assert_allclose(res["logw_out"], total - total.max(), rtol=0, atol=1e-12)
        assert res["logw_out"].max() == 0.0
        st, lw = res["new_state"], res["logw_out"]


def test_sequential_importance_sampling_matches_kalman():
    """Without resampling (ess_min = 0) the carried weights make the weighted particle mean the
    Kalman mean of the linear-Gaussian model, within the Monte-Carlo error of its ESS."""
    rng = np.random.default_rng(21)
    q = (0.5, 0.5, 0.1, 0.1, 1.0)
    r = 0.9
    x0 = np.array([10.0, 12.0, 0.8, -0.4, 100.0])
    truth = x0.copy()
    zs = []
    for _ in range(3):
        truth = truth + np.array([truth[2], truth[3], 0, 0, 0]) + rng.normal(size=5) * np.array(q)
        zs.append(truth[:2] + rng.normal(size=2) * r)
    means, covs = O.ncv_kalman(x0, q, r, zs)
    N = 60000
    st = synth.initial_state(x0, N)
    m = synth.Model(q=q)
    lw = None
    for k, z in enumerate(zs):
        res = O.sir_step_ess(st, lw, None, synth.make_noise(N, q, 35, k), synth.make_u0(35, k), 0.0, m,
                             lik=_lg_lik(z, r))
        assert not res["resampled"]
        for d in range(4):
            sd = math.sqrt(covs[k][d, d] / res["ess"])
            assert abs(res["estimate"][d] - means[k][d]) < 5.0 * sd
        st, lw = res["new_state"], res["logw_out"]


def test_prior_weighted_dummies_bruteforce():
    """Section 4: with carried weights the dummy of a bin is its members' weighted mean."""
    st = np.zeros((5, 6))
    st[0] = [0.10, 0.20, 0.30, 1.10, 1.20, 1.20]
    st[1] = [0.00, 0.10, -0.10, 0.00, 0.20, 0.10]
    st[2] = [0.05, -0.05, 0.025, 0.1, 0.2, -0.1]
    st[4] = [90.0, 100.0, 110.0, 80.0, 120.0, 100.0]
    lw = np.log(np.array([1.0, 2.0, 5.0, 0.5, 0.25, 4.0]))
    res = O.pcsir_step_ess(st, lw, None, np.zeros_like(st), 0.5, 1.0, 0.0, MODEL9,
                           lik=lambda x, y, i0: np.zeros_like(x))
    keys = res["bin_keys"].tolist()
    w = np.exp(lw)
    for b, key in enumerate(keys):
        members = [i for i in range(6) if res["member_bin"][i] == b]
        for d in range(5):
            num = sum(w[i] * (st[d, i] + (st[d + 2, i] if d < 2 else 0.0)) for i in members)
            den = sum(w[i] for i in members)
            assert res["dummies"][d, b] == pytest.approx(num / den, rel=1e-14, abs=1e-14)
    assert len(keys) == 2


def test_ess_closed_form_and_strict_threshold():
    """Two weight classes a (half the particles) and b: N_eff = N (a + b)^2 / (2 (a^2 + b^2));
    the step resamples exactly when N_eff < ess_min."""
    N = 1000
    st = synth.initial_state(np.array([5.0, 5.0, 0.0, 0.0, 100.0]), N)
    la, lb = 0.0, math.log(3.0)
    ll = np.where(np.arange(N) % 2 == 0, la, lb)
    lik = lambda x, y, i0: ll.copy()
    a, b = 1.0, 3.0
    ess_cf = N * (a + b) ** 2 / (2 * (a * a + b * b))
    res = O.sir_step_ess(st, None, None, np.zeros((5, N)), 0.3, 0.0, synth.Model(), lik=lik)
    assert res["ess"] == pytest.approx(ess_cf, rel=1e-12)
    for thr, expect in ((ess_cf * (1 - 1e-9), False), (ess_cf * (1 + 1e-9), True)):
        r2 = O.sir_step_ess(st, None, None, np.zeros((5, N)), 0.3, thr, synth.Model(), lik=lik)
        assert r2["resampled"] is expect


def test_one_particle_per_bin_is_sir_with_carried_weights():
    """Section 4.2: cells holding one particle each give SIR's weights, decisions and
    estimates, also with carried (non-uniform) weights."""
    # the paper's Gaussian likelihood (sigma_xi = 20) keeps N_eff near 10-50 of 300, so that
    # the threshold 0.1 N both resamples and carries weights within these five steps
    m = synth.Model(sigma_psf=1.5, I0=100.0, bg=10.0, patch=9, lik="sse", sigma_xi=20.0)
    seq = synth.make_sequence(48, 48, 5, m, seed=11)
    N = 300
    st = synth.initial_state(seq.gt[0], N)
    lw = None
    decisions = []
    for k in range(5):
        noise = synth.make_noise(N, m.q, 11, k)
        u0 = synth.make_u0(11, k)
        a = O.sir_step_ess(st, lw, seq.images[k], noise, u0, 0.1 * N, m)
        b = O.pcsir_step_ess(st, lw, seq.images[k], noise, u0, 1e-4, 0.1 * N, m)
        assert b["bin_counts"].max() == 1
        # a one-member weighted mean (w x) / w can differ from x in the last bit (FP64)
        np.testing.assert_allclose(a["w"], b["w"], rtol=1e-9, atol=0)
        np.testing.assert_allclose(a["estimate"], b["estimate"], rtol=1e-12, atol=0)
        assert a["resampled"] == b["resampled"]
        np.testing.assert_array_equal(a["new_state"], b["new_state"])
        np.testing.assert_allclose(a["logw_out"], b["logw_out"], rtol=0, atol=1e-9)
        decisions.append(a["resampled"])
        st, lw = a["new_state"], a["logw_out"]
    assert True in decisions and False in decisions


def test_shift_of_carried_log_weights_changes_nothing():
    """Only ratios of weights matter: adding a constant to every carried log-weight leaves
    dummies, weights, the decision and the next step's log-weights unchanged."""
    seq = synth.make_sequence(48, 48, 1, MODEL9, seed=13)
    N = 400
    st = synth.initial_state(seq.gt[0], N)
    rng = np.random.default_rng(13)
    lw = -rng.exponential(2.0, size=N)
    noise = synth.make_noise(N, MODEL9.q, 13, 0)
    a = O.pcsir_step_ess(st, lw, seq.images[0], noise, 0.4, 0.5, 0.3 * N, MODEL9)
    b = O.pcsir_step_ess(st, lw + 37.25, seq.images[0], noise, 0.4, 0.5, 0.3 * N, MODEL9)
    np.testing.assert_allclose(a["dummies"], b["dummies"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a["w"], b["w"], rtol=1e-9, atol=1e-15)
    assert a["resampled"] == b["resampled"]
    np.testing.assert_allclose(a["logw_out"], b["logw_out"], rtol=0, atol=1e-9)


def _two_cell_case():
    st = np.zeros((5, 6))
    st[0] = [0.10, 0.20, 0.30, 1.10, 1.20, 1.20]
    st[1] = [0.00, 0.10, -0.10, 0.00, 0.20, 0.10]
    st[2] = [0.05, -0.05, 0.025, 0.1, 0.2, -0.1]
    st[4] = [90.0, 100.0, 110.0, 80.0, 120.0, 100.0]
    return st


def test_cell_without_weighted_members_takes_the_plain_mean():
    """A cell whose members all carry zero weight has no weighted centre of mass (0/0): it takes the
    plain mean, its members keep zero weight whatever its likelihood, and the rest of the step is
    that of the other cells alone."""
    st = _two_cell_case()
    lw = np.array([0.0, np.log(2.0), -1.0, -np.inf, -np.inf, -np.inf])
    ll_of = lambda x, y, i0: -(x - 0.2) ** 2  # finite everywhere
    res = O.pcsir_step_ess(st, lw, None, np.zeros_like(st), 0.5, 1.0, 0.0, MODEL9, lik=ll_of)
    member = res["member_bin"]
    dead = member[3]
    assert np.all(member[3:] == dead) and np.all(member[:3] != dead)
    for d in range(5):  # brute force: the plain mean of the three zero-weight members' propagated states
        mean = sum(st[d, i] + (st[d + 2, i] if d < 2 else 0.0) for i in (3, 4, 5)) / 3.0
        assert res["dummies"][d, dead] == pytest.approx(mean, rel=1e-14, abs=1e-14)
    assert np.all(np.isfinite(res["dummies"]))
    np.testing.assert_array_equal(res["w"][3:], 0.0)
    assert res["w"][:3].sum() == pytest.approx(1.0, rel=1e-14)
    assert np.all(np.isneginf(res["logw_out"][3:])) and res["logw_out"][:3].max() == 0.0


def test_dummy_depends_on_the_weight_ratios_within_its_cell_only():
    """Section 4's weighted centre of mass of a cell is unchanged when all its members' carried
    log-weights move by one constant, even far below the other cells' (here 500 and 1000 nats:
    beyond the FP32 and the FP64 exponential's range, respectively)."""
    st = _two_cell_case()
    lw = np.log(np.array([1.0, 2.0, 5.0, 0.5, 0.25, 4.0]))
    flat = lambda x, y, i0: np.zeros_like(x)
    a = O.pcsir_step_ess(st, lw, None, np.zeros_like(st), 0.5, 1.0, 0.0, MODEL9, lik=flat)
    for drop in (500.0, 1000.0):
        moved = lw.copy()
        moved[a["member_bin"] == a["member_bin"][3]] -= drop
        b = O.pcsir_step_ess(st, moved, None, np.zeros_like(st), 0.5, 1.0, 0.0, MODEL9, lik=flat)
        np.testing.assert_array_equal(a["member_bin"], b["member_bin"])
        np.testing.assert_allclose(a["dummies"], b["dummies"], rtol=1e-13, atol=1e-13)


def test_far_cell_keeps_its_weighted_mean_bruteforce():
    """A cell 1000 nats below the best one (every FP64 weight relative to the global maximum
    underflows to 0 there): its dummy is still its members' weighted mean, formed here by hand
    with weights taken relative to the cell's FIRST member (a different normaliser from the
    oracle's), and it differs from the plain mean."""
    st = _two_cell_case()
    lw = np.array([0.0, np.log(2.0), -1.0, -1000.0 + np.log(0.5), -1000.0 + np.log(0.25), -1000.0 + np.log(4.0)])
    flat = lambda x, y, i0: np.zeros_like(x)
    res = O.pcsir_step_ess(st, lw, None, np.zeros_like(st), 0.5, 1.0, 0.0, MODEL9, lik=flat)
    far = res["member_bin"][3]
    assert np.all(res["member_bin"][3:] == far) and np.all(res["member_bin"][:3] != far)
    members = (3, 4, 5)
    w = [math.exp(lw[i] - lw[3]) for i in members]  # 1, 1/2, 8
    for d in range(5):
        xs = [st[d, i] + (st[d + 2, i] if d < 2 else 0.0) for i in members]
        wmean = sum(wi * xi for wi, xi in zip(w, xs)) / sum(w)
        assert res["dummies"][d, far] == pytest.approx(wmean, rel=1e-14, abs=1e-14)
        if d == 4:
            assert abs(wmean - sum(xs) / 3.0) > 1.0  # the weights matter for this component
    # the far cell's members carry (relative) weight ~e^-1000: zero after normalisation in FP64
    np.testing.assert_array_equal(res["w"][3:], 0.0)
