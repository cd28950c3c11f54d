"""GPU parity of the ESS-thresholded steps (pcsir_step_ess, sir_step_ess) against the oracle.

Each GPU step is compared with the oracle's step on the same input state and carried
log-weights (fixed point, 2^-32 units, on both sides); a sequence continues from the ORACLE's new
state and log-weights, so that no oracle input comes from the GPU:
  * propagated states, cells, counts, member -> cell map: bit-exact;
  * prior-weighted dummies: the GPU forms sum w_i and sum w_i (s_i - r_b) in FP32 over at most
    m = min(ESS_ROUND = 8192, members) terms per block before adding them in FP64, with
    w_i = exp(logw_i - M_b) in FP32, M_b the cell's largest log-weight rounded down (exponent
    within 2 max|logw| + 1 of zero: relative error <= (2 max|logw| + 4) u, u = 2^-24, with the
    exponential's own; one more rounding per product).  The weighted mean r_b + S / W is then
    within (2 m + 4 (2 + max|logw|)) u max|d| of the exact one, d the members' offsets s_i - r_b;
    the test takes that bound from the data;
  * dummy log-likelihoods: against the oracle's at the oracle's dummies, within
    1e-4 + 4e-7 |ll| (as for pcsir_step) plus the dummy bound times twice the likelihood's slope
    there (central differences of the oracle's likelihood);
  * weights, ESS, posterior mean and the carried log-weights: against the oracle's own, within
    what log-likelihood errors of at most delta (the largest of those tolerances) allow: each
    weight within a factor e^(2 delta), N_eff within e^(4 delta), the mean within
    (e^(2 delta) - 1) sum w |x - mean|; and, as properties of the GPU's own values, its weights,
    N_eff and mean formed from its own log-likelihoods (relative 1e-5);
  * the decision: N_eff < ess_min, asserted unless the oracle's N_eff lies within that
    tolerance of ess_min;
  * resampled steps: every output is its ancestor's propagated state, copies are floor or ceil
    of N w, the carried log-weights are zero; other steps keep the propagated state and the
    identity ancestors.
"""
import numpy as np
import pytest
import torch

from oracle import pcsir_oracle as O
from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 1310554300
SCALE = 4294967296.0
U = 2.0 ** -24
ESS_ROUND = 8192
KEEP_ALL = 1 | 2 | 4 | 8
INT64_MIN = np.iinfo(np.int64).min


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


def _model():
    # the paper's Gaussian likelihood (sigma_xi = 20): N_eff stays a sizeable fraction of N,
    # so both branches of the test occur within a few steps
    return synth.Model(sigma_psf=1.5, I0=100.0, bg=10.0, patch=9, lik="sse", sigma_xi=20.0)


def _ctx(pc, N, model, keep=KEEP_ALL, dummy="com", dtype=torch.float32):
    return pc.Context(N, dtype, lik=model.lik, patch=model.patch, psf_sigma=model.sigma_psf, bg=model.bg,
                      sigma_xi=model.sigma_xi, keep=keep, dummy=dummy)


def _lw_float(lwq):
    out = lwq.astype(np.float64) / SCALE
    out[lwq == INT64_MIN] = -np.inf
    return out


def _run(pc, ctx, kind, st_np, lwq, img, nz, u0, h, ess_min):
    st = torch.from_numpy(np.ascontiguousarray(st_np)).cuda()
    lw = torch.from_numpy(np.ascontiguousarray(lwq)).cuda()
    dimg, dnz = torch.from_numpy(img).cuda(), torch.from_numpy(nz).cuda()
    if kind == "pcsir":
        pc.pcsir_step_ess(ctx, st, lw, dimg, h, dnz, u0, ess_min)
    else:
        pc.sir_step_ess(ctx, st, lw, dimg, dnz, u0, ess_min)
    torch.cuda.synchronize()
    res = ctx.last_result()
    out = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in ctx.outputs().items()}
    return st.cpu().numpy(), lw.cpu().numpy(), res, out


def _dummy_bound(prop, member, order_keys, h, lw, anchors):
    """Per-bin bound on |weighted mean (GPU) - weighted mean (exact)| per component."""
    B = order_keys.shape[0]
    counts = np.bincount(member, minlength=B)
    m = np.minimum(counts, ESS_ROUND).astype(np.float64)
    ref = np.empty((5, prop.shape[1]))
    for a in range(2):
        ref[a] = order_keys[member, a].astype(np.float32) * np.float32(h) - np.float32(0.5)
    for c in range(3):
        ref[2 + c] = anchors[c]
    d = np.abs(prop.astype(np.float64) - ref)
    dmax = np.zeros((5, B))
    for c in range(5):
        np.maximum.at(dmax[c], member, d[c])
    finite = lw[np.isfinite(lw)]
    lwmax = np.abs(finite).max() if finite.size else 0.0
    return (2.0 * m + 4.0 * (2.0 + lwmax)) * U * dmax + 1e-12


def _quantise_lw(logw):
    """Carried log-weights in the library's fixed point (units of 2^-32; INT64_MIN = no weight)."""
    out = np.full(logw.shape, INT64_MIN, np.int64)
    fin = np.isfinite(logw)
    out[fin] = np.rint(logw[fin] * SCALE).astype(np.int64)
    return out


def _ll_slope(img, dum, model, e=1e-3):
    """|d ll / d x|, |d ll / d y|, |d ll / d I0| of the oracle's likelihood at the oracle's dummies,
    by central differences with step e (much larger than any dummy displacement bounded here, so
    that a patch switching pixels within the displacement shows as a large slope)."""
    x, y, a = dum[0], dum[1], dum[4]
    gx = (O.loglik(img, x + e, y, a, model) - O.loglik(img, x - e, y, a, model)) / (2 * e)
    gy = (O.loglik(img, x, y + e, a, model) - O.loglik(img, x, y - e, a, model)) / (2 * e)
    ga = (O.loglik(img, x, y, a + e, model) - O.loglik(img, x, y, a - e, model)) / (2 * e)
    return np.abs(gx), np.abs(gy), np.abs(ga)


def _compare_step(pc, ctx, kind, st_np, lwq, img, nz, u0, h, ess_min, model, dummy="com"):
    """One GPU step against the oracle's step on the same input; returns the ORACLE's next state and
    carried log-weights (in the library's fixed point), so that a sequence feeds both sides with
    oracle values only, and the GPU's result."""
    lw_prev = _lw_float(lwq)
    new, lw_new, res, out = _run(pc, ctx, kind, st_np, lwq, img, nz, u0, h, ess_min)
    assert res["device_error"] == 0
    N = st_np.shape[1]
    if kind == "pcsir":
        ref = O.pcsir_step_ess(st_np, lw_prev, img, nz, u0, h, ess_min, model, dummy=dummy)
    else:
        ref = O.sir_step_ess(st_np, lw_prev, img, nz, u0, ess_min, model)
    prop = ref["prop"]
    np.testing.assert_array_equal(out["prop_state"], prop)
    if kind == "pcsir":
        B = res["n_bins"]
        assert B == ref["bin_keys"].shape[0]
        xy = out["bin_xy"]
        order = np.lexsort((xy[0], xy[1]))
        np.testing.assert_array_equal(xy[:, order].T, ref["bin_keys"])
        np.testing.assert_array_equal(out["bin_count"][order], ref["bin_counts"])
        rank = np.empty(B, np.int64)
        rank[order] = np.arange(B)
        member = ref["member_bin"]
        np.testing.assert_array_equal(rank[out["particle_bin"]], member)
        dum = out["dummy"][:, order]
        anchors = st_np[2:5, 0].astype(np.float32)  # particle 0's input values (the GPU's anchors)
        bound = _dummy_bound(prop, member, ref["bin_keys"], h, lw_prev, anchors)
        # a cell none of whose members carries weight takes the plain mean of its members on both
        # sides: the GPU's from its exact fixed-point sums
        weighted = np.bincount(member, weights=np.isfinite(lw_prev).astype(np.float64), minlength=B) > 0
        bound[:2, ~weighted] = 1e-9
        bound[2:, ~weighted] = 2.5e-7
        want = ref["dummies"]
        if dummy == "coc":  # the cells' geometric centres, exact on both sides
            bound[:2] = 1e-12
        err = np.abs(dum - want)
        assert np.all(err <= bound), ("dummies", (err / bound).max())
        # the dummies' log-likelihoods against the oracle's at the oracle's dummies: the likelihood
        # tolerance plus the dummies' displacement bound times twice the likelihood's slope there
        ll_ref = ref["ll_bins"]
        gx, gy, ga = _ll_slope(img, want, model)
        tol_bins = 1e-4 + 4e-7 * np.abs(ll_ref) + 2.0 * (gx * bound[0] + gy * bound[1] + ga * bound[4])
        ll_bins = out["bin_loglik"][order]
        assert np.all(np.abs(ll_bins - ll_ref) <= tol_bins), ("dummy loglik", np.abs(ll_bins - ll_ref).max())
        ll, tol = ll_bins[member], tol_bins[member]
        ll_want = ll_ref[member]
    else:
        ll, ll_want = out["loglik"], ref["ll"]
        tol = 1e-4 + 4e-7 * np.abs(ll_want)
        assert np.all(np.abs(ll - ll_want) <= tol)
    fin = np.isfinite(lw_prev)
    delta = float(tol[fin].max()) if fin.any() else 0.0
    # independent: the oracle's own weights, N_eff and posterior mean, within what log-likelihood
    # errors of at most delta allow (each normalised weight within a factor e^(2 delta))
    w_ref, ess_ref, est_ref = ref["w"], ref["ess"], ref["estimate"]
    rw = np.expm1(2.0 * delta) + 1e-5
    wmax = w_ref.max()
    sig = w_ref >= 1e-3 * wmax
    assert np.abs(out["weight"][sig] / w_ref[sig] - 1.0).max() <= rw
    assert np.all(np.abs(out["weight"][~sig] - w_ref[~sig]) <= rw * 1e-3 * wmax)
    assert abs(res["ess"] / ess_ref - 1.0) <= np.expm1(4.0 * delta) + 1e-5, (res["ess"], ess_ref)
    # sum_i (w'_i - w_i) x_i = sum_i (w'_i - w_i)(x_i - est): within rw sum_i w_i |x_i - est|
    spread = (w_ref[None, :] * np.abs(prop.astype(np.float64) - est_ref[:, None])).sum(axis=1)
    assert np.all(np.abs(np.array(res["estimate"]) - est_ref) <= rw * spread + 1e-5 * np.abs(est_ref) + 1e-6)
    # properties of the GPU's own values: its weights are the normalised exponentials of its carried
    # plus new log-weights, and its N_eff and estimate are formed from them
    logw = lw_prev + ll
    wg = np.exp(logw - logw[fin].max()) if fin.any() else np.zeros(N)
    wg /= wg.sum()
    sig = wg >= 1e-3 * wg.max()
    assert np.abs(out["weight"][sig] / wg[sig] - 1.0).max() <= 1e-5
    ess_g = 1.0 / np.sum(wg * wg)
    assert abs(res["ess"] - ess_g) <= 1e-5 * ess_g
    est_g = (prop.astype(np.float64) * wg[None, :]).sum(axis=1)
    assert np.all(np.abs(np.array(res["estimate"]) - est_g) <= 1e-5 * np.abs(est_g) + 1e-6)
    # the decision: N_eff < ess_min, unless the oracle's N_eff lies within the tolerance of ess_min
    near = ess_min > 0 and abs(ess_ref / ess_min - 1.0) <= np.expm1(4.0 * delta) + 1e-5
    if not near:
        assert res["resampled"] == (ess_ref < ess_min), (ess_ref, ess_min)
        assert ref["resampled"] == res["resampled"]
    anc = out["ancestor"]
    if res["resampled"]:
        np.testing.assert_array_equal(lw_new, np.zeros(N, np.int64))
        np.testing.assert_array_equal(new, prop[:, anc])
        copies = np.bincount(anc, minlength=N)
        nw = N * out["weight"]
        assert np.all(copies >= np.floor(nw - 1e-4)) and np.all(copies <= np.ceil(nw + 1e-4))
    else:
        np.testing.assert_array_equal(new, prop)
        np.testing.assert_array_equal(anc, np.arange(N))
        carried = _lw_float(lw_new)
        ok = np.isfinite(ref["logw_out"])
        np.testing.assert_array_equal(np.isfinite(carried), ok)
        # log-weights relative to the maximum: each particle's own error plus that of the maximum
        assert np.all(np.abs(carried[ok] - ref["logw_out"][ok]) <= tol[ok] + delta + 2.0 ** -31)
        assert lw_new[ok].max() == 0
    res["gpu_logw"] = lw_new
    return ref["new_state"], _quantise_lw(ref["logw_out"]), res


@pytest.mark.parametrize("kind", ["pcsir", "sir"])
def test_ess_steps_match_oracle_over_a_sequence(pc, kind):
    m = _model()
    seq = synth.make_sequence(64, 64, 6, m, seed=SEED)
    N = 20000 if kind == "pcsir" else 4096
    ctx = _ctx(pc, N, m)
    st = synth.initial_state(seq.gt[0], N, np.float32)
    lwq = np.zeros(N, np.int64)
    decisions = []
    for k in range(6):
        nz = synth.make_noise(N, m.q, SEED + 1, k, np.float32)
        u0 = synth.make_u0(SEED + 1, k)
        # N_eff / N runs 0.02-0.27 on this sequence: 0.1 N alternates the two branches
        st, lwq, res = _compare_step(pc, ctx, kind, st, lwq, seq.images[k], nz, u0, 0.5, 0.1 * N, m)
        decisions.append(res["resampled"])
    ctx.close()
    print(kind, "resampled:", decisions)
    assert True in decisions and False in decisions


def test_ess_pcsir_ragged_large_cells_and_coc(pc):
    """N not a multiple of the tile or chunk, several tiles, large cells and the CoC dummy."""
    m = _model()
    seq = synth.make_sequence(64, 64, 3, m, seed=SEED + 5)
    N = 3 * 4096 + 777
    for dummy, h in (("com", 2.0), ("coc", 0.75)):
        ctx = _ctx(pc, N, m, dummy=dummy)
        st = synth.initial_state(seq.gt[0], N, np.float32)
        lwq = np.zeros(N, np.int64)
        for k in range(3):
            nz = synth.make_noise(N, m.q, SEED + 6, k, np.float32)
            u0 = synth.make_u0(SEED + 6, k)
            st, lwq, res = _compare_step(pc, ctx, "pcsir", st, lwq, seq.images[k], nz, u0, h, 0.0, m, dummy=dummy)
            assert not res["resampled"]
        ctx.close()


def test_ess_threshold_limits(pc):
    """ess_min > N resamples every step with uniform carried weights; ess_min = 0 never does."""
    m = _model()
    seq = synth.make_sequence(64, 64, 2, m, seed=SEED + 9)
    N = 8192
    ctx = _ctx(pc, N, m)
    for ess_min, expect in ((N + 1.0, True), (0.0, False)):
        st = synth.initial_state(seq.gt[0], N, np.float32)
        lwq = np.zeros(N, np.int64)
        for k in range(2):
            nz = synth.make_noise(N, m.q, SEED + 10, k, np.float32)
            st, lwq, res = _compare_step(pc, ctx, "pcsir", st, lwq, seq.images[k], nz, synth.make_u0(SEED + 10, k),
                                         0.5, ess_min, m)
            assert res["resampled"] is expect
    ctx.close()


def test_ess_zero_weight_particles(pc):
    """INT64_MIN marks a particle of zero weight: it adds nothing to its cell's centre of mass,
    gets no weight, and stays at INT64_MIN while the step does not resample.  Every member of the
    three smallest cells is among them: those cells take their plain mean."""
    m = _model()
    seq = synth.make_sequence(64, 64, 1, m, seed=SEED + 12)
    N = 5000
    ctx = _ctx(pc, N, m)
    st = synth.initial_state(seq.gt[0], N, np.float32)
    rng = np.random.default_rng(SEED)
    lwq = (-rng.exponential(1.5, N) * SCALE).astype(np.int64)
    nz = synth.make_noise(N, m.q, SEED + 13, 0, np.float32)
    prop = O.propagate(st, nz)
    _, member, counts = O.segment(*O.bin_coords(prop[0], prop[1], 0.5))
    empty = np.argsort(counts, kind="stable")[:3]
    dead = np.union1d(rng.choice(np.arange(N), 300, replace=False), np.flatnonzero(np.isin(member, empty)))
    lwq[dead] = INT64_MIN
    live = np.setdiff1d(np.arange(N), dead)
    lwq[live[np.argmax(lwq[live])]] = 0
    _, _, res = _compare_step(pc, ctx, "pcsir", st, lwq, seq.images[0], nz, 0.3, 0.5, 0.0, m)
    assert np.all(res["gpu_logw"][dead] == INT64_MIN)
    ctx.close()


def test_ess_step_in_a_cuda_graph(pc):
    m = _model()
    seq = synth.make_sequence(64, 64, 1, m, seed=SEED + 14)
    N = 6000
    ctx = _ctx(pc, N, m)
    st0 = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).cuda()
    nz = torch.from_numpy(synth.make_noise(N, m.q, SEED + 15, 0, np.float32)).cuda()
    img = torch.from_numpy(seq.images[0]).cuda()
    s = torch.cuda.Stream()
    st, lw = st0.clone(), torch.zeros(N, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        pc.pcsir_step_ess(ctx, st, lw, img, 0.5, nz, 0.4, 0.0, stream=s)
    torch.cuda.synchronize()
    ref_st, ref_lw = st.clone(), lw.clone()
    g = torch.cuda.CUDAGraph()
    st.copy_(st0)
    lw.zero_()
    with torch.cuda.graph(g, stream=s):
        pc.pcsir_step_ess(ctx, st, lw, img, 0.5, nz, 0.4, 0.0, stream=s)
    st.copy_(st0)
    lw.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    # without resampling the state is the propagated state; the log-weights agree to the
    # FP32 rounding of the weighted centres of mass
    assert torch.equal(st, ref_st)
    assert (lw - ref_lw).abs().max().item() <= 1e-5 * SCALE
    ctx.close()


def test_ess_argument_errors(pc):
    m = _model()
    N = 1024
    ctx = _ctx(pc, N, m)
    st = torch.zeros(5, N, device="cuda")
    img = torch.zeros(16, 16, device="cuda")
    lw = torch.zeros(N, dtype=torch.int64, device="cuda")
    with pytest.raises(pc.PcsirError):
        pc.pcsir_step_ess(ctx, st, lw, img, 0.5, st, 0.3, float("nan"))
    with pytest.raises(pc.PcsirError):
        pc.pcsir_step_ess(ctx, st, lw, img, 0.0, st, 0.3, 10.0)
    ctx.close()
    ctx64 = _ctx(pc, N, m, dtype=torch.float64)
    st64 = torch.zeros(5, N, dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcsirError) as ei:
        ctx64_lib = pc.lib
        r = ctx64_lib.pcsir_step_ess(ctx64.handle, pc._ptr(st64), pc._ptr(lw), N, pc._ptr(img), 16, 16, 0.5,
                                     pc._ptr(st64), 0.3, 10.0, None, None)
        if r != pc.OK:
            ctx64._raise(r)
    assert ei.value.status == -6  # PCSIR_ENOTSUP
    ctx64.close()


def test_sir_ess_always_resampling_is_sir_step_bit_for_bit(pc):
    """With N_thr > N every step resamples, and the SIR step with carried (uniform) weights forms the
    same integer weights as sir_step: states, ancestors and scalars agree bit for bit."""
    m = _model()
    seq = synth.make_sequence(64, 64, 3, m, seed=SEED + 40)
    N = 3 * 4096 + 5
    a = _ctx(pc, N, m)
    b = _ctx(pc, N, m)
    sa = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).cuda()
    sb = sa.clone()
    lw = torch.zeros(N, dtype=torch.int64, device="cuda")
    for k in range(3):
        nz = torch.from_numpy(synth.make_noise(N, m.q, SEED + 41, k, np.float32)).cuda()
        img = torch.from_numpy(seq.images[k]).cuda()
        u0 = synth.make_u0(SEED + 41, k)
        pc.sir_step(a, sa, img, nz, u0)
        pc.sir_step_ess(b, sb, lw, img, nz, u0, N + 1.0)
        torch.cuda.synchronize()
        ra, rb = a.last_result(), b.last_result()
        assert torch.equal(sa, sb)
        assert torch.equal(a.outputs()["ancestor"], b.outputs()["ancestor"])
        # the blocks' partial sums meet in FP64 atomics, whose order varies from run to run
        assert abs(ra["ess"] - rb["ess"]) <= 1e-12 * ra["ess"]
        np.testing.assert_allclose(rb["estimate"], ra["estimate"], rtol=1e-12, atol=0)
        assert rb["resampled"] and int(lw.abs().max().item()) == 0
    a.close()
    b.close()


@pytest.mark.parametrize("N", [1, 3, 4095, 4097])
@pytest.mark.parametrize("kind", ["pcsir", "sir"])
def test_ess_small_and_ragged_sizes(pc, kind, N):
    m = _model()
    seq = synth.make_sequence(48, 48, 2, m, seed=SEED + 50)
    ctx = _ctx(pc, N, m)
    st = synth.initial_state(seq.gt[0], N, np.float32)
    lwq = np.zeros(N, np.int64)
    for k in range(2):
        nz = synth.make_noise(N, m.q, SEED + 51, k, np.float32)
        # k = 0 keeps the particles (threshold 0), k = 1 resamples (threshold above N)
        st, lwq, res = _compare_step(pc, ctx, kind, st, lwq, seq.images[k], nz, synth.make_u0(SEED + 51, k), 0.5,
                                     0.0 if k == 0 else N + 1.0, m)
        assert res["resampled"] == (k == 1)
    ctx.close()
