"""GPU parity: the CUDA path through the C ABI against the CPU oracle on identical inputs.

Tolerances (FP32/double-float GPU arithmetic against the FP64 oracle):
  * propagated states, cells, member counts, member -> cell map: bit-exact;
  * dummies: positions 1e-9 px, other components 2.5e-7 (fixed-point sums
    round velocities and intensities to 2^-22 per particle);
  * log-likelihoods: absolute 1e-4 + 4e-7 |ll| (a few float ulps per pixel
    term, summed over the patch);
  * normalised weights: relative 1e-5 for every weight carrying mass
    (w >= 1e-3 max w), absolute 1e-5 max w below;
  * ESS and posterior mean: relative 1e-5 (plus 1e-6 absolute for
    components near zero);
  * resampling: every output is the propagated state of its reported
    ancestor; the ancestors are exactly the systematic resample of the
    integer weights the step reports (``resample_checks.exact_systematic``),
    and those weights, normalised, meet the weight tolerance against the
    oracle's; every ancestor lies in the range the oracle's weights allow
    under that tolerance (``resample_checks.oracle_band``).  The number of
    ancestors that differ from the oracle's is reported: they can differ
    only where the allowed range holds more than one particle.
"""
import numpy as np
import pytest
import torch

import resample_checks as RC
from oracle import pcsir_oracle as O
from paper_1310_5541_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 1310554100


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


KEEP_ALL = 1 | 2 | 4 | 8 | 16


def _ctx(pc, N, dtype, model, keep=KEEP_ALL, dummy="com"):
    return pc.Context(N, dtype, lik=model.lik, patch=model.patch, psf_sigma=model.sigma_psf, bg=model.bg,
                      sigma_xi=model.sigma_xi, keep=keep, dummy=dummy)


def _warm_state(seq, N, model, dtype, frames, h=None):
    """A realistic posterior cloud: the oracle filter run for a few frames."""
    st = synth.initial_state(seq.gt[0], N, dtype)
    for k in range(frames):
        nz = synth.make_noise(N, model.q, SEED + 7, k, dtype)
        u0 = synth.make_u0(SEED + 7, k)
        if h is None:
            st = O.sir_step(st, seq.images[k], nz, u0, model)["new_state"]
        else:
            st = O.pcsir_step(st, seq.images[k], nz, u0, h, model)["new_state"]
    return st


def check_weights(w_gpu, w_ref):
    wmax = w_ref.max()
    sig = w_ref >= 1e-3 * wmax
    rel = np.abs(w_gpu[sig] - w_ref[sig]) / w_ref[sig]
    assert rel.max() <= 1e-5, ("weight rel err", rel.max())
    assert np.abs(w_gpu[~sig] - w_ref[~sig]).max(initial=0.0) <= 1e-5 * wmax
    return float(rel.max())


def check_scalars(res, ref):
    est = np.array(res["estimate"])
    tol = 1e-5 * np.abs(ref["estimate"]) + 1e-6
    assert np.all(np.abs(est - ref["estimate"]) <= tol), (est, ref["estimate"])
    assert abs(res["ess"] - ref["ess"]) <= 1e-5 * ref["ess"], (res["ess"], ref["ess"])


def check_resampling(new_state, prop, anc, q, u0, ref_w, ref_anc):
    """Outputs are their ancestors' propagated states; the ancestors are exactly the systematic
    resample of the step's own integer weights q, which meet the weight tolerance against the
    oracle's; and every ancestor lies in the range the oracle's weights allow under it.
    Returns (ancestors that differ from the oracle's, outputs left open by the FP64 bound of the
    exact check, outputs whose oracle range holds more than one particle)."""
    N = anc.shape[0]
    assert anc.min() >= 0 and anc.max() < N
    np.testing.assert_array_equal(new_state, prop[:, anc])
    open_exact = RC.exact_systematic(anc, q, u0)
    qn = q.astype(np.float64) / float(q.sum())
    check_weights(qn, ref_w)
    open_band, _ = RC.oracle_band(anc, ref_w, u0, RC.weight_tolerance(ref_w))
    mism = int(np.sum(anc != ref_anc))
    assert mism <= open_band
    return mism, open_exact, open_band


def run_pcsir(pc, ctx, st_np, img_np, nz_np, u0, h):
    st = torch.from_numpy(np.ascontiguousarray(st_np)).cuda()
    pc.pcsir_step(ctx, st, torch.from_numpy(img_np).cuda(), h, torch.from_numpy(nz_np).cuda(), u0)
    torch.cuda.synchronize()
    res = ctx.last_result()
    out = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in ctx.outputs().items()}
    return st.cpu().numpy(), res, out


def run_sir(pc, ctx, st_np, img_np, nz_np, u0):
    st = torch.from_numpy(np.ascontiguousarray(st_np)).cuda()
    pc.sir_step(ctx, st, torch.from_numpy(img_np).cuda(), torch.from_numpy(nz_np).cuda(), u0)
    torch.cuda.synchronize()
    res = ctx.last_result()
    out = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in ctx.outputs().items()}
    return st.cpu().numpy(), res, out


def compare_pcsir(pc, ctx, st_np, img, nz, u0, h, model, dummy="com", return_step=False):
    ref = O.pcsir_step(st_np, img, nz, u0, h, model, dummy=dummy)
    new, res, out = run_pcsir(pc, ctx, st_np, img, nz, u0, h)
    assert res["device_error"] == 0 and res["kind"] == 1
    np.testing.assert_array_equal(out["prop_state"], ref["prop"])
    B = res["n_bins"]
    assert B == ref["bin_keys"].shape[0]
    # bins in canonical (by, bx) order
    xy = out["bin_xy"]
    order = np.lexsort((xy[0], xy[1]))
    np.testing.assert_array_equal(xy[:, order].T, ref["bin_keys"])
    np.testing.assert_array_equal(out["bin_count"][order], ref["bin_counts"])
    # member -> cell map, bit-exact
    rank = np.empty(B, np.int64)
    rank[order] = np.arange(B)
    np.testing.assert_array_equal(rank[out["particle_bin"]], ref["member_bin"])
    dum = out["dummy"][:, order]
    np.testing.assert_allclose(dum[:2], ref["dummies"][:2], rtol=0, atol=1e-9)
    np.testing.assert_allclose(dum[2:], ref["dummies"][2:], rtol=0, atol=2.5e-7)
    ll = out["bin_loglik"][order]
    assert np.all(np.abs(ll - ref["ll_bins"]) <= 1e-4 + 4e-7 * np.abs(ref["ll_bins"]))
    werr = check_weights(out["weight"], ref["w"])
    check_scalars(res, ref)
    mism, open_exact, open_band = check_resampling(new, out["prop_state"], out["ancestor"], out["qweight"], u0,
                                                   ref["w"], ref["ancestors"])
    r = dict(B=B, werr=werr, mismatches=mism, open_exact=open_exact, open_band=open_band, N=st_np.shape[1])
    return (r, new, res) if return_step else r


def compare_sir(pc, ctx, st_np, img, nz, u0, model):
    ref = O.sir_step(st_np, img, nz, u0, model)
    new, res, out = run_sir(pc, ctx, st_np, img, nz, u0)
    assert res["device_error"] == 0 and res["kind"] == 0
    np.testing.assert_array_equal(out["prop_state"], ref["prop"])
    ll = out["loglik"]
    assert np.all(np.abs(ll - ref["ll"]) <= 1e-4 + 4e-7 * np.abs(ref["ll"]))
    werr = check_weights(out["weight"], ref["w"])
    check_scalars(res, ref)
    mism, open_exact, open_band = check_resampling(new, out["prop_state"], out["ancestor"], out["qweight"], u0,
                                                   ref["w"], ref["ancestors"])
    return dict(werr=werr, mismatches=mism, open_exact=open_exact, open_band=open_band, N=st_np.shape[1])


# ---------------------------------------------------------------------------
# Single-target workload, FP64 state, 64 x 64 image, 9 x 9 patch, N = 10^4
# ---------------------------------------------------------------------------
MODEL_SMALL = synth.Model(sigma_psf=1.5, I0=100.0, bg=10.0, patch=9)


@pytest.mark.parametrize("h,dummy", [(0.5, "com"), (1.0, "com"), (0.1, "com"), (1.0, "coc"), (0.3, "coc")])
def test_pcsir_fp64_small_image(pc, h, dummy):
    seq = synth.make_sequence(64, 64, 4, MODEL_SMALL, seed=SEED + 1)
    N = 10_000
    st = _warm_state(seq, N, MODEL_SMALL, np.float64, 2, h=0.5)
    ctx = _ctx(pc, N, torch.float64, MODEL_SMALL, dummy=dummy)
    for k in (2, 3):
        nz = synth.make_noise(N, MODEL_SMALL.q, SEED + 1, k, np.float64)
        r = compare_pcsir(pc, ctx, st, seq.images[k], nz, synth.make_u0(SEED + 1, k), h, MODEL_SMALL, dummy=dummy)
        print("pcSIR-%s fp64 h=%g frame %d: %s" % (dummy, h, k, r))
        st = O.pcsir_step(st, seq.images[k], nz, synth.make_u0(SEED + 1, k), h, MODEL_SMALL,
                          dummy=dummy)["new_state"]
    ctx.close()


def test_sir_fp64_small_image(pc):
    seq = synth.make_sequence(64, 64, 3, MODEL_SMALL, seed=SEED + 2)
    N = 10_000
    st = _warm_state(seq, N, MODEL_SMALL, np.float64, 2)
    ctx = _ctx(pc, N, torch.float64, MODEL_SMALL, keep=1 | 2 | 8 | 16)
    nz = synth.make_noise(N, MODEL_SMALL.q, SEED + 2, 2, np.float64)
    r = compare_sir(pc, ctx, st, seq.images[2], nz, synth.make_u0(SEED + 2, 2), MODEL_SMALL)
    print("SIR fp64:", r)
    ctx.close()


# ---------------------------------------------------------------------------
# 512 x 512 image, 21 x 21 patch, FP32 state; several tiles and a ragged tail
# ---------------------------------------------------------------------------
MODEL_BIG = synth.Model(sigma_psf=1.5, I0=100.0, bg=10.0, patch=21)


@pytest.fixture(scope="module")
def big_case():
    seq = synth.make_sequence(512, 512, 3, MODEL_BIG, seed=SEED + 3)
    N = (1 << 18) + 777
    st = _warm_state(seq, N, MODEL_BIG, np.float32, 2, h=0.5)
    return seq, N, st


@pytest.mark.parametrize("h", [0.05, 0.25, 0.5, 2.0])
def test_pcsir_fp32_big_image(pc, big_case, h):
    seq, N, st = big_case
    ctx = _ctx(pc, N, torch.float32, MODEL_BIG)
    nz = synth.make_noise(N, MODEL_BIG.q, SEED + 3, 2, np.float32)
    r = compare_pcsir(pc, ctx, st, seq.images[2], nz, synth.make_u0(SEED + 3, 2), h, MODEL_BIG)
    print("pcSIR fp32 h=%g: %s" % (h, r))
    ctx.close()


def test_cell_table_size_does_not_change_the_step(pc, big_case):
    """The propagate/bin kernel has a small and a large shared-memory cell table, chosen per step
    from the previous step's cell count; both must give the same step bit for bit."""
    seq, N, st = big_case
    nz = torch.from_numpy(synth.make_noise(N, MODEL_BIG.q, SEED + 5, 2, np.float32)).cuda()
    img = torch.from_numpy(seq.images[2]).cuda()
    outs = []
    for prime_h in (None, 4.0, 0.03):
        ctx = _ctx(pc, N, torch.float32, MODEL_BIG)
        if prime_h is not None:  # a previous step with few (large table off) or many cells (on)
            s0 = torch.from_numpy(st).cuda()
            pc.pcsir_step(ctx, s0, img, prime_h, nz, 0.5)
            torch.cuda.synchronize()
        s1 = torch.from_numpy(st).cuda()
        pc.pcsir_step(ctx, s1, img, 0.1, nz, 0.3)
        torch.cuda.synchronize()
        o = ctx.outputs()
        order = np.lexsort((o["bin_xy"][0].cpu().numpy(), o["bin_xy"][1].cpu().numpy()))
        outs.append((s1.cpu().numpy(), o["dummy"].cpu().numpy()[:, order], o["bin_count"].cpu().numpy()[order],
                     o["weight"].cpu().numpy(), ctx.last_result()["estimate"]))
        ctx.close()
    for other in outs[1:]:
        np.testing.assert_array_equal(outs[0][0], other[0])
        np.testing.assert_array_equal(outs[0][1], other[1])
        np.testing.assert_array_equal(outs[0][2], other[2])
        # normalised weights divide by a sum accumulated with atomics: equal up to its rounding order
        np.testing.assert_allclose(outs[0][3], other[3], rtol=1e-12, atol=0)
        np.testing.assert_allclose(outs[0][4], other[4], rtol=1e-12)


@pytest.mark.parametrize("h", [0.25, 1.0])
def test_pcsir_coc_fp32_big_image(pc, big_case, h):
    """pcSIR-CoC (Section 5.4): dummies at the cells' geometric centres."""
    seq, N, st = big_case
    ctx = _ctx(pc, N, torch.float32, MODEL_BIG, dummy="coc")
    nz = synth.make_noise(N, MODEL_BIG.q, SEED + 6, 2, np.float32)
    r = compare_pcsir(pc, ctx, st, seq.images[2], nz, synth.make_u0(SEED + 6, 2), h, MODEL_BIG, dummy="coc")
    print("pcSIR-CoC fp32 h=%g: %s" % (h, r))
    ctx.close()


def test_sir_fp32_big_image(pc, big_case):
    seq, N, st = big_case
    N2 = 40_000 + 123
    st = np.ascontiguousarray(st[:, :N2])
    ctx = _ctx(pc, N2, torch.float32, MODEL_BIG, keep=1 | 2 | 8 | 16)
    nz = synth.make_noise(N2, MODEL_BIG.q, SEED + 4, 2, np.float32)
    r = compare_sir(pc, ctx, st, seq.images[2], nz, synth.make_u0(SEED + 4, 2), MODEL_BIG)
    print("SIR fp32:", r)
    ctx.close()


# ---------------------------------------------------------------------------
# The single-target workload at its full size: N = 2^24 FP32 particles, 512 x 512 image, 21 x 21
# patch, h = 0.5 px (the configuration whose throughput is measured)
# ---------------------------------------------------------------------------
N_FULL = 1 << 24
CLOUD = (0.6, 0.6, 0.15, 0.15, 5.0)  # spread of the synthetic particle cloud about the ground truth


@pytest.fixture(scope="module")
def full_case():
    seq = synth.make_sequence(512, 512, 1, MODEL_BIG, seed=SEED + 50)
    st = synth.initial_state(seq.gt[0], N_FULL, np.float32)
    st += synth.make_noise(N_FULL, CLOUD, SEED + 51, 0, np.float32)
    nz = synth.make_noise(N_FULL, MODEL_BIG.q, SEED + 52, 0, np.float32)
    return seq.images[0], st, nz, synth.make_u0(SEED + 52, 0)


def test_pcsir_full_size_workload(pc, full_case):
    """One pcSIR step at the full size, first as throughput is measured (no per-particle outputs
    kept), then with every output kept: both give the same new state bit for bit, and the kept
    outputs match the oracle's full step element by element (cells, counts and member -> cell map
    bit-exact; dummies, likelihoods, weights, N_eff and posterior mean within the parity
    tolerances; resampling properties; ancestors that differ from the oracle's counted)."""
    img, st, nz, u0 = full_case
    ctx = _ctx(pc, N_FULL, torch.float32, MODEL_BIG, keep=0)
    s = torch.from_numpy(st).cuda()
    pc.pcsir_step(ctx, s, torch.from_numpy(img).cuda(), 0.5, torch.from_numpy(nz).cuda(), u0)
    torch.cuda.synchronize()
    res0 = ctx.last_result()
    new0 = s.cpu().numpy()
    ctx.close()
    del s
    assert res0["device_error"] == 0
    ctx = _ctx(pc, N_FULL, torch.float32, MODEL_BIG)
    r, new, res = compare_pcsir(pc, ctx, st, img, nz, u0, 0.5, MODEL_BIG, return_step=True)
    ctx.close()
    print("pcSIR full size: %s" % r)
    np.testing.assert_array_equal(new, new0)
    # the weight sum meets in FP64 atomics whose order varies from run to run
    np.testing.assert_allclose(res["estimate"], res0["estimate"], rtol=1e-12, atol=0)


def test_sir_full_size_workload_sampled(pc, full_case):
    """SIR, the comparison path, on the same full-size input.  Against the oracle: the propagated
    state of every particle bit-exact, and the log-likelihoods of 4096 sampled particles one by one.
    Properties over all particles: the weights are the normalised exponentials of the step's own
    log-likelihoods, N_eff and the posterior mean are formed from them, and the resampling is
    exactly the systematic resample of the step's own integer weights (outputs are their
    ancestors' propagated states), which are the normalised weights within the tolerance."""
    img, st, nz, u0 = full_case
    ctx = _ctx(pc, N_FULL, torch.float32, MODEL_BIG, keep=1 | 2 | 8 | 16)
    new, res, out = run_sir(pc, ctx, st, img, nz, u0)
    ctx.close()
    assert res["device_error"] == 0 and res["kind"] == 0
    prop = O.propagate(st, nz)
    np.testing.assert_array_equal(out["prop_state"], prop)
    idx = np.sort(np.random.default_rng(SEED + 53).choice(N_FULL, 4096, replace=False))
    p = prop[:, idx].astype(np.float64)
    ll_ref = O.loglik(img, p[0], p[1], p[4], MODEL_BIG)
    ll = out["loglik"]
    assert np.all(np.abs(ll[idx] - ll_ref) <= 1e-4 + 4e-7 * np.abs(ll_ref))
    w = np.exp(ll - ll.max())
    w /= w.sum()
    check_weights(out["weight"], w)
    check_scalars(res, {"estimate": (prop.astype(np.float64) * w[None, :]).sum(axis=1), "ess": 1.0 / np.sum(w * w)})
    anc = out["ancestor"]
    assert anc.min() >= 0 and anc.max() < N_FULL
    np.testing.assert_array_equal(new, prop[:, anc])
    q = out["qweight"]
    check_weights(q.astype(np.float64) / float(q.sum()), w)
    open_exact = RC.exact_systematic(anc, q, u0)
    print("SIR full size: outputs left open by the FP64 bound of the exact check: %d" % open_exact)


def test_sse_likelihood_pcsir(pc):
    m = synth.Model(sigma_psf=1.16, I0=60.0, bg=10.0, patch=9, lik="sse", sigma_xi=20.0)
    seq = synth.make_sequence(64, 64, 3, m, seed=SEED + 5)
    N = 8192 + 5
    st = _warm_state(seq, N, m, np.float32, 2, h=0.5)
    ctx = _ctx(pc, N, torch.float32, m)
    nz = synth.make_noise(N, m.q, SEED + 5, 2, np.float32)
    r = compare_pcsir(pc, ctx, st, seq.images[2], nz, synth.make_u0(SEED + 5, 2), 0.5, m)
    print("pcSIR SSE:", r)
    ctx.close()


# ---------------------------------------------------------------------------
# Stand-alone likelihood and resampling entry points
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("h", [1.0, 0.5])
def test_sse_large_object_65x65(pc, h):
    """The paper's large-object regime (Section 5.3): PSF sigma 13 px, SNR 2, the Gaussian (SSE)
    likelihood over a 65 x 65 kernel, pcSIR-1x1 and pcSIR-2x2."""
    m = synth.large_object_model()
    seq = synth.make_sequence(192, 160, 3, m, seed=SEED + 30, margin=40)
    N = 20_000 + 37
    st = _warm_state(seq, N, m, np.float32, 2, h=h)
    ctx = _ctx(pc, N, torch.float32, m)
    nz = synth.make_noise(N, m.q, SEED + 30, 2, np.float32)
    r = compare_pcsir(pc, ctx, st, seq.images[2], nz, synth.make_u0(SEED + 30, 2), h, m)
    print("pcSIR SSE 65x65 h=%g: %s" % (h, r))
    ctx.close()


def test_sse_large_object_sir_65x65(pc):
    m = synth.large_object_model()
    seq = synth.make_sequence(192, 160, 3, m, seed=SEED + 31, margin=40)
    N = 3000 + 5
    st = _warm_state(seq, N, m, np.float32, 2, h=1.0)
    ctx = _ctx(pc, N, torch.float32, m, keep=1 | 2 | 8 | 16)
    nz = synth.make_noise(N, m.q, SEED + 31, 2, np.float32)
    r = compare_sir(pc, ctx, st, seq.images[2], nz, synth.make_u0(SEED + 31, 2), m)
    print("SIR SSE 65x65:", r)
    ctx.close()


def test_loglik_entry_point(pc):
    seq = synth.make_sequence(96, 80, 1, MODEL_BIG, seed=SEED + 6)
    img = seq.images[0]
    rng = np.random.default_rng(6)
    n = 3000
    x = seq.gt[1, 0] + rng.normal(size=n) * 1.5
    y = seq.gt[1, 1] + rng.normal(size=n) * 1.5
    a = 100.0 + rng.normal(size=n) * 5
    # a few positions at and beyond the border (clipped patch) and a negative intensity
    x[:4] = [0.2, 95.6, -3.0, 50.0]
    y[:4] = [0.3, 79.4, 10.0, 90.0]
    a[4] = -5.0
    ctx = _ctx(pc, 16, torch.float32, MODEL_BIG)
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    ll = pc.pcsir_loglik(ctx, t(x), t(y), t(a), t(img)).cpu().numpy()
    ref = O.loglik(img, x, y, a, MODEL_BIG)
    err = ll - ref
    assert np.abs(err).max() <= 1e-4 + 4e-7 * np.abs(ref).max()
    w = np.exp(ref - ref.max())
    sig = w >= 1e-3
    assert np.abs(err[sig] - err[sig].mean()).max() <= 1e-5
    ctx.close()


def test_resample_entry_point_exact_when_weights_are_exact(pc):
    rng = np.random.default_rng(12)
    ctx = _ctx(pc, 300_000, torch.float32, MODEL_SMALL)
    for N in (1, 7, 4096, 4097, 250_001):
        lw = np.where(rng.random(N) < 0.3, -np.inf, 0.0)
        lw[rng.integers(N)] = 0.0
        u0 = float(rng.random())
        anc = pc.pcsir_resample(ctx, torch.from_numpy(lw).cuda(), u0).cpu().numpy()
        w, _, _ = O.normalise(lw)
        np.testing.assert_array_equal(anc, O.systematic_resample(w, u0))
    ctx.close()


def test_resample_entry_point_into_an_unaligned_ancestor_array(pc):
    """The caller's ancestor array may start on any 4-byte boundary (here a slice one element into
    a buffer): the same ancestors as into an aligned array, for the context and the no-allocation
    entry points."""
    rng = np.random.default_rng(14)
    ctx = _ctx(pc, 300_000, torch.float32, MODEL_SMALL)
    for N in (2, 4097, 250_001):
        lw = torch.from_numpy(rng.normal(size=N)).cuda()
        u0 = float(rng.random())
        ref = pc.pcsir_resample(ctx, lw, u0).clone()
        buf = torch.full((N + 1,), -7, dtype=torch.int32, device="cuda")
        pc.pcsir_resample(ctx, lw, u0, out=buf[1:])
        assert torch.equal(buf[1:], ref) and int(buf[0]) == -7
        buf2 = torch.full((N + 1,), -7, dtype=torch.int32, device="cuda")
        pc.pcsir_resample_noalloc(lw, u0, out=buf2[1:])
        torch.cuda.synchronize()
        assert torch.equal(buf2[1:], ref) and int(buf2[0]) == -7
    ctx.close()


def test_resample_entry_point_random_weights(pc):
    rng = np.random.default_rng(13)
    N = 1_000_003
    ctx = _ctx(pc, N, torch.float32, MODEL_SMALL)
    lw = rng.normal(size=N) * 2.0
    u0 = float(rng.random())
    anc = pc.pcsir_resample(ctx, torch.from_numpy(lw).cuda(), u0).cpu().numpy()
    w, _, _ = O.normalise(lw)
    ref = O.systematic_resample(w, u0)
    copies = np.bincount(anc, minlength=N)
    assert copies.sum() == N and np.all(np.diff(anc) >= 0)
    assert np.all(copies >= np.floor(N * w - 1e-3)) and np.all(copies <= np.ceil(N * w + 1e-3))
    mism = int(np.sum(anc != ref))
    # the library's weights: log-weights rounded to 2^-32 (relative weight error <= 2^-33), a
    # double-float exponential, integers of N 2^s <= 2^61 (absolute 2^-42 of the largest here)
    tol = 1e-9 * w + 1e-12 * w.max()
    open_band, width = RC.oracle_band(anc, w, u0, tol)
    print("resample mismatches %d of %d; outputs with more than one allowed ancestor %d" % (mism, N, open_band))
    assert mism <= open_band
    ctx.close()


# ---------------------------------------------------------------------------
# Degenerate and edge cases
# ---------------------------------------------------------------------------
def test_single_particle(pc):
    seq = synth.make_sequence(32, 32, 1, MODEL_SMALL, seed=SEED + 8)
    st = synth.initial_state(seq.gt[0], 1, np.float32)
    nz = synth.make_noise(1, MODEL_SMALL.q, SEED + 8, 0, np.float32)
    ctx = _ctx(pc, 1, torch.float32, MODEL_SMALL)
    r = compare_pcsir(pc, ctx, st, seq.images[0], nz, 0.3, 0.5, MODEL_SMALL)
    assert r["B"] == 1
    compare_sir(pc, ctx, st, seq.images[0], nz, 0.3, MODEL_SMALL)
    ctx.close()


def test_one_particle_per_bin_matches_sir_on_gpu(pc):
    """Section 4.2 on the GPU: with tiny cells every bin holds one particle, the dummies are
    the particles themselves and the log-likelihoods equal SIR's bit for bit."""
    seq = synth.make_sequence(64, 64, 3, MODEL_SMALL, seed=SEED + 9)
    N = 5000
    st = _warm_state(seq, N, MODEL_SMALL, np.float32, 2)
    st = st + np.random.default_rng(9).normal(size=st.shape).astype(np.float32) * np.float32(0.01)
    nz = synth.make_noise(N, MODEL_SMALL.q, SEED + 9, 2, np.float32)
    ctx = _ctx(pc, N, torch.float32, MODEL_SMALL)
    _, res_p, out_p = run_pcsir(pc, ctx, st, seq.images[2], nz, 0.4, 1e-5)
    assert res_p["n_bins"] == N and np.all(out_p["bin_count"] == 1)
    ll_p = out_p["bin_loglik"][out_p["particle_bin"]]
    w_p = out_p["weight"]
    _, res_s, out_s = run_sir(pc, ctx, st, seq.images[2], nz, 0.4)
    np.testing.assert_array_equal(ll_p, out_s["loglik"])
    # weights below e^-87 are 0 on the per-particle path (float exponent range) and are 0 as
    # integer weights on both paths
    np.testing.assert_allclose(w_p, out_s["weight"], rtol=1e-6, atol=1e-12 * w_p.max())
    np.testing.assert_allclose(res_p["estimate"], res_s["estimate"], rtol=1e-6)
    ctx.close()


def test_patch_clipped_at_image_corner(pc):
    m = MODEL_SMALL
    seq = synth.make_sequence(40, 40, 1, m, seed=SEED + 10, start=(2.0, 1.5), vmax=0.1, margin=0)
    N = 3000
    st = synth.initial_state(seq.gt[0], N, np.float64)
    nz = synth.make_noise(N, m.q, SEED + 10, 0, np.float64)
    ctx = _ctx(pc, N, torch.float64, m)
    compare_pcsir(pc, ctx, st, seq.images[0], nz, 0.7, 0.5, m)
    compare_sir(pc, ctx, st, seq.images[0], nz, 0.7, m)
    ctx.close()


def test_all_particles_in_one_coarse_bin(pc):
    seq = synth.make_sequence(64, 64, 1, MODEL_SMALL, seed=SEED + 11)
    N = 20000
    st = synth.initial_state(seq.gt[0], N, np.float32)
    nz = (synth.make_noise(N, MODEL_SMALL.q, SEED + 11, 0, np.float32) * np.float32(0.01)).astype(np.float32)
    ctx = _ctx(pc, N, torch.float32, MODEL_SMALL)
    r = compare_pcsir(pc, ctx, st, seq.images[0], nz, 0.2, 8.0, MODEL_SMALL)
    assert r["B"] <= 4
    ctx.close()


def test_nonfinite_state_is_flagged(pc):
    seq = synth.make_sequence(32, 32, 1, MODEL_SMALL, seed=SEED + 12)
    N = 100
    st = synth.initial_state(seq.gt[0], N, np.float32)
    st[0, 5] = np.nan
    nz = synth.make_noise(N, MODEL_SMALL.q, SEED + 12, 0, np.float32)
    ctx = _ctx(pc, N, torch.float32, MODEL_SMALL)
    t = torch.from_numpy(np.ascontiguousarray(st)).cuda()
    pc.pcsir_step(ctx, t, torch.from_numpy(seq.images[0]).cuda(), 0.5, torch.from_numpy(nz).cuda(), 0.5)
    torch.cuda.synchronize()
    assert ctx.last_result()["device_error"] & pc.DERR_RANGE
    # the context stays usable
    st[0, 5] = st[0, 4]
    compare_pcsir(pc, ctx, st, seq.images[0], nz, 0.5, 0.5, MODEL_SMALL)
    ctx.close()


@pytest.mark.parametrize("comp,value", [(2, np.inf), (3, -np.inf), (4, np.nan), (2, 2.0e9), (3, 20000.0),
                                        (4, -5000.0), (0, 3.0e9)])
def test_out_of_range_component_is_flagged(pc, comp, value):
    """A state component that is not finite, of magnitude 10^9 or more, or (velocities and
    intensity) 2^12 or more away from particle 0's value, outside what the fixed-point sums
    represent (biased by 2^12 below it and 3 2^12 above), raises the range flag; the context
    stays usable."""
    seq = synth.make_sequence(32, 32, 1, MODEL_SMALL, seed=SEED + 13)
    N = 4096 + 8
    st = synth.initial_state(seq.gt[0], N, np.float32)
    nz = np.zeros((5, N), np.float32)
    bad = st.copy()
    bad[comp, 4100] = np.float32(value)
    ctx = _ctx(pc, N, torch.float32, MODEL_SMALL)
    t = torch.from_numpy(np.ascontiguousarray(bad)).cuda()
    pc.pcsir_step(ctx, t, torch.from_numpy(seq.images[0]).cuda(), 0.5, torch.from_numpy(nz).cuda(), 0.5)
    torch.cuda.synchronize()
    assert ctx.last_result()["device_error"] & pc.DERR_RANGE, (comp, value)
    compare_pcsir(pc, ctx, st, seq.images[0], nz, 0.5, 0.5, MODEL_SMALL)
    ctx.close()


def test_host_side_argument_errors(pc):
    ctx = _ctx(pc, 100, torch.float32, MODEL_SMALL)
    st = torch.zeros(5, 100, device="cuda")
    img = torch.zeros(16, 16, device="cuda")
    with pytest.raises(pc.PcsirError) as e:
        pc.pcsir_step(ctx, st, img, 0.0, st.clone(), 0.5)
    assert e.value.status == pc.EINVAL
    with pytest.raises(pc.PcsirError) as e:
        pc.pcsir_step(ctx, st, img, 0.5, st.clone(), 1.0)
    assert e.value.status == pc.EINVAL
    big = torch.zeros(5, 101, device="cuda")
    with pytest.raises(pc.PcsirError) as e:
        pc.pcsir_step(ctx, big, img, 0.5, big.clone(), 0.5)
    assert e.value.status == pc.ERANGE
    ctx.close()


def test_graph_capture_of_steps(pc):
    """A step is capturable in a CUDA graph and replays to the same result."""
    seq = synth.make_sequence(64, 64, 1, MODEL_SMALL, seed=SEED + 13)
    N = 50_000
    st0 = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).cuda()
    nz = torch.from_numpy(synth.make_noise(N, MODEL_SMALL.q, SEED + 13, 0, np.float32)).cuda()
    img = torch.from_numpy(seq.images[0]).cuda()
    ctx = _ctx(pc, N, torch.float32, MODEL_SMALL, keep=0)
    st = st0.clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pc.pcsir_step(ctx, st, img, 0.5, nz, 0.25)  # warm-up outside capture
    torch.cuda.synchronize()
    ref = st.clone()
    g = torch.cuda.CUDAGraph()
    st.copy_(st0)
    with torch.cuda.graph(g, stream=s):
        pc.pcsir_step(ctx, st, img, 0.5, nz, 0.25)
    st.copy_(st0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(st, ref)
    ctx.close()
