"""Plain FP64 CPU oracle of one SIR / pcSIR filter step (Demirel et al., arXiv 1310.5541).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code with
the CUDA library; the two meet only through the seeded inputs of
``paper_1310_5541_gb300.synth``.

The oracle follows the paper's pseudocode step by step with whole-array numpy
operations (a sort, a cumulative sum and a binary search serve as library
primitives) and no fusion or reordering:

* Algorithm 1 (SIR): draw from the proposal, weight by the likelihood,
  normalise, effective sample size, resample.
* Algorithm 2 (pcSIR): draw from the proposal, assign to equal-size bins,
  one dummy particle per bin at the mean state of its members, likelihood of
  the dummy only, copy of the dummy's weight to every member, then as SIR.

Readings of points the paper leaves open:

* Proposal = dynamics (bootstrap), so the ratio p(x|x')/pi(x|x') in
  Algorithm 1/2 equals one.
* Dynamics (Section 5.1, nearly-constant velocity, unit frame time):
  ``x += vx + e_x; y += vy + e_y; vx += e_vx; vy += e_vy; I0 += e_I`` with the
  noise supplied by the caller.  The propagation runs in the state's own
  precision (FP32 or FP64), exactly as the GPU path must, because it decides
  the integer bins.
* Bins: square cells of edge h over position only (Section 4.1), aligned so
  that h = 1 cells are image pixels centred on integers:
  ``b = floor((x + 0.5) / h)`` evaluated in the state precision.
* Dummy weight (Algorithm 2, weight update): ``w_k^i = w_{k-1}^i L(x_dum)`` for
  every member i, which is the only reading for which one particle per bin
  gives back SIR exactly (Section 4.2).  The dummy state is the mean of all
  state components, weighted by w_{k-1} (Section 4 forms the centre of mass
  from both the states and their weights); after resampling the weights are
  uniform and this is the plain mean of Algorithm 2.  The weighted mean of a
  cell is a ratio of two sums over that cell, so each cell's weights are
  taken relative to the largest carried weight among its own members: a cell
  lying any distance below the others keeps its weighted mean.
* Likelihood patch S_x: a fixed odd P x P block of pixels centred on the pixel
  nearest the evaluated position, ``c = floor(x + 0.5)``; pixels outside the
  image contribute nothing.  The PSF is point-sampled at pixel centres
  (Eq. object) with intensity ``max(I0, 0)``.
* Likelihood terms (Eq. likelihood):
    - "sse": the paper's Gaussian form ``-(Z - I)^2 / (2 sigma_xi^2)``.
    - "poisson": the Poisson log-likelihood ratio against a perfect fit,
      ``z log(lambda / z) - (lambda - z)`` (0 at lambda = z, ``-lambda`` at
      z = 0).  Like the paper's SSE term it is 0 for a perfectly predicted
      pixel, so pixels outside S_x count as predicted; for two evaluations
      with the same patch it differs from the full Poisson log-pmf by a
      constant.
* Resampling: systematic, with one uniform u0 shared by all outputs,
  ``U_i = (i + u0) / N`` and ``s(i) = min{l : C_l > U_i}`` where C is the
  inclusive cumulative sum of the normalised weights in particle order; at
  every step (``sir_step``, ``pcsir_step``), or only when N_eff < N_thr
  (``sir_step_ess``, ``pcsir_step_ess``: Algorithm 1's test, with the weights
  carried to the next step when it fails).
* Estimate: posterior mean before resampling.
"""
from __future__ import annotations

import numpy as np

# State component order (Section 5.1): position, velocity, intensity.
X, Y, VX, VY, I0 = range(5)


# ----------------------------------------------------------------------------
# Algorithm 1/2, sampling step: the proposal is the NCV dynamics (Sec. 5.1)
# ----------------------------------------------------------------------------
def propagate(state: np.ndarray, noise: np.ndarray) -> np.ndarray:
    """Nearly-constant-velocity transition in the state's own precision.

    state, noise: [5, N] arrays of one dtype (float32 or float64).
    """
    assert state.dtype == noise.dtype
    out = np.empty_like(state)
    out[X] = (state[X] + state[VX]) + noise[X]
    out[Y] = (state[Y] + state[VY]) + noise[Y]
    out[VX] = state[VX] + noise[VX]
    out[VY] = state[VY] + noise[VY]
    out[I0] = state[I0] + noise[I0]
    return out


# ----------------------------------------------------------------------------
# Algorithm 2, binning: equal cells over position, each particle put in its cell
# ----------------------------------------------------------------------------
def bin_coords(x: np.ndarray, y: np.ndarray, h: float):
    """Integer cell coordinates (bx, by) of positions, in the positions' precision."""
    t = x.dtype.type
    hh = t(h)
    half = t(0.5)
    bx = np.floor((x + half) / hh)
    by = np.floor((y + half) / hh)
    return bx.astype(np.int64), by.astype(np.int64)


def segment(bx: np.ndarray, by: np.ndarray):
    """Group particles by cell.

    Returns (keys [B, 2] in ascending (by, bx) order, member -> bin index [N],
    member counts [B]).
    """
    if bx.size == 0:
        return np.zeros((0, 2), np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64)
    pairs = np.stack([by, bx], axis=1)
    keys, inverse, counts = np.unique(pairs, axis=0, return_inverse=True, return_counts=True)
    keys = keys[:, ::-1].copy()  # columns (bx, by)
    return keys, inverse.reshape(-1), counts


def cell_relative_weights(prior_logw, member_bin: np.ndarray, n_bins: int) -> np.ndarray:
    """Prior weights of the centre of mass, each relative to its own bin's largest (Section 4).

    w_i = exp(log w_i - M_b) with M_b = max of log w over the members of i's
    bin b.  The factor exp(-M_b) is common to every term of bin b's weighted
    sums, so the weighted mean is that of the weights exp(log w_i) themselves;
    taking it per bin keeps every bin's largest weight at 1, so no bin's
    weights underflow because another bin lies far above it.  Members of zero
    weight (log w = -inf) get 0; so do all members of a bin that has only such
    members.  FP64.
    """
    lw = np.asarray(prior_logw, np.float64)
    M = np.full(n_bins, -np.inf)
    np.maximum.at(M, member_bin, lw)
    Mi = M[member_bin]
    out = np.zeros_like(lw)
    live = ~np.isneginf(lw)
    out[live] = np.exp(lw[live] - Mi[live])
    return out


def dummies(state: np.ndarray, member_bin: np.ndarray, n_bins: int, prior_w=None) -> np.ndarray:
    """Dummy particle of each bin: the (prior-weighted) mean of every state component.

    Algorithm 2 (the dummy is the mean state of the bin's members); Section 4
    (the centre of mass uses the members' weights as well).  ``prior_w`` may
    carry any positive factor common to one bin's members (it cancels in the
    bin's ratio).  A bin none of whose members carries weight has no weighted
    mean; it takes the plain mean (its members' weights stay zero whatever its
    likelihood).  FP64.
    """
    s = state.astype(np.float64)
    if prior_w is None:
        wts = np.ones(s.shape[1])
    else:
        wts = np.asarray(prior_w, dtype=np.float64)
    den = np.bincount(member_bin, weights=wts, minlength=n_bins)
    out = np.empty((s.shape[0], n_bins))
    with np.errstate(invalid="ignore", divide="ignore"):  # 0/0 only where the plain mean replaces it
        for d in range(s.shape[0]):
            out[d] = np.bincount(member_bin, weights=wts * s[d], minlength=n_bins) / den
    empty = den == 0  # no member carries weight: the weighted mean is 0/0, the plain mean is taken
    if empty.any():
        cnt = np.bincount(member_bin, minlength=n_bins)
        for d in range(s.shape[0]):
            out[d, empty] = (np.bincount(member_bin, weights=s[d], minlength=n_bins) / np.maximum(cnt, 1))[empty]
    return out


# ----------------------------------------------------------------------------
# Eq. (object) and Eq. (likelihood): Gaussian-PSF image model over patch S_x
# ----------------------------------------------------------------------------
def _patch_lambda(x, y, i0, sigma, bg, P):
    """Predicted intensities on each evaluation's P x P patch (FP64).

    Returns (pixel x coords [n,P], pixel y coords [n,P], lambda [n,P,P]).
    """
    R = P // 2
    cx = np.floor(x + 0.5)
    cy = np.floor(y + 0.5)
    off = np.arange(-R, R + 1, dtype=np.float64)
    px = cx[:, None] + off[None, :]
    py = cy[:, None] + off[None, :]
    r2 = (px[:, None, :] - x[:, None, None]) ** 2 + (py[:, :, None] - y[:, None, None]) ** 2
    lam = np.maximum(i0, 0.0)[:, None, None] * np.exp(-r2 / (2.0 * sigma * sigma)) + bg
    return px, py, lam


def loglik(image: np.ndarray, x, y, i0, model, chunk: int = 4096) -> np.ndarray:
    """Log-likelihood of each evaluated position (x, y, I0) against one image (FP64).

    Sum over the P x P patch of the per-pixel term chosen by ``model.lik``;
    pixels outside the image are skipped.
    """
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    i0 = np.asarray(i0, np.float64)
    Hh, Ww = image.shape
    img = image.astype(np.float64)
    P = model.patch
    out = np.empty(x.shape[0])
    for s0 in range(0, x.shape[0], chunk):
        sl = slice(s0, s0 + chunk)
        px, py, lam = _patch_lambda(x[sl], y[sl], i0[sl], model.sigma_psf, model.bg, P)
        pxi = px.astype(np.int64)
        pyi = py.astype(np.int64)
        inx = (pxi >= 0) & (pxi < Ww)
        iny = (pyi >= 0) & (pyi < Hh)
        inside = iny[:, :, None] & inx[:, None, :]
        z = img[np.clip(pyi, 0, Hh - 1)[:, :, None], np.clip(pxi, 0, Ww - 1)[:, None, :]]
        if model.lik == "poisson":
            with np.errstate(divide="ignore", invalid="ignore"):
                zlog = np.where(z > 0, z * np.log(lam / np.where(z > 0, z, 1.0)), 0.0)
            term = zlog - (lam - z)
        elif model.lik == "sse":
            term = -((z - lam) ** 2) / (2.0 * model.sigma_xi ** 2)
        else:
            raise ValueError(model.lik)
        out[sl] = np.where(inside, term, 0.0).sum(axis=(1, 2))
    return out


# ----------------------------------------------------------------------------
# Algorithm 1, weight normalisation, effective sample size, resampling
# ----------------------------------------------------------------------------
def normalise(logw: np.ndarray):
    """w_i = exp(logw_i) / sum_j exp(logw_j), computed with the maximum subtracted."""
    m = np.max(logw)
    wt = np.exp(logw - m)
    T = wt.sum()
    return wt / T, m, T


def ess(w: np.ndarray) -> float:
    """N_eff = 1 / sum_j w_j^2 (Algorithm 1)."""
    return 1.0 / np.sum(w * w)


def systematic_resample(w: np.ndarray, u0: float) -> np.ndarray:
    """Indices s(i) with Pr[s(i) = l] = w_l, systematic scheme (Algorithm 1 resampling).

    U_i = (i + u0) / N over the normalised inclusive cumulative weights C;
    s(i) is the first l with C_l > U_i.
    """
    N = w.shape[0]
    C = np.cumsum(w) / np.sum(w)
    U = (np.arange(N, dtype=np.float64) + u0) / N
    s = np.searchsorted(C, U, side="right")
    return np.minimum(s, N - 1)


def posterior_mean(w: np.ndarray, state: np.ndarray) -> np.ndarray:
    """State estimate: sum_i w_i x_i with normalised weights (before resampling)."""
    return (state.astype(np.float64) * w[None, :]).sum(axis=1)


# ----------------------------------------------------------------------------
# One full step of each filter
# ----------------------------------------------------------------------------
def _add_logw(prior_logw, ll):
    """log w_k = log w_{k-1} + log p(z | x): a particle of zero prior weight keeps zero weight."""
    prior = np.asarray(prior_logw, np.float64)
    return np.where(np.isneginf(prior), -np.inf, prior + ll)


def _lik_fn(image, model):
    return lambda x, y, i0: loglik(image, x, y, i0, model)


def sir_step(state, image, noise, u0, model, lik=None, prior_logw=None):
    """Algorithm 1, one time step k, with resampling at every step.

    ``lik`` (optional) replaces the image likelihood: a function
    (x, y, I0) -> log-likelihood, used by the linear-Gaussian tests.
    Returns a dict with the propagated state, per-particle log-likelihood,
    normalised weights, ESS, posterior mean, ancestors and the new state.
    """
    lik = lik or _lik_fn(image, model)
    prop = propagate(state, noise)
    ll = lik(prop[X].astype(np.float64), prop[Y].astype(np.float64), prop[I0].astype(np.float64))
    logw = ll if prior_logw is None else _add_logw(prior_logw, ll)
    w, m, T = normalise(logw)
    anc = systematic_resample(w, u0)
    return dict(prop=prop, ll=ll, w=w, max_logw=m, ess=ess(w),
                estimate=posterior_mean(w, prop), ancestors=anc, new_state=np.ascontiguousarray(prop[:, anc]))


def cell_centres(keys: np.ndarray, h: float) -> np.ndarray:
    """Geometric centres of cells (bx, by): the cell [b h - 1/2, (b + 1) h - 1/2) has its
    centre at (b + 1/2) h - 1/2 (Section 5.4, pcSIR-CoC).  FP64, [2, B]."""
    k = np.asarray(keys, np.float64)
    return np.stack([(k[:, 0] + 0.5) * h - 0.5, (k[:, 1] + 0.5) * h - 0.5])


def pcsir_step(state, image, noise, u0, h, model, lik=None, prior_logw=None, dummy="com"):
    """Algorithm 2, one time step k, with resampling at every step.

    ``dummy``: "com" places each dummy at the centre of mass of its members
    (pcSIR-CoM); "coc" at the geometric centre of its cell for the binned
    components (x, y), the members' mean for the others (pcSIR-CoC,
    Section 5.4).

    Returns the same keys as ``sir_step`` plus the bins (keys [B, 2] as
    (bx, by) in ascending (by, bx) order, counts), the member -> bin map, the
    dummies [5, B] and the dummies' log-likelihoods.
    """
    lik = lik or _lik_fn(image, model)
    prop = propagate(state, noise)
    bx, by = bin_coords(prop[X], prop[Y], h)
    keys, member, counts = segment(bx, by)
    prior_w = None if prior_logw is None else cell_relative_weights(prior_logw, member, keys.shape[0])
    dum = dummies(prop, member, keys.shape[0], prior_w)
    if dummy == "coc":
        dum[[X, Y]] = cell_centres(keys, h)
    elif dummy != "com":
        raise ValueError(dummy)
    ll_bins = lik(dum[X], dum[Y], dum[I0])
    ll = ll_bins[member]
    logw = ll if prior_logw is None else _add_logw(prior_logw, ll)
    w, m, T = normalise(logw)
    anc = systematic_resample(w, u0)
    return dict(prop=prop, bin_keys=keys, bin_counts=counts, member_bin=member,
                dummies=dum, ll_bins=ll_bins, ll=ll, w=w, max_logw=m, ess=ess(w),
                estimate=posterior_mean(w, prop), ancestors=anc, new_state=np.ascontiguousarray(prop[:, anc]))


def _ess_branch(r, logw_prev, ess_min):
    """Algorithm 1/2's resampling branch: resample only when N_eff < ess_min.

    Adds 'resampled' and 'logw_out' (the log-weights the next step starts
    from: zeros after resampling, else this step's log-weights minus their
    maximum) and replaces 'new_state' by the propagated state when the step
    does not resample.
    """
    logw = r["ll"] if logw_prev is None else _add_logw(logw_prev, r["ll"])
    r["logw"] = logw
    r["resampled"] = bool(r["ess"] < ess_min)
    if r["resampled"]:
        r["logw_out"] = np.zeros_like(logw)
    else:
        r["logw_out"] = logw - np.max(logw)
        r["ancestors"] = np.arange(logw.shape[0])
        r["new_state"] = np.ascontiguousarray(r["prop"])
    return r


def sir_step_ess(state, logw_prev, image, noise, u0, ess_min, model, lik=None):
    """Algorithm 1 with its threshold test: weights carry the previous step's
    log-weights (``logw_prev``, None for uniform), w_k = w_{k-1} p(z|x_k), and
    the particles are resampled only when N_eff < ess_min."""
    r = sir_step(state, image, noise, u0, model, lik=lik, prior_logw=logw_prev)
    return _ess_branch(r, logw_prev, ess_min)


def pcsir_step_ess(state, logw_prev, image, noise, u0, h, ess_min, model, lik=None, dummy="com"):
    """Algorithm 2 with its threshold test: the dummy of a bin is the mean of
    its members weighted by w_{k-1} (Section 4), every member's weight is
    multiplied by the dummy's likelihood, and the particles are resampled only
    when N_eff < ess_min."""
    r = pcsir_step(state, image, noise, u0, h, model, lik=lik, prior_logw=logw_prev, dummy=dummy)
    return _ess_branch(r, logw_prev, ess_min)


def run_filter(kind, seq_images, gt0, N, noise_fn, u0_fn, model, h=None, dtype=np.float64,
               n_frames=None, lik_fn=None):
    """Run SIR or pcSIR over a sequence; returns the per-frame estimates [K, 5]."""
    st = np.empty((5, N), dtype=dtype)
    for d in range(5):
        st[d] = gt0[d]
    K = len(seq_images) if n_frames is None else n_frames
    est = []
    for k in range(K):
        lik = None if lik_fn is None else lik_fn(k)
        if kind == "sir":
            r = sir_step(st, seq_images[k], noise_fn(k), u0_fn(k), model, lik=lik)
        else:
            r = pcsir_step(st, seq_images[k], noise_fn(k), u0_fn(k), h, model, lik=lik)
        st = r["new_state"]
        est.append(r["estimate"])
    return np.array(est)


# ----------------------------------------------------------------------------
# Closed-form comparators used only to pin the oracle
# ----------------------------------------------------------------------------
def ncv_kalman(x0, q, r, zs):
    """Kalman filter for the NCV model with observation z = (x, y) + N(0, r^2 I).

    Exact posterior mean/covariance of the linear-Gaussian case, used to pin
    the particle filters.  Returns lists of means [5] and covariances [5, 5]
    after each update.
    """
    F = np.eye(5)
    F[X, VX] = 1.0
    F[Y, VY] = 1.0
    Q = np.diag(np.asarray(q, np.float64) ** 2)
    Hm = np.zeros((2, 5))
    Hm[0, X] = 1.0
    Hm[1, Y] = 1.0
    Rm = np.eye(2) * r * r
    m = np.asarray(x0, np.float64).copy()
    Pc = np.zeros((5, 5))
    means, covs = [], []
    for z in zs:
        m = F @ m
        Pc = F @ Pc @ F.T + Q
        S = Hm @ Pc @ Hm.T + Rm
        K = Pc @ Hm.T @ np.linalg.inv(S)
        m = m + K @ (np.asarray(z) - Hm @ m)
        Pc = (np.eye(5) - K @ Hm) @ Pc
        means.append(m.copy())
        covs.append(Pc.copy())
    return means, covs
