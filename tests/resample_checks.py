"""Checks of a GPU step's systematic resampling (Algorithm 1/2 resampling step), shared by the
GPU parity tests.

Two checks replace a budget of ancestors allowed to differ from the oracle's:

* ``exact_systematic``: a property of the GPU's own values.  The step reports the integer
  weights q_j it resampled with (PCSIR_KEEP_QWEIGHTS); with C_j = q_0 + ... + q_j (exact
  integers) output i must take the first j with C_j > (i + u0) C_{N-1} / N.  The bound is
  formed here in FP64, whose error is derived below, so the ancestor of every output is fixed
  exactly except where some C_j lies within that error of the bound (counted and returned).
  A wrong u0, a shifted tile offset or a lost carry between tiles fails this check.
* ``oracle_band``: parity with the oracle.  The oracle's normalised weights, each moved by at
  most the weight tolerance the parity tests assert, bound every cumulative weight; output i's
  ancestor must lie among the particles those bounds allow.  Returns how many outputs allow
  more than one ancestor (the only outputs where the GPU may differ from the oracle).
"""
import numpy as np

# |(i + u0) * (T / N) in FP64 - exact| <= 4.5 * 2^-53 * T <= 4.5 * 2^8 for T <= 2^61 (four
# roundings: T to double, the quotient, i + u0 and the product); the GPU's 64.64 map truncates
# Delta and U0 by at most 2^-64 each, i.e. (N + 1) 2^-64 < 1 in total, and may lower the floor by
# one where the exact bound is an integer.  4096 covers both with a wide margin.
FP64_BAND = 4096.0


def exact_systematic(anc, q, u0):
    """Assert that ancestors ``anc`` are the systematic resample over integer weights ``q``.

    Returns the number of outputs whose ancestor the FP64 bound leaves open (expected 0 or a
    handful); every other output must match exactly, and those must lie in their open range.
    """
    anc = np.asarray(anc, np.int64)
    q = np.asarray(q, np.int64)
    N = q.shape[0]
    assert anc.shape[0] == N
    assert np.all(q >= 0)
    C = np.cumsum(q)  # exact: sum q <= 2^61
    T = int(C[-1])
    assert 0 < T <= (1 << 61)
    U = (np.arange(N, dtype=np.float64) + u0) * (float(T) / N)
    lo = np.floor(U - FP64_BAND).astype(np.int64)
    hi = np.floor(U + FP64_BAND).astype(np.int64)
    s_lo = np.minimum(np.searchsorted(C, lo, side="right"), N - 1)
    s_hi = np.minimum(np.searchsorted(C, hi, side="right"), N - 1)
    bad = np.flatnonzero((anc < s_lo) | (anc > s_hi))
    assert bad.size == 0, ("ancestors not the systematic resample of the step's own integer weights",
                           bad[:8], anc[bad[:8]], s_lo[bad[:8]], s_hi[bad[:8]], bad.size)
    return int(np.sum(s_lo != s_hi))


def weight_tolerance(w_ref, rel=1e-5, floor_frac=1e-3):
    """Per-weight tolerance of the parity tests: relative ``rel`` for weights >= floor_frac max w,
    absolute rel * max w below."""
    wmax = w_ref.max()
    return np.where(w_ref >= floor_frac * wmax, rel * w_ref, rel * wmax)


def oracle_band(anc, w_ref, u0, tol):
    """Assert that every ancestor is allowed by the oracle's weights moved by at most ``tol``.

    With |w'_j - w_j| <= tol_j the cumulative weights satisfy |C'_j - C_j| <= E_j = sum_{k<=j}
    tol_k, so output i (bound U_i = (i + u0) / N) takes some j with C_j + E_j > U_i and
    C_{j-1} - E_{j-1} <= U_i.  Returns (outputs with more than one allowed ancestor, mean width
    of the allowed range)."""
    anc = np.asarray(anc, np.int64)
    w = np.asarray(w_ref, np.float64)
    N = w.shape[0]
    s = w.sum()
    C = np.cumsum(w) / s
    E = np.cumsum(np.asarray(tol, np.float64)) / s + 4.0 * N * np.finfo(np.float64).eps
    U = (np.arange(N, dtype=np.float64) + u0) / N
    lo = np.minimum(np.searchsorted(C + E, U, side="right"), N - 1)
    hi = np.minimum(np.searchsorted(np.maximum.accumulate(C - E), U, side="right"), N - 1)
    bad = np.flatnonzero((anc < lo) | (anc > hi))
    assert bad.size == 0, ("ancestor outside the oracle's allowed range", bad[:8], anc[bad[:8]], lo[bad[:8]],
                           hi[bad[:8]], bad.size)
    return int(np.sum(hi > lo)), float(np.mean(hi - lo))
