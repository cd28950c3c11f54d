"""CPU pins of the resampling checks the GPU parity tests use (tests/resample_checks.py).

The exact check is compared with systematic resampling computed in exact rational arithmetic
(pure Python, small N), and both checks must reject the mistakes they exist to catch: a wrong u0,
one block of outputs shifted by one particle, a swapped pair of ancestors.
"""
from fractions import Fraction

import numpy as np
import pytest

import resample_checks as RC
from oracle import pcsir_oracle as O


def _exact_rational(q, u0):
    """s(i) = first j with C_j > (i + u0) T / N, in exact rationals."""
    C = np.cumsum(q).tolist()
    N, T = len(q), C[-1]
    u = Fraction(u0)
    out, j = [], 0
    for i in range(N):
        U = (i + u) * T / N
        while C[j] <= U:
            j += 1
        out.append(j)
    return np.array(out, np.int64)


@pytest.mark.parametrize("N,seed", [(1, 1), (7, 2), (3000, 3), (5003, 4)])
def test_exact_check_accepts_the_rational_systematic_resample(N, seed):
    rng = np.random.default_rng(seed)
    q = rng.integers(0, 1 << 40, size=N).astype(np.int64)
    q[rng.random(N) < 0.3] = 0
    q[rng.integers(N)] = 1 << 41
    u0 = float(rng.random())
    anc = _exact_rational(q, u0)
    assert RC.exact_systematic(anc, q, u0) == 0


def test_exact_check_rejects_planted_mistakes():
    rng = np.random.default_rng(9)
    N = 4096 * 3 + 17
    q = rng.integers(1, 1 << 36, size=N).astype(np.int64)
    u0 = 0.37
    anc = _exact_rational(q, u0)
    wrong_u0 = _exact_rational(q, 0.87)
    shifted = anc.copy()
    shifted[4096:8192] = np.minimum(shifted[4096:8192] + 1, N - 1)
    swapped = anc.copy()
    k = int(np.flatnonzero(np.diff(anc) > 0)[10])
    swapped[k], swapped[k + 1] = swapped[k + 1], swapped[k]
    for bad in (wrong_u0, shifted, swapped):
        assert np.any(bad != anc)
        with pytest.raises(AssertionError):
            RC.exact_systematic(bad, q, u0)


def test_oracle_band_accepts_the_oracle_and_rejects_a_shift():
    rng = np.random.default_rng(10)
    N = 20_000
    w, _, _ = O.normalise(rng.normal(size=N) * 2.0)
    u0 = 0.61
    anc = O.systematic_resample(w, u0)
    n_open, width = RC.oracle_band(anc, w, u0, 1e-9 * w)
    assert n_open <= 5 and width < 1e-2
    # weights perturbed within the tolerance: still inside the allowed range
    w2 = w * (1.0 + 1e-9 * rng.uniform(-1, 1, N))
    RC.oracle_band(O.systematic_resample(w2 / w2.sum(), u0), w, u0, 2e-9 * w)
    # outputs shifted by one particle over a block: outside it
    bad = anc.copy()
    bad[1000:3000] = np.minimum(bad[1000:3000] + 1, N - 1)
    with pytest.raises(AssertionError):
        RC.oracle_band(bad, w, u0, 1e-9 * w)
