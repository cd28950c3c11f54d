"""Counter-based process noise: the CPU oracle of the in-kernel noise of ``pcsir_step_philox``.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this module:
only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm
use it.  It shares no code with the CUDA library.

The noise of the nearly-constant-velocity transition (Section 5.1: e_d ~ N(0, q_d^2) for the five
state components) is normally drawn on the host and passed in; a step may instead draw it from a
counter-based generator, which both sides implement from its published definition so that the
oracle reproduces the kernel's noise bit for bit:

* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
  SC 2011): a 128-bit counter and a 64-bit key, ten rounds of two 32 x 32 -> 64-bit products with
  the published multipliers, the cross-over and xor of the round keys, which advance by the
  published Weyl constants.
* Counter of particle i in frame k: (i mod 2^32, i div 2^32, k, j) with j = 0, 1; key: the 64-bit
  seed as (low, high) words.  The eight 32-bit outputs r_0..r_7 feed three Box-Muller pairs
  (r_0, r_1), (r_2, r_3), (r_4, r_5): normals z_0..z_4 (z_5, r_6, r_7 unused).
* Uniforms from the top 24 bits: u1 = (r >> 8 + 1) 2^-24 in (0, 1], u2 = (r >> 8) 2^-24 in [0, 1).
* Box-Muller: z = sqrt(-2 log u1) (cos 2 pi u2, sin 2 pi u2).  So that both sides round alike,
  every step is an IEEE single-precision +, -, x, / or square root (each correctly rounded, no
  fused multiply-add) or an exact bit operation: log u1 = e ln 2 + log m with the exponent e read
  from the bits and m in [sqrt(1/2), sqrt(2)), log m = 2 atanh(s), s = (m - 1) / (m + 1), by its
  series to s^9; the angle reduced exactly to a quadrant of 4 u2 and a fraction folded to
  [0, 1/2], whose sine and cosine come from their Taylor series to x^9 and x^10.
* Noise e_d = float32(q_d) z_d, the propagation's FP32 state precision.
"""
from __future__ import annotations

import numpy as np

_M32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)

F = np.float32


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with ten rounds on uint32 arrays (counter words c0..c3, key words k0, k1)."""
    c = [np.asarray(x, np.uint32).copy() for x in (c0, c1, c2, c3)]
    k0 = np.asarray(k0, np.uint32).copy()
    k1 = np.asarray(k1, np.uint32).copy()
    for rnd in range(10):
        p0 = c[0].astype(np.uint64) * PHILOX_M0
        p1 = c[2].astype(np.uint64) * PHILOX_M1
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & _M32).astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & _M32).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        if rnd < 9:  # round keys advance modulo 2^32
            k0 = ((k0.astype(np.uint64) + np.uint64(PHILOX_W0)) & _M32).astype(np.uint32)
            k1 = ((k1.astype(np.uint64) + np.uint64(PHILOX_W1)) & _M32).astype(np.uint32)
    return c


def uniform_open0(r):
    """(r >> 8 + 1) 2^-24 in (0, 1], exact in float32."""
    return ((np.asarray(r, np.uint32) >> np.uint32(8)) + np.uint32(1)).astype(F) * F(2.0 ** -24)


def uniform_open1(r):
    """(r >> 8) 2^-24 in [0, 1), exact in float32."""
    return (np.asarray(r, np.uint32) >> np.uint32(8)).astype(F) * F(2.0 ** -24)


# series coefficients, rounded to float32 once
_L3, _L5, _L7, _L9 = F(1.0 / 3.0), F(1.0 / 5.0), F(1.0 / 7.0), F(1.0 / 9.0)
_LN2 = F(np.log(2.0))
_SQRT2 = F(np.sqrt(2.0))
_S3, _S5, _S7, _S9 = F(-1.0 / 6.0), F(1.0 / 120.0), F(-1.0 / 5040.0), F(1.0 / 362880.0)
_C2, _C4, _C6, _C8, _C10 = (F(-1.0 / 2.0), F(1.0 / 24.0), F(-1.0 / 720.0), F(1.0 / 40320.0),
                           F(-1.0 / 3628800.0))
_HALF_PI = F(np.pi / 2.0)


def log_f32(u):
    """log u for float32 u in (0, 1] (normal numbers), in the operation order the kernel uses."""
    u = np.asarray(u, F)
    bits = u.view(np.uint32)
    e = (bits >> np.uint32(23)).astype(np.int32) - 127
    m = ((bits & np.uint32(0x7FFFFF)) | np.uint32(0x3F800000)).view(F)
    big = m > _SQRT2
    m = np.where(big, m * F(0.5), m).astype(F)
    e = np.where(big, e + 1, e)
    s = ((m - F(1.0)) / (m + F(1.0))).astype(F)
    s2 = (s * s).astype(F)
    p = _L9
    p = (p * s2 + _L7).astype(F)
    p = (p * s2 + _L5).astype(F)
    p = (p * s2 + _L3).astype(F)
    a = (s * s2).astype(F)
    a = (a * p).astype(F)
    a = (s + a).astype(F)
    logm = (a + a).astype(F)
    return (e.astype(F) * _LN2 + logm).astype(F)


def sincos_quarter_f32(x):
    """sin and cos of x in [0, pi/4] by their Taylor series (to x^9 and x^10), float32."""
    x = np.asarray(x, F)
    x2 = (x * x).astype(F)
    p = _S9
    p = (p * x2 + _S7).astype(F)
    p = (p * x2 + _S5).astype(F)
    p = (p * x2 + _S3).astype(F)
    sn = (x + (x * x2).astype(F) * p).astype(F)
    c = _C10
    c = (c * x2 + _C8).astype(F)
    c = (c * x2 + _C6).astype(F)
    c = (c * x2 + _C4).astype(F)
    c = (c * x2 + _C2).astype(F)
    cs = (F(1.0) + x2 * c).astype(F)
    return sn, cs


def sincos_turn_f32(u):
    """cos(2 pi u) and sin(2 pi u) for u in [0, 1): quadrant q = floor(4 u) and fraction f = 4 u - q
    (both exact), f folded to [0, 1/2] by the complement, angle f pi/2."""
    u = np.asarray(u, F)
    q4 = (u * F(4.0)).astype(F)
    quad = np.floor(q4).astype(F)
    f = (q4 - quad).astype(F)
    fold = f > F(0.5)
    g = np.where(fold, F(1.0) - f, f).astype(F)
    sn, cs = sincos_quarter_f32((g * _HALF_PI).astype(F))
    ca = np.where(fold, sn, cs)  # cos and sin of the angle within the quadrant
    sa = np.where(fold, cs, sn)
    qi = quad.astype(np.int32)
    c = np.select([qi == 0, qi == 1, qi == 2], [ca, -sa, -ca], sa).astype(F)
    s = np.select([qi == 0, qi == 1, qi == 2], [sa, ca, -sa], -ca).astype(F)
    return c, s


def box_muller_f32(r_a, r_b):
    """Two normals from two 32-bit outputs."""
    u1 = uniform_open0(r_a)
    u2 = uniform_open1(r_b)
    rad = np.sqrt((log_f32(u1) * F(-2.0)).astype(F)).astype(F)
    c, s = sincos_turn_f32(u2)
    return (rad * c).astype(F), (rad * s).astype(F)


def normals5(idx, frame: int, seed: int) -> np.ndarray:
    """The five standard normals of particles ``idx`` in ``frame``: float32 [5, len(idx)]."""
    idx = np.asarray(idx, np.uint64)
    c0 = (idx & _M32).astype(np.uint32)
    c1 = (idx >> np.uint64(32)).astype(np.uint32)
    c2 = np.full(idx.shape, frame & 0xFFFFFFFF, np.uint32)
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32((seed >> 32) & 0xFFFFFFFF)
    r = philox4x32_10(c0, c1, c2, np.zeros(idx.shape, np.uint32), k0, k1)
    r += philox4x32_10(c0, c1, c2, np.ones(idx.shape, np.uint32), k0, k1)
    z0, z1 = box_muller_f32(r[0], r[1])
    z2, z3 = box_muller_f32(r[2], r[3])
    z4, _ = box_muller_f32(r[4], r[5])
    return np.stack([z0, z1, z2, z3, z4])


def process_noise(N: int, q, seed: int, frame: int) -> np.ndarray:
    """Noise e_d = float32(q_d) z_d of the N particles in ``frame``: float32 [5, N]."""
    z = normals5(np.arange(N, dtype=np.uint64), frame, seed)
    return (np.asarray(q, np.float64).astype(F)[:, None] * z).astype(F)
