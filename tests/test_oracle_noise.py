"""Pins of the counter-based noise oracle (oracle/noise_oracle.py) against what fixes it from outside:
Philox4x32-10's published known-answer vectors, the logarithm, sine and cosine against the FP64
library functions, and the Box-Muller normals' distribution against the standard normal."""
import numpy as np
import pytest
from scipy import stats

from oracle import noise_oracle as NO


def _philox(c, k):
    r = NO.philox4x32_10(*[np.array([x], np.uint32) for x in c], np.uint32(k[0]), np.uint32(k[1]))
    return tuple(int(x[0]) for x in r)


def test_philox_published_known_answers():
    """The known-answer vectors distributed with the generator's reference implementation."""
    assert _philox((0, 0, 0, 0), (0, 0)) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    assert _philox((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF)) == (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)
    assert _philox((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0)) == (
        0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)


def test_uniforms_are_exact_and_in_range():
    r = np.array([0, 255, 256, 0xFFFFFFFF], np.uint32)
    np.testing.assert_array_equal(NO.uniform_open0(r), np.array([1, 1, 2, 2 ** 24], np.float64) * 2.0 ** -24)
    np.testing.assert_array_equal(NO.uniform_open1(r), np.array([0, 0, 1, 2 ** 24 - 1], np.float64) * 2.0 ** -24)


def _ulp(x):
    return np.spacing(np.abs(np.asarray(x, np.float32))).astype(np.float64)


def test_log_within_two_ulp_of_the_library():
    u = np.concatenate([np.arange(1, 1 << 16, dtype=np.float64) * 2.0 ** -24,
                        np.random.default_rng(1).random(200_000), [1.0, 0.5, 2.0 ** -24]]).astype(np.float32)
    got = NO.log_f32(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    assert np.all(np.abs(got - ref) <= 2.0 * _ulp(ref) + 1e-12)
    assert NO.log_f32(np.float32(1.0)) == 0.0


def test_sine_and_cosine_within_two_ulp_of_the_library():
    u = np.concatenate([np.arange(1 << 16, dtype=np.float64) / (1 << 16), [0.25, 0.5, 0.75, 0.125]]).astype(
        np.float32)
    c, s = NO.sincos_turn_f32(u)
    ang = 2.0 * np.pi * u.astype(np.float64)
    for got, ref in ((c, np.cos(ang)), (s, np.sin(ang))):
        # absolute error relative to the unit circle: the angle 2 pi u itself is exact here, the
        # reduction to a quadrant is exact, and the series' truncation is below 2e-9
        assert np.max(np.abs(got.astype(np.float64) - ref)) <= 3.0 * 2.0 ** -24
    # exact special angles
    assert (c[-4], s[-4]) == (0.0, 1.0) and (c[-3], s[-3]) == (-1.0, 0.0) and (c[-2], s[-2]) == (0.0, -1.0)
    np.testing.assert_allclose(c * c + s * s, 1.0, atol=4e-7)


def test_normals_follow_the_standard_normal():
    z = NO.normals5(np.arange(400_000, dtype=np.uint64), 7, 12345)
    for d in range(5):
        zd = z[d].astype(np.float64)
        assert abs(zd.mean()) < 5.0 / np.sqrt(zd.size)
        assert abs(zd.var() - 1.0) < 8.0 * np.sqrt(2.0 / zd.size)
        assert stats.kstest(zd, "norm").pvalue > 1e-4
    c = np.corrcoef(z.astype(np.float64))
    assert np.max(np.abs(c - np.eye(5))) < 5.0 / np.sqrt(z.shape[1])


def test_noise_is_a_function_of_particle_frame_and_seed():
    q = (0.5, 0.5, 0.1, 0.1, 1.0)
    a = NO.process_noise(1000, q, 99, 3)
    np.testing.assert_array_equal(NO.process_noise(10, q, 99, 3), a[:, :10])
    np.testing.assert_array_equal(NO.normals5(np.array([777], np.uint64), 3, 99)[:2, 0] * np.float32(0.5),
                                  a[:2, 777])
    assert not np.array_equal(NO.process_noise(10, q, 99, 4), a[:, :10])
    assert not np.array_equal(NO.process_noise(10, q, 98, 3), a[:, :10])
    # the components' spreads are the given standard deviations
    big = NO.process_noise(200_000, q, 5, 0)
    np.testing.assert_allclose(big.std(axis=1), q, rtol=0.01)


@pytest.mark.parametrize("planted", ["cos_sign", "log_coefficient"])
def test_a_planted_mistake_fails_a_pin(planted, monkeypatch):
    """A wrong sign in the quadrant table or a wrong series coefficient is caught by the pins above."""
    if planted == "cos_sign":
        real = NO.sincos_turn_f32
        monkeypatch.setattr(NO, "sincos_turn_f32", lambda u: (lambda cs: (np.abs(cs[0]), cs[1]))(real(u)))
        with pytest.raises(AssertionError):
            test_sine_and_cosine_within_two_ulp_of_the_library()
    else:
        monkeypatch.setattr(NO, "_L5", np.float32(1.0 / 6.0))
        with pytest.raises(AssertionError):
            test_log_within_two_ulp_of_the_library()
