"""Pins of the 3D oracle (CPU only).

* the voxel loop: the vectorised likelihood against a plain loop over a
  small volume, including voxels outside it;
* reduction to 2D: one z slice with the object in it (P_z = 1, z = 0)
  gives exactly the 2D oracle's likelihood, whose own pins hold;
* scipy's Poisson log-pmf: differences between positions sharing the patch;
* cells against a per-particle loop in FP32;
* one particle per cell: pcSIR equals SIR bit for bit (Section 4.2);
* convergence of pcSIR's estimate to SIR's as the cells shrink.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import pcsir3_oracle as O3
from oracle import pcsir_oracle as O2
from paper_1310_5541_gb300 import synth


def _vol(seed, W=14, H=12, D=9, pos=(6.3, 5.8, 4.4)):
    rng = np.random.default_rng(seed)
    lam = synth.render3(W, H, D, *pos, 100.0, 10.0, 1.5, 3.0)
    return rng.poisson(lam).astype(np.float32)


def test_loglik_matches_voxel_loop():
    m = O3.Model3(patch_xy=5, patch_z=3)
    vol = _vol(1)
    D, H, W = vol.shape
    pts = [(6.3, 5.8, 4.4, 100.0), (0.6, 11.2, 8.9, 80.0), (13.4, 0.2, 0.1, 120.0), (7.5, 6.5, 4.5, -3.0)]
    got = O3.loglik(vol, *[np.array(c) for c in zip(*pts)], m)
    for n, (x, y, z, a) in enumerate(pts):
        cx, cy, cz = math.floor(x + 0.5), math.floor(y + 0.5), math.floor(z + 0.5)
        s = 0.0
        for vz in range(cz - 1, cz + 2):
            for vy in range(cy - 2, cy + 3):
                for vx in range(cx - 2, cx + 3):
                    if not (0 <= vx < W and 0 <= vy < H and 0 <= vz < D):
                        continue
                    lam = max(a, 0.0) * math.exp(-((vx - x) ** 2 + (vy - y) ** 2) / (2 * 1.5 ** 2)
                                                 - (vz - z) ** 2 / (2 * 3.0 ** 2)) + 10.0
                    zz = float(vol[vz, vy, vx])
                    s += (zz * math.log(lam / zz) if zz > 0 else 0.0) - (lam - zz)
        assert got[n] == pytest.approx(s, rel=1e-12, abs=1e-9)


def test_single_slice_reduces_to_2d():
    rng = np.random.default_rng(2)
    img = rng.poisson(synth.render(20, 18, 9.2, 8.7, 100.0, 10.0, 1.5)).astype(np.float32)
    vol = img[None]
    m3 = O3.Model3(patch_xy=9, patch_z=1)
    m2 = synth.Model(sigma_psf=1.5, bg=10.0, patch=9)
    x = rng.uniform(3, 16, 50)
    y = rng.uniform(3, 15, 50)
    a = rng.uniform(50, 150, 50)
    np.testing.assert_allclose(O3.loglik(vol, x, y, np.zeros(50), a, m3), O2.loglik(img, x, y, a, m2),
                               rtol=1e-13, atol=1e-10)


def test_poisson_differences_match_scipy():
    m = O3.Model3(patch_xy=5, patch_z=3)
    vol = _vol(3)
    # two positions with the same nearest voxel share the patch
    pts = np.array([[6.2, 5.9, 4.3, 90.0], [6.4, 5.7, 4.45, 110.0]])
    ll = O3.loglik(vol, pts[:, 0], pts[:, 1], pts[:, 2], pts[:, 3], m)
    full = []
    for x, y, z, a in pts:
        s = 0.0
        for vz in range(3, 6):
            for vy in range(4, 9):
                for vx in range(4, 9):
                    lam = a * math.exp(-((vx - x) ** 2 + (vy - y) ** 2) / (2 * 1.5 ** 2)
                                       - (vz - z) ** 2 / (2 * 3.0 ** 2)) + 10.0
                    s += stats.poisson.logpmf(vol[vz, vy, vx], lam)
        full.append(s)
    assert ll[0] - ll[1] == pytest.approx(full[0] - full[1], rel=1e-9, abs=1e-8)


def test_cells_match_particle_loop():
    rng = np.random.default_rng(4)
    p = rng.uniform(-5, 20, (3, 300)).astype(np.float32)
    h = (0.5, 0.5, 1.0)
    bx, by, bz = O3.bin_coords(p[0], p[1], p[2], h)
    for i in range(300):
        for c, b in zip(range(3), (bx, by, bz)):
            assert b[i] == math.floor(float(np.float32(np.float32(p[c, i]) + np.float32(0.5))
                                            / np.float32(h[c])))
    keys, member, counts = O3.segment(bx, by, bz)
    assert counts.sum() == 300
    for i in range(300):
        assert tuple(keys[member[i]]) == (bx[i], by[i], bz[i])


def test_one_particle_per_cell_is_sir():
    m = O3.Model3()
    seq = synth.make_sequence3(40, 36, 20, 1, seed=5)
    N = 3000
    rng = np.random.default_rng(6)
    st = synth.initial_state3(seq.gt[0], N, np.float64)
    st[:3] += rng.normal(0, 1.0, (3, N))
    nz = synth.make_noise(N, synth.Q3, 7, 0, np.float64)
    a = O3.sir_step(st, seq.images[0], nz, 0.37, m)
    b = O3.pcsir_step(st, seq.images[0], nz, 0.37, (1e-6, 1e-6, 1e-6), m)
    assert b["bin_keys"].shape[0] == N
    np.testing.assert_array_equal(a["ll"], b["ll"])
    np.testing.assert_array_equal(a["ancestors"], b["ancestors"])
    np.testing.assert_array_equal(a["estimate"], b["estimate"])


def test_estimate_converges_to_sir_as_cells_shrink():
    m = O3.Model3()
    seq = synth.make_sequence3(40, 36, 20, 1, seed=8)
    N = 4000
    rng = np.random.default_rng(9)
    st = synth.initial_state3(seq.gt[0], N, np.float64)
    st[:3] += rng.normal(0, 0.8, (3, N))
    nz = synth.make_noise(N, synth.Q3, 10, 0, np.float64)
    sir = O3.sir_step(st, seq.images[0], nz, 0.5, m)["estimate"][:3]
    errs = []
    for h in (2.0, 1.0, 0.5, 0.1, 0.02):
        est = O3.pcsir_step(st, seq.images[0], nz, 0.5, (h, h, 2 * h), m)["estimate"][:3]
        errs.append(np.linalg.norm(est - sir))
    assert errs[-1] < 0.05 * errs[0]
    assert errs[-1] < 1e-2
