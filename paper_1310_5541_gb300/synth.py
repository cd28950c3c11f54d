"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This module holds no filter arithmetic.  It only draws the random numbers the
filter consumes (process noise, resampling uniforms) and simulates the
microscope that produces the observed images, so that both implementations
can be fed identical inputs.

Workload shape follows the paper's simulated fluorescence-microscopy
sequences (Section 5.3): a single Gaussian-PSF spot (Eq. object) on a constant
background, Poisson photon noise, moving under a nearly-constant-velocity
model (Section 5.1).  The SNR of a Poisson image is taken as
SNR = I0 / sqrt(I0 + bg), so I0 is recovered from a target SNR by solving that
quadratic.

State layout is structure-of-arrays: ``state[d, i]`` with
``d in (x, y, vx, vy, I0)``; images are row-major ``Z[y, x]`` with pixel
(x, y) centred on integer coordinates.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

D2 = 5  # (x, y, vx, vy, I0)


@dataclasses.dataclass(frozen=True)
class Model:
    """Parameters of the tracking model (dynamics, appearance and likelihood)."""

    sigma_psf: float = 1.5        # PSF standard deviation in pixels
    I0: float = 100.0             # peak intensity of the spot
    bg: float = 10.0              # background intensity
    patch: int = 9                # odd side of the likelihood patch S_x
    q: tuple = (0.5, 0.5, 0.1, 0.1, 1.0)  # process-noise std per state component
    lik: str = "poisson"          # "poisson" or "sse"
    sigma_xi: float = 20.0        # SSE likelihood peakiness (paper Eq. likelihood)


def i0_from_snr(snr: float, bg: float) -> float:
    """Peak intensity for a Poisson SNR defined as I0 / sqrt(I0 + bg)."""
    s2 = snr * snr
    return 0.5 * (s2 + math.sqrt(s2 * s2 + 4.0 * s2 * bg))


def render(W: int, H: int, x0: float, y0: float, I0: float, bg: float, sigma: float) -> np.ndarray:
    """Noise-free image of one spot, point-sampled at integer pixel centres (FP64)."""
    xs = np.arange(W, dtype=np.float64)
    ys = np.arange(H, dtype=np.float64)
    gx = np.exp(-((xs - x0) ** 2) / (2.0 * sigma * sigma))
    gy = np.exp(-((ys - y0) ** 2) / (2.0 * sigma * sigma))
    return I0 * np.outer(gy, gx) + bg


@dataclasses.dataclass
class Sequence:
    gt: np.ndarray        # [K+1, 5] ground-truth states, frame 0 = initial state
    images: np.ndarray    # [K, H, W] float32 Poisson images for frames 1..K


def make_sequence(W: int, H: int, n_frames: int, model: Model, seed: int,
                  start=None, vmax=None, margin=None, vmin=None) -> Sequence:
    """Ground-truth track and its noisy image sequence.

    The track starts at ``start`` (default: image centre) with a speed drawn
    uniformly in [vmin, vmax] px/frame (vmin defaults to vmax/2) in a uniformly random direction and
    then follows the nearly-constant-velocity model with the model's process
    noise on velocity and intensity (positions advance by the velocity only,
    so the spot moves smoothly).  ``vmax`` defaults to the largest speed that
    keeps a straight track inside the image margin for the whole sequence.
    """
    rng = np.random.default_rng([seed, 0x5EED])
    if margin is None:
        margin = model.patch
    if start is None:
        start = ((W - 1) / 2.0, (H - 1) / 2.0)
    if vmax is None:
        vmax = max(0.05, (min(W, H) / 2.0 - margin) / max(n_frames, 1))
    for _attempt in range(1000):
        speed = rng.uniform(vmax / 2.0 if vmin is None else vmin, vmax)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        s = np.array([start[0], start[1], speed * math.cos(ang), speed * math.sin(ang), model.I0])
        gt = [s.copy()]
        ok = True
        for _k in range(n_frames):
            s = s.copy()
            s[0] += s[2]
            s[1] += s[3]
            s[2] += rng.normal() * model.q[2]
            s[3] += rng.normal() * model.q[3]
            s[4] = max(1.0, s[4] + rng.normal() * model.q[4])
            if not (margin <= s[0] <= W - 1 - margin and margin <= s[1] <= H - 1 - margin):
                ok = False
                break
            gt.append(s)
        if ok:
            break
    gt = np.array(gt)
    images = np.empty((n_frames, H, W), dtype=np.float32)
    for k in range(n_frames):
        lam = render(W, H, gt[k + 1, 0], gt[k + 1, 1], gt[k + 1, 4], model.bg, model.sigma_psf)
        images[k] = rng.poisson(lam).astype(np.float32)
    return Sequence(gt=gt, images=images)


def initial_state(gt0, N: int, dtype=np.float64) -> np.ndarray:
    """All N particles at the ground-truth initial state (paper Section 5.3)."""
    st = np.empty((D2, N), dtype=dtype)
    for d in range(D2):
        st[d, :] = gt0[d]
    return st


def make_noise(N: int, q, seed: int, frame: int, dtype=np.float64) -> np.ndarray:
    """Process noise epsilon[d, i] ~ N(0, q_d^2), drawn in FP64 and rounded to the state dtype."""
    rng = np.random.default_rng([seed, 1, frame])
    out = np.empty((len(q), N), dtype=dtype)
    for d, qd in enumerate(q):
        out[d] = (rng.standard_normal(N) * qd).astype(dtype)
    return out


def make_u0(seed: int, frame: int) -> float:
    """Systematic-resampling offset u0 ~ U[0, 1)."""
    return float(np.random.default_rng([seed, 2, frame]).random())


def random_weights_case(N: int, seed: int):
    """Random positive log-weights for resampling tests (no filter arithmetic)."""
    rng = np.random.default_rng([seed, 3])
    return rng.normal(size=N) * 3.0


@dataclasses.dataclass
class Batch:
    """Many independent targets in one frame sequence."""

    n: np.ndarray          # [T] particles per target
    sigma: np.ndarray      # [T] PSF std per target
    i0: np.ndarray         # [T] peak intensity per target
    patch: np.ndarray      # [T] odd likelihood patch side per target
    h: np.ndarray          # [T] cell edge per target
    bg: float
    gt: np.ndarray         # [K+1, T, 5] ground-truth states
    images: np.ndarray     # [K, H, W] float32 Poisson images with every target's spot


def make_batch(T: int, W: int, H: int, n_frames: int, seed: int, n_range=(1000, 100000), sigma_range=(1.2, 2.0),
               snr_range=(2.0, 8.0), bg: float = 10.0, min_sep: float = 16.0, h_of_sigma=None, q=None,
               n_values=None) -> Batch:
    """Multi-target workload: positions by dart throwing with a minimum separation,
    particle counts log-uniform in n_range (or given), PSF std uniform in sigma_range,
    SNR uniform in snr_range (I0 from the Poisson SNR), patch side 2 ceil(3 sigma) + 1,
    slow nearly-constant-velocity tracks."""
    rng = np.random.default_rng([seed, 0xBA7C])
    q = q or (0.5, 0.5, 0.1, 0.1, 1.0)
    margin = 24.0
    pos = []
    for _ in range(T * 200):
        if len(pos) == T:
            break
        p = rng.uniform([margin, margin], [W - 1 - margin, H - 1 - margin])
        if all((p[0] - a) ** 2 + (p[1] - b) ** 2 >= min_sep ** 2 for a, b in pos):
            pos.append(p)
    if len(pos) < T:
        raise ValueError("cannot place %d targets with separation %g in %dx%d" % (T, min_sep, W, H))
    if n_values is None:
        n = np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]), T)).astype(np.int64)
    else:
        n = np.asarray(n_values, dtype=np.int64)
    sigma = rng.uniform(sigma_range[0], sigma_range[1], T)
    i0 = np.array([i0_from_snr(s, bg) for s in rng.uniform(snr_range[0], snr_range[1], T)])
    patch = (2 * np.ceil(3.0 * sigma) + 1).astype(np.int64)
    h = np.full(T, 0.5) if h_of_sigma is None else np.asarray([h_of_sigma(s) for s in sigma])
    gt = np.zeros((n_frames + 1, T, 5))
    ang = rng.uniform(0, 2 * math.pi, T)
    speed = rng.uniform(0.05, 0.3, T)
    gt[0, :, 0] = [p[0] for p in pos]
    gt[0, :, 1] = [p[1] for p in pos]
    gt[0, :, 2] = speed * np.cos(ang)
    gt[0, :, 3] = speed * np.sin(ang)
    gt[0, :, 4] = i0
    for k in range(n_frames):
        s = gt[k].copy()
        s[:, 0] += s[:, 2]
        s[:, 1] += s[:, 3]
        s[:, 2] += rng.normal(size=T) * q[2] * 0.1
        s[:, 3] += rng.normal(size=T) * q[3] * 0.1
        gt[k + 1] = s
    images = np.empty((n_frames, H, W), dtype=np.float32)
    xs = np.arange(W, dtype=np.float64)
    ys = np.arange(H, dtype=np.float64)
    for k in range(n_frames):
        lam = np.full((H, W), bg)
        for t in range(T):
            x0, y0, a = gt[k + 1, t, 0], gt[k + 1, t, 1], gt[k + 1, t, 4]
            r = int(np.ceil(5 * sigma[t]))
            cx, cy = int(round(x0)), int(round(y0))
            xa, xb = max(0, cx - r), min(W, cx + r + 1)
            ya, yb = max(0, cy - r), min(H, cy + r + 1)
            gx = np.exp(-((xs[xa:xb] - x0) ** 2) / (2 * sigma[t] ** 2))
            gy = np.exp(-((ys[ya:yb] - y0) ** 2) / (2 * sigma[t] ** 2))
            lam[ya:yb, xa:xb] += a * np.outer(gy, gx)
        images[k] = rng.poisson(lam).astype(np.float32)
    return Batch(n=n, sigma=sigma, i0=i0, patch=patch, h=h, bg=bg, gt=gt, images=images)


def batch_initial_state(batch: Batch, dtype=np.float32) -> np.ndarray:
    """Concatenated [5, sum N_t] state with each target's particles at its ground truth."""
    parts = [initial_state(batch.gt[0, t], int(batch.n[t]), dtype) for t in range(len(batch.n))]
    return np.ascontiguousarray(np.concatenate(parts, axis=1))


def batch_noise(batch: Batch, q, seed: int, frame: int, dtype=np.float32) -> np.ndarray:
    return make_noise(int(batch.n.sum()), q, seed, frame, dtype)


def batch_u0(T: int, seed: int, frame: int) -> np.ndarray:
    return np.random.default_rng([seed, 4, frame]).random(T)


# ----------------------------------------------------------------------------
# Pseudo-tracking (Section 5.4): no dynamics, particles drawn from a fixed prior
# around the true position, one weighting of a single image.
# ----------------------------------------------------------------------------
PSEUDO_PRIORS = ("uniform3", "uniform5", "gauss0.5", "gauss0.8")


def pseudo_case(prior: str, N: int, seed: int, rep: int, W: int = 32, sigma_psf: float = 1.16,
                snr: float = 2.0, sigma_xi: float = 20.0, bg: float = 10.0, dtype=np.float32):
    """One repetition of the pseudo-tracking experiment.

    The object (Gaussian PSF ``sigma_psf``) sits at a uniformly random sub-pixel
    position near the image centre; the image carries Gaussian noise of
    standard deviation ``sigma_xi`` and the peak intensity is ``snr * sigma_xi``.
    The N particles are drawn from the prior centred on the true position:
    uniform over a 3 x 3 or 5 x 5 pixel square, or Gaussian with standard
    deviation 0.5 or 0.8 pixel; velocities are 0 and the intensity is the true
    one.  Returns (image [W, W], truth (x, y), state [5, N], u0).
    """
    rng = np.random.default_rng([seed, 7, rep])
    c = (W - 1) / 2.0
    x0, y0 = c + rng.uniform(-0.5, 0.5), c + rng.uniform(-0.5, 0.5)
    i0 = snr * sigma_xi
    img = render(W, W, x0, y0, i0, bg, sigma_psf) + rng.normal(0.0, sigma_xi, (W, W))
    st = np.zeros((D2, N), dtype=np.float64)
    if prior.startswith("uniform"):
        half = float(prior[len("uniform"):]) / 2.0
        st[0] = x0 + rng.uniform(-half, half, N)
        st[1] = y0 + rng.uniform(-half, half, N)
    elif prior.startswith("gauss"):
        sd = float(prior[len("gauss"):])
        st[0] = x0 + rng.normal(0.0, sd, N)
        st[1] = y0 + rng.normal(0.0, sd, N)
    else:
        raise ValueError(prior)
    st[4] = i0
    return img.astype(np.float32), (x0, y0), st.astype(dtype), float(rng.random())


# Large-object tracking (Section 5.3): PSF sigma 13 px, SNR 2, speed U[2, 7]
# px/frame, 512 x 512 frames, 65 x 65 likelihood kernel with the paper's
# Gaussian (SSE) likelihood.
def large_object_model(sigma_xi: float = 30.0) -> Model:
    bg = 10.0
    return Model(sigma_psf=13.0, I0=i0_from_snr(2.0, bg), bg=bg, patch=65, lik="sse", sigma_xi=sigma_xi,
                 q=(0.5, 0.5, 0.1, 0.1, 0.1))


def large_object_sequence(n_frames: int, seed: int, W: int = 512) -> Sequence:
    """A track starting at a random position, speed U[2, 7] px/frame, kept 40 px inside the frame."""
    m = large_object_model()
    rng = np.random.default_rng([seed, 9])
    margin = 40.0
    vmax = 7.0
    # start far enough from the border for the whole straight-line track
    room = margin + vmax * n_frames
    lo, hi = min(room, W / 2.0), max(W - 1 - room, W / 2.0)
    start = (rng.uniform(lo, hi), rng.uniform(lo, hi))
    return make_sequence(W, W, n_frames, m, seed, start=start, vmax=vmax, vmin=2.0, margin=margin)


# ----------------------------------------------------------------------------
# 3D tracking: state (x, y, z, vx, vy, vz, I0), volumes V[z, y, x] with an
# anisotropic Gaussian PSF and Poisson noise.
# ----------------------------------------------------------------------------
D3 = 7
Q3 = (0.5, 0.5, 0.5, 0.1, 0.1, 0.1, 1.0)


def render3(W: int, H: int, D: int, x0: float, y0: float, z0: float, I0: float, bg: float, sigma_xy: float,
            sigma_z: float) -> np.ndarray:
    """Noise-free volume of one spot, point-sampled at integer voxel centres (FP64, [D, H, W])."""
    gx = np.exp(-((np.arange(W) - x0) ** 2) / (2.0 * sigma_xy * sigma_xy))
    gy = np.exp(-((np.arange(H) - y0) ** 2) / (2.0 * sigma_xy * sigma_xy))
    gz = np.exp(-((np.arange(D) - z0) ** 2) / (2.0 * sigma_z * sigma_z))
    return I0 * gz[:, None, None] * gy[None, :, None] * gx[None, None, :] + bg


def make_sequence3(W: int, H: int, D: int, n_frames: int, seed: int, I0: float = 100.0, bg: float = 10.0,
                   sigma_xy: float = 1.5, sigma_z: float = 3.0, q=Q3, margin: float = 8.0, vmax: float = 1.5):
    """Ground-truth 3D track (NCV, speed U[vmax/2, vmax] voxel/frame, random direction) and its Poisson
    volumes; the track stays ``margin`` voxels inside the volume (z: margin / 2)."""
    rng = np.random.default_rng([seed, 0x3D])
    for _attempt in range(1000):
        speed = rng.uniform(vmax / 2.0, vmax)
        v = rng.normal(size=3)
        v = v / np.linalg.norm(v) * speed
        s = np.array([(W - 1) / 2.0, (H - 1) / 2.0, (D - 1) / 2.0, v[0], v[1], v[2], I0])
        gt = [s.copy()]
        ok = True
        for _k in range(n_frames):
            s = s.copy()
            s[0:3] += s[3:6]
            s[3:6] += rng.normal(size=3) * np.asarray(q[3:6])
            s[6] = max(1.0, s[6] + rng.normal() * q[6])
            if not (margin <= s[0] <= W - 1 - margin and margin <= s[1] <= H - 1 - margin
                    and margin / 2 <= s[2] <= D - 1 - margin / 2):
                ok = False
                break
            gt.append(s)
        if ok:
            break
    gt = np.array(gt)
    vols = np.empty((n_frames, D, H, W), dtype=np.float32)
    for k in range(n_frames):
        lam = render3(W, H, D, gt[k + 1, 0], gt[k + 1, 1], gt[k + 1, 2], gt[k + 1, 6], bg, sigma_xy, sigma_z)
        vols[k] = rng.poisson(lam).astype(np.float32)
    return Sequence(gt=gt, images=vols)


def initial_state3(gt0, N: int, dtype=np.float32) -> np.ndarray:
    st = np.empty((D3, N), dtype=dtype)
    for d in range(D3):
        st[d, :] = gt0[d]
    return st


@dataclasses.dataclass
class Batch3:
    """Many independent targets in one 3D volume sequence."""

    n: np.ndarray          # [T] particles per target
    sigma_xy: np.ndarray   # [T] lateral PSF std per target
    sigma_z: np.ndarray    # [T] axial PSF std per target
    i0: np.ndarray         # [T] peak intensity per target
    bg: np.ndarray         # [T] background per target (one shared background)
    patch_xy: np.ndarray   # [T] odd lateral patch side
    patch_z: np.ndarray    # [T] odd axial patch side
    h: np.ndarray          # [T, 3] cell edges per target
    gt: np.ndarray         # [K+1, T, 7] ground-truth states
    images: np.ndarray     # [K, D, H, W] float32 Poisson volumes with every target's spot


def make_batch3(T: int, W: int, H: int, D: int, n_frames: int, seed: int, n_values=None, n_particles: int = 200_000,
                sigma_xy: float = 1.5, sigma_z: float = 3.0, i0: float = 100.0, bg: float = 10.0,
                patch_xy: int = 11, patch_z: int = 7, h=(0.5, 0.5, 1.0), min_sep: float = 10.0,
                margin_xy: float = 10.0, margin_z: float = 5.0, q=Q3) -> Batch3:
    """3D multi-target workload: spot centres by dart throwing with a minimum separation inside the
    margins, slow nearly-constant-velocity tracks (speed U[0.05, 0.3] voxel/frame), one shared
    Poisson volume per frame (every spot rendered within 4 PSF stds of its centre, plus the
    background)."""
    rng = np.random.default_rng([seed, 0xB3D])
    lo = np.array([margin_xy, margin_xy, margin_z])
    hi = np.array([W - 1 - margin_xy, H - 1 - margin_xy, D - 1 - margin_z])
    pos = []
    for _ in range(T * 500):
        if len(pos) == T:
            break
        p = rng.uniform(lo, hi)
        if all(np.sum((p - a) ** 2) >= min_sep ** 2 for a in pos):
            pos.append(p)
    if len(pos) < T:
        raise ValueError("cannot place %d targets with separation %g in %dx%dx%d" % (T, min_sep, W, H, D))
    n = np.full(T, n_particles, np.int64) if n_values is None else np.asarray(n_values, np.int64)
    gt = np.zeros((n_frames + 1, T, D3))
    v = rng.normal(size=(T, 3))
    v *= (rng.uniform(0.05, 0.3, T) / np.linalg.norm(v, axis=1))[:, None]
    gt[0, :, 0:3] = np.array(pos)
    gt[0, :, 3:6] = v
    gt[0, :, 6] = i0
    for k in range(n_frames):
        s = gt[k].copy()
        s[:, 0:3] += s[:, 3:6]
        s[:, 3:6] += rng.normal(size=(T, 3)) * np.asarray(q[3:6]) * 0.1
        gt[k + 1] = s
    images = np.empty((n_frames, D, H, W), dtype=np.float32)
    rxy, rz = int(np.ceil(4 * sigma_xy)), int(np.ceil(4 * sigma_z))
    for k in range(n_frames):
        lam = np.full((D, H, W), bg)
        for t in range(T):
            x0, y0, z0, a = gt[k + 1, t, 0], gt[k + 1, t, 1], gt[k + 1, t, 2], gt[k + 1, t, 6]
            cx, cy, cz = int(round(x0)), int(round(y0)), int(round(z0))
            xa, xb = max(0, cx - rxy), min(W, cx + rxy + 1)
            ya, yb = max(0, cy - rxy), min(H, cy + rxy + 1)
            za, zb = max(0, cz - rz), min(D, cz + rz + 1)
            gx = np.exp(-((np.arange(xa, xb) - x0) ** 2) / (2 * sigma_xy ** 2))
            gy = np.exp(-((np.arange(ya, yb) - y0) ** 2) / (2 * sigma_xy ** 2))
            gz = np.exp(-((np.arange(za, zb) - z0) ** 2) / (2 * sigma_z ** 2))
            lam[za:zb, ya:yb, xa:xb] += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        images[k] = rng.poisson(lam).astype(np.float32)
    full = lambda v_: np.full(T, v_)
    return Batch3(n=n, sigma_xy=full(float(sigma_xy)), sigma_z=full(float(sigma_z)), i0=full(float(i0)),
                  bg=full(float(bg)), patch_xy=full(int(patch_xy)).astype(np.int64),
                  patch_z=full(int(patch_z)).astype(np.int64), h=np.tile(np.asarray(h, np.float64), (T, 1)),
                  gt=gt, images=images)


def batch3_initial_state(batch: Batch3, dtype=np.float32) -> np.ndarray:
    """Concatenated [7, sum N_t] state with each target's particles at its ground truth."""
    parts = [initial_state3(batch.gt[0, t], int(batch.n[t]), dtype) for t in range(len(batch.n))]
    return np.ascontiguousarray(np.concatenate(parts, axis=1))
