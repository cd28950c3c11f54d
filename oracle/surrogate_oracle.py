"""Plain FP64 CPU oracle of the learned likelihood surrogate.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the test suite and the CPU-baseline / reference arm
of ``bench.py`` use it.  It shares no code with the CUDA library.

The surrogate is an addition to the paper's method, not part of it.  In the
pcSIR step (Algorithm 2) the costly quantity is the log-likelihood of each
dummy particle against its image patch (Eq. likelihood with the PSF of
Eq. object); the surrogate predicts that number from the patch and the
dummy's sub-pixel state with a small fully connected network, and the exact
likelihood stays the measure of its error.  Definitions written out here:

* Inputs (445 = P*P + 4 with P = 21): the P x P patch centred on the pixel
  nearest the position, ``c = floor(x + 0.5)`` as in the exact likelihood,
  read row by row (image row cy-R .. cy+R, columns cx-R .. cx+R) and mapped
  to ``(z - bg) / i0_ref``; then ``2 (x - cx)``, ``2 (y - cy)`` (the sub-pixel
  offset, in [-1, 1)), ``I0 / i0_ref`` and ``sigma / sigma_ref``.  A patch that
  leaves the image is "clipped": the exact likelihood drops the outside
  pixels, which the network cannot see, so clipped dummies always take the
  exact likelihood.
* Exact window term.  With lambda_j = bg + I0 g_j (Eq. object) the Poisson
  term of Eq. likelihood splits, pixel by pixel, into
  ``z log(lambda/z) - (lambda - z) = [z - z log z + z log bg - bg]
  + [z log(1 + I0 g / bg) - I0 g]``.  The first bracket depends on the image
  alone; summed over the window it is ``T(cx, cy) = sum (z - z log z) +
  log(bg) sum z - P^2 bg`` (0 log 0 = 0), which a box filter gives for every
  window of a frame.  The network learns only the second bracket, the
  residual ``r = ll - T``, which involves the pixels near the spot alone;
  the part of ll that sums noise over all 441 pixels is computed exactly.
* Network: ``z1 = W1 x + b1, a1 = silu(z1), z2 = W2 a1 + b2, a2 = silu(z2),
  out = w3 . a2 + b3`` with ``silu(t) = t / (1 + exp(-t))``; W1 is 256 x 445,
  W2 256 x 256.  The prediction of the log-likelihood is
  ``T + mean + scale * out`` with the mean and standard deviation of the
  training rows' residual labels.
* Training: squared error of ``out`` against the standardised label
  ``(r - mean) / scale``, averaged over a minibatch; gradients by
  backpropagation; the Adam update (Kingma and Ba, 2015) with bias-corrected
  moments.  A "censored" row carries a floor instead of its log-likelihood
  (the exact value lies below it, so far below the step's best dummy that its
  weight is negligible; the label is ``floor - T``): its error counts only
  where ``out`` exceeds the label, ``max(out - label, 0)^2``, the one-sided
  loss of censored regression.
* Held-out check: a dummy is held out when a splitmix64 hash (Steele, Lea
  and Flood, 2014) of its cell index and the step's salt falls below the
  requested fraction; its exact likelihood is computed beside the
  prediction.  A held-out dummy is significant when its exact or predicted
  log-likelihood lies within ``window`` of the step's maximum prediction; the
  step falls back to the exact likelihood for every dummy when the largest
  error over the significant held-out dummies exceeds ``max_err`` (or is not
  finite).
"""
from __future__ import annotations

import numpy as np

P = 21
R = P // 2
N_IN = P * P + 4
HIDDEN = 256
PARAM_SHAPES = (("W1", (HIDDEN, N_IN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
                ("w3", (HIDDEN,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in PARAM_SHAPES)


# 3D surrogate: an 11 x 11 x 7 voxel patch, then the sub-voxel offsets along x, y, z, I0 and sigma_xy
P3XY, P3Z = 11, 7
R3XY, R3Z = P3XY // 2, P3Z // 2
NPIX3 = P3XY * P3XY * P3Z
N_IN3 = NPIX3 + 5
PARAM_SHAPES3 = (("W1", (HIDDEN, N_IN3)),) + PARAM_SHAPES[1:]
N_PARAMS3 = sum(int(np.prod(s)) for _, s in PARAM_SHAPES3)


def pack(params: dict, shapes=PARAM_SHAPES) -> np.ndarray:
    """Flatten parameters in the fixed order W1, b1, W2, b2, w3, b3 (float64)."""
    return np.concatenate([np.asarray(params[k], np.float64).reshape(-1) for k, _ in shapes])


def unpack(flat: np.ndarray, shapes=PARAM_SHAPES) -> dict:
    """Parameters from their packed form (``shapes``: PARAM_SHAPES, or PARAM_SHAPES3 in 3D)."""
    out, o = {}, 0
    for k, s in shapes:
        n = int(np.prod(s))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(s)
        o += n
    return out


# ----------------------------------------------------------------------------
# Network inputs
# ----------------------------------------------------------------------------
def features(image: np.ndarray, x, y, i0, sigma, bg: float, i0_ref: float, sigma_ref: float):
    """Network inputs of evaluated states; returns (X [n, 445] float64, clipped [n] bool)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    i0 = np.asarray(i0, np.float64)
    sigma = np.broadcast_to(np.asarray(sigma, np.float64), x.shape)
    Hh, Ww = image.shape
    img = image.astype(np.float64)
    cx = np.floor(x + 0.5)
    cy = np.floor(y + 0.5)
    off = np.arange(-R, R + 1, dtype=np.float64)
    cols = (cx[:, None] + off[None, :]).astype(np.int64)
    rows = (cy[:, None] + off[None, :]).astype(np.int64)
    clipped = (cx - R < 0) | (cx + R > Ww - 1) | (cy - R < 0) | (cy + R > Hh - 1)
    inside = ((rows >= 0) & (rows < Hh))[:, :, None] & ((cols >= 0) & (cols < Ww))[:, None, :]
    z = img[np.clip(rows, 0, Hh - 1)[:, :, None], np.clip(cols, 0, Ww - 1)[:, None, :]]
    z = np.where(inside, z, bg)
    X = np.empty((x.shape[0], N_IN))
    X[:, :P * P] = ((z - bg) / i0_ref).reshape(x.shape[0], P * P)
    X[:, P * P] = 2.0 * (x - cx)
    X[:, P * P + 1] = 2.0 * (y - cy)
    X[:, P * P + 2] = i0 / i0_ref
    X[:, P * P + 3] = sigma / sigma_ref
    return X, clipped


def window_term(image: np.ndarray, x, y, bg: float) -> np.ndarray:
    """T(cx, cy) of the windows around the states' nearest pixels (windows inside the image)."""
    z = image.astype(np.float64)
    e = np.where(z > 0, z - z * np.log(np.where(z > 0, z, 1.0)), 0.0) + np.log(bg) * z
    cx = np.floor(np.asarray(x, np.float64) + 0.5).astype(np.int64)
    cy = np.floor(np.asarray(y, np.float64) + 0.5).astype(np.int64)
    out = np.empty(cx.shape[0])
    for i in range(cx.shape[0]):
        out[i] = e[cy[i] - R:cy[i] + R + 1, cx[i] - R:cx[i] + R + 1].sum() - P * P * bg
    return out


def features3(volume: np.ndarray, x, y, z, i0, sigma_xy, bg: float, i0_ref: float, sigma_ref: float):
    """3D network inputs; returns (X [n, 852] float64, clipped [n] bool).

    The 11 x 11 x 7 patch centred on the nearest voxel (cx, cy, cz) = floor(. + 0.5), x fastest,
    then y, then z, as (v - bg) / i0_ref; then 2 (x - cx), 2 (y - cy), 2 (z - cz), I0 / i0_ref and
    sigma_xy / sigma_ref.  A patch that leaves the volume is clipped."""
    x, y, z, i0 = (np.asarray(v, np.float64) for v in (x, y, z, i0))
    sig = np.broadcast_to(np.asarray(sigma_xy, np.float64), x.shape)
    Dd, Hh, Ww = volume.shape
    vol = volume.astype(np.float64)
    cx, cy, cz = np.floor(x + 0.5), np.floor(y + 0.5), np.floor(z + 0.5)
    clipped = ((cx - R3XY < 0) | (cx + R3XY > Ww - 1) | (cy - R3XY < 0) | (cy + R3XY > Hh - 1) |
               (cz - R3Z < 0) | (cz + R3Z > Dd - 1))
    n = x.shape[0]
    X = np.empty((n, N_IN3))
    for i in range(n):
        if clipped[i]:
            X[i, :NPIX3] = 0.0
        else:
            a, b, c = int(cx[i]), int(cy[i]), int(cz[i])
            blk = vol[c - R3Z:c + R3Z + 1, b - R3XY:b + R3XY + 1, a - R3XY:a + R3XY + 1]
            X[i, :NPIX3] = ((blk - bg) / i0_ref).reshape(-1)  # x fastest, then y, then z
    X[:, NPIX3] = 2.0 * (x - cx)
    X[:, NPIX3 + 1] = 2.0 * (y - cy)
    X[:, NPIX3 + 2] = 2.0 * (z - cz)
    X[:, NPIX3 + 3] = i0 / i0_ref
    X[:, NPIX3 + 4] = sig / sigma_ref
    return X, clipped


def window_term3(volume: np.ndarray, x, y, z, bg: float) -> np.ndarray:
    """T(cx, cy, cz): the image-only part of the Poisson term summed over the 11 x 11 x 7 window
    around the states' nearest voxels (windows inside the volume), minus 847 bg."""
    v = volume.astype(np.float64)
    e = np.where(v > 0, v - v * np.log(np.where(v > 0, v, 1.0)), 0.0) + np.log(bg) * v
    cx = np.floor(np.asarray(x, np.float64) + 0.5).astype(np.int64)
    cy = np.floor(np.asarray(y, np.float64) + 0.5).astype(np.int64)
    cz = np.floor(np.asarray(z, np.float64) + 0.5).astype(np.int64)
    out = np.empty(cx.shape[0])
    for i in range(cx.shape[0]):
        out[i] = e[cz[i] - R3Z:cz[i] + R3Z + 1, cy[i] - R3XY:cy[i] + R3XY + 1,
                   cx[i] - R3XY:cx[i] + R3XY + 1].sum() - NPIX3 * bg
    return out


# ----------------------------------------------------------------------------
# Forward and backward passes
# ----------------------------------------------------------------------------
def silu(t):
    return t / (1.0 + np.exp(-t))


def silu_grad(t):
    s = 1.0 / (1.0 + np.exp(-t))
    return s * (1.0 + t * (1.0 - s))


def forward(params: dict, X: np.ndarray):
    """Network output ``out`` [n] and the intermediate values of the pass."""
    z1 = X @ params["W1"].T + params["b1"]
    a1 = silu(z1)
    z2 = a1 @ params["W2"].T + params["b2"]
    a2 = silu(z2)
    out = a2 @ params["w3"] + params["b3"][0]
    return out, {"X": X, "z1": z1, "a1": a1, "z2": z2, "a2": a2}


def predict_ll(params: dict, mean: float, scale: float, X: np.ndarray, T) -> np.ndarray:
    """Predicted log-likelihood: the exact window term plus the network's residual."""
    return np.asarray(T, np.float64) + mean + scale * forward(params, X)[0]


def loss_and_grads(params: dict, X: np.ndarray, t: np.ndarray, censored=None):
    """Mean squared error L = mean(d^2), d = out - t (0 where a censored row has out <= t), and its
    gradient with respect to every parameter."""
    out, c = forward(params, X)
    n = X.shape[0]
    d = out - t
    if censored is not None:
        d = np.where(np.asarray(censored, bool) & (d < 0), 0.0, d)
    loss = float(np.mean(d * d))
    g_out = 2.0 * d / n                                  # dL/d out
    g = {"w3": c["a2"].T @ g_out, "b3": np.array([g_out.sum()])}
    g_z2 = (g_out[:, None] * params["w3"][None, :]) * silu_grad(c["z2"])
    g["W2"] = g_z2.T @ c["a1"]
    g["b2"] = g_z2.sum(axis=0)
    g_a1 = g_z2 @ params["W2"]
    g_z1 = g_a1 * silu_grad(c["z1"])
    g["W1"] = g_z1.T @ X
    g["b1"] = g_z1.sum(axis=0)
    return loss, g


def standardise(ll: np.ndarray):
    """Label mean and standard deviation of the training rows."""
    ll = np.asarray(ll, np.float64)
    mean = float(ll.mean())
    scale = float(ll.std())
    return mean, (scale if scale > 0 else 1.0)


def adam_step(params: dict, grads: dict, state: dict, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; ``state`` holds the moments and the step count."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k, _ in PARAM_SHAPES:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m *= beta1
        m += (1.0 - beta1) * grads[k]
        v *= beta2
        v += (1.0 - beta2) * grads[k] * grads[k]
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        params[k] -= lr * mhat / (np.sqrt(vhat) + eps)
    return params


# ----------------------------------------------------------------------------
# Held-out selection and check
# ----------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of the splitmix64 generator whose state has just become ``x - golden``."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def holdout_mask(bx, by, salt: int, frac: float) -> np.ndarray:
    """Held-out cells: splitmix64 of the cell index (bx, by as 32-bit words) plus salt * golden.

    A cell is held out when the top 24 bits of the hash fall below floor(frac * 2^24).
    """
    thr = int(np.floor(frac * (1 << 24)))
    out = np.zeros(len(bx), bool)
    for i, (a, b) in enumerate(zip(np.asarray(bx).tolist(), np.asarray(by).tolist())):
        key = (a & 0xFFFFFFFF) | ((b & 0xFFFFFFFF) << 32)
        h = splitmix64((key + salt * 0x9E3779B97F4A7C15) & _M64)
        out[i] = (h >> 40) < thr
    return out


def holdout_mask3(bx, by, bz, salt: int, frac: float) -> np.ndarray:
    """Held-out 3D cells: the same rule with the key (bx + 2^20) | (by + 2^20) << 21 | (bz + 2^20) << 42."""
    thr = int(np.floor(frac * (1 << 24)))
    out = np.zeros(len(bx), bool)
    for i, (a, b, c) in enumerate(zip(np.asarray(bx).tolist(), np.asarray(by).tolist(), np.asarray(bz).tolist())):
        key = (a + (1 << 20)) | ((b + (1 << 20)) << 21) | ((c + (1 << 20)) << 42)
        h = splitmix64((key + salt * 0x9E3779B97F4A7C15) & _M64)
        out[i] = (h >> 40) < thr
    return out


def holdout_check(ll_pred: np.ndarray, ll_exact: np.ndarray, max_pred: float, window: float, max_err: float):
    """Error statistics of the held-out dummies and the fallback decision."""
    ll_pred = np.asarray(ll_pred, np.float64)
    ll_exact = np.asarray(ll_exact, np.float64)
    err = np.abs(ll_pred - ll_exact)
    sig = (np.maximum(ll_pred, ll_exact) >= max_pred - window)
    n_sig = int(sig.sum())
    max_sig = float(err[sig].max()) if n_sig else 0.0
    rms = float(np.sqrt(np.mean(err * err))) if err.size else 0.0
    fallback = (not np.isfinite(max_sig)) or max_sig > max_err or (err.size and not np.all(np.isfinite(err)))
    return {"n_holdout": int(err.size), "n_significant": n_sig, "max_abs_err": max_sig, "rms_err": rms,
            "fallback": bool(fallback)}
