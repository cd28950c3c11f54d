"""Training workflow of the likelihood surrogate on top of the C ABI.

The network and every training and inference pass run in the library's
kernels (``pcsir_surrogate.h``); this module only sequences the calls:

* ``collect`` runs exact pcSIR steps (Algorithm 2) over a frame sequence and
  appends every step's dummies with their exact log-likelihoods to the
  surrogate's dataset, so the training pairs come from the method itself
  (``collect3``: the same for the 3D step and a 3D surrogate);
* ``fit`` normalises the labels of the training rows, trains with Adam and
  reports the error on the held-back rows in log-likelihood units.
"""
from __future__ import annotations

import math

import torch

from . import pcsir


def collect(ctx, sur, state, frames, h, bg, psf_sigma, depth=40.0, stream=None):
    """Exact pcSIR steps over ``frames``: iterable of (image, noise, u0); ``state`` advances in place.

    Each step's dummies become rows labelled with their exact log-likelihood,
    floored ``depth`` nats below the step's largest (a dummy that far down
    carries a relative weight below exp(-depth)).  Returns the number of
    dummies seen.  The context must have no surrogate attached (the labels
    have to be exact log-likelihoods).
    """
    if getattr(ctx, "surrogate", None) is not None:
        raise ValueError("collect needs exact likelihoods: detach the surrogate first")
    seen = 0
    for image, noise, u0 in frames:
        pcsir.pcsir_step(ctx, state, image, h, noise, u0, stream=stream)
        torch.cuda.synchronize()
        out = ctx.outputs()
        if out["n_bins"] > 0:
            floor = ctx.last_result()["max_loglik"] - depth
            sur.add(out["dummy"], out["bin_loglik"], image, bg, psf_sigma, label_floor=floor, stream=stream)
            seen += out["n_bins"]
    torch.cuda.synchronize()
    return seen


def collect3(ctx3, sur, state, frames, h, bg, psf_sigma_xy, depth=40.0, keep_exact=1.0, keep_censored=1.0, seed=0,
             stream=None):
    """The same for the 3D step: exact pcSIR steps of ``ctx3`` (cell edges ``h``) over ``frames``
    (iterable of (volume, noise, u0)); each step's dummies become rows of the 3D surrogate ``sur``.

    The 3D likelihood is far more peaked than the 2D one (about 4700 nats per squared voxel of
    curvature at I0 = 100, bg = 10 and PSF sigmas 1.5 / 3), so at the tracking cell sizes almost
    every dummy lies more than ``depth`` nats below the step's best.  A seeded random choice keeps
    each exactly labelled dummy with probability ``keep_exact`` and each censored one with
    ``keep_censored``, so that neither kind swamps the dataset."""
    if getattr(ctx3, "surrogate", None) is not None:
        raise ValueError("collect3 needs exact likelihoods: detach the surrogate first")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(int(seed))
    seen = 0
    for volume, noise, u0 in frames:
        ctx3.step(state, volume, h, noise, u0, stream=stream)
        torch.cuda.synchronize()
        out = ctx3.outputs()
        if out["n_bins"] > 0:
            floor = ctx3.last_result()["max_loglik"] - depth
            dummy, ll = out["dummy"], out["bin_loglik"]
            if keep_exact < 1.0 or keep_censored < 1.0:
                p = torch.where(ll >= floor, keep_exact, keep_censored)
                idx = (torch.rand(ll.shape[0], device=ll.device, generator=gen, dtype=torch.float64) < p)
                idx = idx.nonzero().squeeze(1)
                dummy, ll = dummy[:, idx].contiguous(), ll[idx].contiguous()
            if ll.shape[0] > 0:
                sur.add3(dummy, ll, volume, bg, psf_sigma_xy, label_floor=floor, stream=stream)
            seen += out["n_bins"]
    torch.cuda.synchronize()
    return seen


# Training data of the 3D surrogate: (noise scale, cell edges) of the exact steps that make it.  The
# first is the model's own process noise at the tracking cell size; the others scale the noise down and
# shrink the cells, so that the dummies crowd the likelihood's peak, where the network must be accurate.
COLLECT3 = ((1.0, (0.1, 0.1, 0.2)), (0.3, (0.03, 0.03, 0.06)), (0.1, (0.01, 0.01, 0.02)))


def collect3_sequences(sur, n_seq, n_frames, n_particles, seed, shape=(64, 64, 32), recipes=COLLECT3,
                       keep_exact=0.06, keep_censored=0.005, bg=10.0, psf_sigma_xy=1.5, on_sequence=None):
    """Rows of the 3D surrogate from ``n_seq`` synthetic sequences of ``n_frames`` Poisson volumes
    (``synth.make_sequence3``, W x H x D = ``shape``), sequence i filtered by exact 3D pcSIR steps of
    ``n_particles`` particles with recipe i mod len(recipes).  What the network learns depends on the
    volume around each dummy only, so small volumes serve: many short sequences give many distinct
    noise patterns, which is what it needs to generalise.  ``on_sequence(i)`` runs after each."""
    import numpy as np

    from . import synth

    W, H, D = shape
    ctx = pcsir.Context3(n_particles)
    try:
        for i in range(n_seq):
            sd = int(seed) + i
            scale, h = recipes[i % len(recipes)]
            seq = synth.make_sequence3(W, H, D, n_frames, sd)
            st = torch.from_numpy(synth.initial_state3(seq.gt[0], n_particles, np.float32)).cuda()
            frames = ((torch.from_numpy(seq.images[k]).cuda(),
                       torch.from_numpy(synth.make_noise(n_particles, synth.Q3, sd, k, np.float32)
                                        * np.float32(scale)).cuda(),
                       synth.make_u0(sd, k)) for k in range(n_frames))
            collect3(ctx, sur, st, frames, h, bg, psf_sigma_xy, keep_exact=keep_exact, keep_censored=keep_censored,
                     seed=sd)
            if on_sequence is not None:
                on_sequence(i)
    finally:
        ctx.close()


def fit(sur, steps, lr=1e-3, seed=1, n_train=None, val_frac=0.05, chunk=500, lr_final=None):
    """Train on the first ``n_train`` rows (default: all but the last ``val_frac``), validate on the rest.

    The learning rate decays from ``lr`` to ``lr_final`` (default lr / 20) along a
    cosine over the chunks.  Returns a dict with the per-step training loss
    (normalised units), the label scale and the validation error in nats.
    """
    rows = sur.rows()
    n_tr = rows - max(1, int(rows * val_frac)) if n_train is None else int(n_train)
    n_val = rows - n_tr
    if n_tr < 1 or n_val < 1:
        raise ValueError("not enough rows to train and validate")
    sur.fit_scale(0, n_tr)
    _, mean, scale = sur.get_params()
    lr_final = lr / 20.0 if lr_final is None else lr_final
    losses = []
    done = 0
    n_chunks = max(1, math.ceil(steps / chunk))
    for c in range(n_chunks):
        k = min(chunk, steps - done)
        if k <= 0:
            break
        rate = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * c / n_chunks))
        buf = torch.zeros(k, dtype=torch.float32, device="cuda")
        sur.train(0, n_tr, k, rate, seed, loss=buf)
        losses.append(buf)
        done += k
    torch.cuda.synchronize()
    loss = torch.cat(losses).cpu().numpy() if losses else None
    val = validate(sur, n_tr, rows)
    val.update(loss=loss, label_mean=mean, label_scale=scale, n_train=n_tr, n_val=n_val)
    return val


def validate(sur, begin, end):
    """Errors of the predictions on dataset rows [begin, end), in nats: over the exactly labelled
    rows, and the share of censored rows predicted above their floor."""
    pred = sur.predict_rows(begin, end)
    _, labels, cens = sur.dataset()
    lab = labels[begin:end].double()
    c = cens[begin:end].bool()
    err = (pred - lab)[~c].abs()
    above = (pred > lab)[c]
    torch.cuda.synchronize()
    return dict(val_rmse=float(err.pow(2).mean().sqrt()) if err.numel() else 0.0,
                val_max=float(err.max()) if err.numel() else 0.0,
                val_label_std=float(lab[~c].std()) if err.numel() > 1 else 0.0,
                val_censored=int(c.sum()), val_censored_above=float(above.double().mean()) if above.numel() else 0.0)
