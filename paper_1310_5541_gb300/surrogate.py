"""Training workflow of the likelihood surrogate on top of the C ABI.

The network and every training and inference pass run in the library's
kernels (``pcsir_surrogate.h``); this module only sequences the calls:

* ``collect`` runs exact pcSIR steps (Algorithm 2) over a frame sequence and
  appends every step's dummies with their exact log-likelihoods to the
  surrogate's dataset, so the training pairs come from the method itself;
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
