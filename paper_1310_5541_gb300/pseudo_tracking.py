"""The pseudo-tracking convergence experiment (Section 5.4) on the GPU.

Dynamics are left out: each repetition draws N particles from a fixed prior
around the true object position (``synth.pseudo_case``), weights them once
against a noisy image with the Gaussian (SSE) likelihood of Eq. (likelihood)
(sigma_xi = 20, 9 x 9 patch) and takes the posterior mean.  SIR, pcSIR-CoC
and pcSIR-CoM (cells = pixels, h = 1) see identical particles and images.

Two errors are reported per prior and particle count, as root mean squares
over the repetitions: the distance of the estimate to the exact posterior
mean of the same image and prior (midpoint rule on 0.005 px cells whose edges
include the pixel boundaries; likelihood from the library's own likelihood
entry point, prior density on the host), and its distance to the true
position.  The first isolates the Monte Carlo error, which falls as N^-1/2
for SIR, and pcSIR's cell discretisation; the second levels off at the
posterior's own spread.  Every step runs
through the C ABI (the filter step with zero process noise).
"""
from __future__ import annotations

import numpy as np
import torch

from . import pcsir, synth

METHODS = ("sir", "coc", "com")


def _axis_cells(lo, hi, spacing):
    """Midpoints and lengths of the integration cells on [lo, hi]: cell edges on a grid of
    ``spacing`` (1/spacing an integer) through the pixel boundaries k + 1/2, so the likelihood,
    which jumps where its patch shifts by a pixel, is smooth within every cell; the end cells are
    cut at lo and hi."""
    a = np.floor(lo - 0.5) + 0.5
    k0 = int(np.floor((lo - a) / spacing))
    k1 = int(np.ceil((hi - a) / spacing))
    e = a + spacing * np.arange(k0, k1 + 1)
    e[0], e[-1] = lo, hi
    e = np.unique(np.clip(e, lo, hi))
    return 0.5 * (e[:-1] + e[1:]), np.diff(e)


def posterior_mean(ctx, image, prior, x0, y0, i0, spacing=0.005):
    """Exact posterior mean of (x, y) under the prior centred on (x0, y0), by the midpoint rule on
    cells aligned with the pixel boundaries (see _axis_cells)."""
    if prior.startswith("uniform"):
        half = float(prior[len("uniform"):]) / 2.0
        sd = None
    else:
        sd = float(prior[len("gauss"):])
        half = 5.0 * sd
    mx, lx = _axis_cells(x0 - half, x0 + half, spacing)
    my, ly = _axis_cells(y0 - half, y0 + half, spacing)
    gx, gy = np.meshgrid(mx, my)
    area = np.outer(ly, lx).ravel()
    x = torch.from_numpy(gx.ravel()).cuda()
    y = torch.from_numpy(gy.ravel()).cuda()
    a = torch.full_like(x, i0)
    ll = pcsir.pcsir_loglik(ctx, x, y, a, image).cpu().numpy()
    logp = ll - ll.max()
    if sd is not None:
        logp = logp - ((gx.ravel() - x0) ** 2 + (gy.ravel() - y0) ** 2) / (2.0 * sd * sd)
    w = np.exp(logp - logp.max()) * area
    return float(np.sum(w * gx.ravel()) / w.sum()), float(np.sum(w * gy.ravel()) / w.sum())


def run(priors=synth.PSEUDO_PRIORS, counts=(1000, 10000, 100000), reps=200, seed=1310554500, h=1.0):
    """RMSE table: {prior: {method: [rmse per count]}}, plus the counts and repetitions."""
    nmax = max(counts)
    ctx = {m: pcsir.Context(nmax, torch.float32, lik="sse", patch=9, psf_sigma=1.16, bg=10.0, sigma_xi=20.0,
                            dummy="coc" if m == "coc" else "com") for m in METHODS}
    out, out_truth = {}, {}
    for prior in priors:
        tab = {m: [] for m in METHODS}
        tab_t = {m: [] for m in METHODS}
        for N in counts:
            zero = torch.zeros((5, N), dtype=torch.float32, device="cuda")
            err = {m: [] for m in METHODS}
            err_t = {m: [] for m in METHODS}
            for r in range(reps):
                img, _truth, st, u0 = synth.pseudo_case(prior, N, seed, r)
                d_img = torch.from_numpy(img).cuda()
                # the prior is centred on the truth, which pseudo_case draws first
                x0, y0 = _truth
                ref = posterior_mean(ctx["sir"], d_img, prior, x0, y0, float(st[4, 0]))
                d_st0 = torch.from_numpy(st).cuda()
                for m in METHODS:
                    s = d_st0.clone()
                    if m == "sir":
                        pcsir.sir_step(ctx[m], s, d_img, zero, u0)
                    else:
                        pcsir.pcsir_step(ctx[m], s, d_img, h, zero, u0)
                    torch.cuda.synchronize()
                    res = ctx[m].last_result()
                    err[m].append((res["estimate"][0] - ref[0]) ** 2 + (res["estimate"][1] - ref[1]) ** 2)
                    err_t[m].append((res["estimate"][0] - x0) ** 2 + (res["estimate"][1] - y0) ** 2)
            for m in METHODS:
                tab[m].append(float(np.sqrt(np.mean(err[m]))))
                tab_t[m].append(float(np.sqrt(np.mean(err_t[m]))))
        out[prior] = tab
        out_truth[prior] = tab_t
    for c in ctx.values():
        c.close()
    return {"counts": list(counts), "reps": reps, "rmse_px": out, "rmse_truth_px": out_truth}


def convergence_slope(counts, rmse):
    """Least-squares slope of log RMSE against log N (about -1/2 for a Monte Carlo method)."""
    return float(np.polyfit(np.log(np.asarray(counts, float)), np.log(np.asarray(rmse, float)), 1)[0])
