"""Plain FP64 CPU oracle of SIR and pcSIR for 3D tracking (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the test suite and the CPU-baseline / reference arm
of ``bench.py`` use it.  It shares no code with the CUDA library.

The paper states its method for any state dimension (Section 4: bins over the
state space, "extended to higher-dimensional settings" in the outlook) and
evaluates it in 2D; this is the 3D form of Algorithms 1 and 2, written the
same way as the 2D oracle (``pcsir_oracle``), whose normalisation, ESS,
systematic resampling and posterior mean it reuses unchanged.  Readings:

* State (x, y, z, vx, vy, vz, I0); nearly-constant-velocity dynamics with a
  unit frame time, in the state precision:
  ``x += vx + e_x`` (likewise y, z), ``vx += e_vx`` (likewise vy, vz),
  ``I0 += e_I``.
* Cells: boxes of edges (hx, hy, hz) over position,
  ``b = floor((x + 1/2) / hx)`` per axis in the state precision, so unit
  edges are voxels centred on integers.
* Dummy: the mean of all seven components over the cell's members.
* Likelihood (Eq. object with an anisotropic Gaussian PSF, Eq. likelihood):
  over a Px x Py x Pz block of voxels centred on the nearest voxel
  (floor(x + 1/2), ...), with
  ``lambda = max(I0, 0) exp(-((vx - x)^2 + (vy - y)^2) / (2 s_xy^2) - (vz - z)^2 / (2 s_z^2)) + bg``
  and the Poisson term ``z log(lambda / z) - (lambda - z)``; voxels outside
  the volume contribute nothing.  The volume is indexed ``V[z, y, x]``.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import pcsir_oracle as O2

X, Y, Z, VX, VY, VZ, I0 = range(7)


@dataclasses.dataclass(frozen=True)
class Model3:
    sigma_xy: float = 1.5
    sigma_z: float = 3.0
    I0: float = 100.0
    bg: float = 10.0
    patch_xy: int = 11
    patch_z: int = 7
    q: tuple = (0.5, 0.5, 0.5, 0.1, 0.1, 0.1, 1.0)


def propagate(state: np.ndarray, noise: np.ndarray) -> np.ndarray:
    """3D nearly-constant-velocity transition in the state's own precision ([7, N] arrays)."""
    assert state.dtype == noise.dtype
    out = np.empty_like(state)
    for p, v in ((X, VX), (Y, VY), (Z, VZ)):
        out[p] = (state[p] + state[v]) + noise[p]
        out[v] = state[v] + noise[v]
    out[I0] = state[I0] + noise[I0]
    return out


def bin_coords(x, y, z, h):
    """Integer cell coordinates of positions, in the positions' precision; h = (hx, hy, hz)."""
    t = x.dtype.type
    half = t(0.5)
    out = []
    for c, hh in zip((x, y, z), h):
        out.append(np.floor((c + half) / t(hh)).astype(np.int64))
    return out


def segment(bx, by, bz):
    """Keys [B, 3] as (bx, by, bz) in ascending (bz, by, bx) order, member -> bin, counts."""
    keys = np.stack([bz, by, bx], axis=1)
    uk, member, counts = np.unique(keys, axis=0, return_inverse=True, return_counts=True)
    return uk[:, ::-1].copy(), member.reshape(-1), counts


def dummies(state, member_bin, n_bins):
    return O2.dummies(state, member_bin, n_bins)


def loglik(volume: np.ndarray, x, y, z, i0, model: Model3, chunk: int = 2048) -> np.ndarray:
    """Log-likelihood of positions (x, y, z) with intensity I0 against one volume (FP64)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64)
    i0 = np.asarray(i0, np.float64)
    D, H, W = volume.shape
    vol = volume.astype(np.float64)
    Rxy, Rz = model.patch_xy // 2, model.patch_z // 2
    oxy = np.arange(-Rxy, Rxy + 1, dtype=np.float64)
    oz = np.arange(-Rz, Rz + 1, dtype=np.float64)
    out = np.empty(x.shape[0])
    for s0 in range(0, x.shape[0], chunk):
        sl = slice(s0, s0 + chunk)
        cx, cy, cz = np.floor(x[sl] + 0.5), np.floor(y[sl] + 0.5), np.floor(z[sl] + 0.5)
        px = cx[:, None] + oxy[None, :]
        py = cy[:, None] + oxy[None, :]
        pz = cz[:, None] + oz[None, :]
        gx = np.exp(-((px - x[sl, None]) ** 2) / (2 * model.sigma_xy ** 2))
        gy = np.exp(-((py - y[sl, None]) ** 2) / (2 * model.sigma_xy ** 2))
        gz = np.exp(-((pz - z[sl, None]) ** 2) / (2 * model.sigma_z ** 2))
        lam = (np.maximum(i0[sl], 0.0)[:, None, None, None] * gz[:, :, None, None] * gy[:, None, :, None]
               * gx[:, None, None, :] + model.bg)
        ix, iy, iz = px.astype(np.int64), py.astype(np.int64), pz.astype(np.int64)
        inside = (((iz >= 0) & (iz < D))[:, :, None, None] & ((iy >= 0) & (iy < H))[:, None, :, None]
                  & ((ix >= 0) & (ix < W))[:, None, None, :])
        zz = vol[np.clip(iz, 0, D - 1)[:, :, None, None], np.clip(iy, 0, H - 1)[:, None, :, None],
                 np.clip(ix, 0, W - 1)[:, None, None, :]]
        with np.errstate(divide="ignore", invalid="ignore"):
            zlog = np.where(zz > 0, zz * np.log(lam / np.where(zz > 0, zz, 1.0)), 0.0)
        term = zlog - (lam - zz)
        out[sl] = np.where(inside, term, 0.0).sum(axis=(1, 2, 3))
    return out


def sir_step(state, volume, noise, u0, model: Model3):
    """Algorithm 1 in 3D, one time step, resampling at every step."""
    prop = propagate(state, noise)
    ll = loglik(volume, prop[X], prop[Y], prop[Z], prop[I0], model)
    w, m, T = O2.normalise(ll)
    anc = O2.systematic_resample(w, u0)
    return dict(prop=prop, ll=ll, w=w, max_logw=m, ess=O2.ess(w), estimate=O2.posterior_mean(w, prop),
                ancestors=anc, new_state=np.ascontiguousarray(prop[:, anc]))


def pcsir_step(state, volume, noise, u0, h, model: Model3):
    """Algorithm 2 in 3D, one time step, resampling at every step; h = (hx, hy, hz)."""
    prop = propagate(state, noise)
    bx, by, bz = bin_coords(prop[X], prop[Y], prop[Z], h)
    keys, member, counts = segment(bx, by, bz)
    dum = dummies(prop, member, keys.shape[0])
    ll_bins = loglik(volume, dum[X], dum[Y], dum[Z], dum[I0], model)
    ll = ll_bins[member]
    w, m, T = O2.normalise(ll)
    anc = O2.systematic_resample(w, u0)
    return dict(prop=prop, bin_keys=keys, bin_counts=counts, member_bin=member, dummies=dum, ll_bins=ll_bins,
                ll=ll, w=w, max_logw=m, ess=O2.ess(w), estimate=O2.posterior_mean(w, prop), ancestors=anc,
                new_state=np.ascontiguousarray(prop[:, anc]))
