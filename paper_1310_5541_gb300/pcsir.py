"""Thin ctypes binding of ``libpcsir.so`` (see ``include/pcsir.h``).

Only argument marshalling happens here: every step of the filter runs in the
library's CUDA kernels.  Tensors are torch CUDA tensors (torch provides device
memory and streams); the current torch stream is used unless one is given.
Importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcsir.so")

# enums of pcsir.h
OK, EINVAL, ENOMEM, ECUDA, ETIMEDOUT, ESTATE, ENOTSUP, ERANGE = 0, -1, -2, -3, -4, -5, -6, -7
F32, F64 = 0, 1
LIK_POISSON, LIK_SSE = 0, 1
KEEP_ANCESTORS, KEEP_WEIGHTS, KEEP_PARTICLE_BIN, KEEP_LOGLIK, KEEP_QWEIGHTS = 1, 2, 4, 8, 16
DUMMY_COM, DUMMY_COC = 0, 1
DERR_RANGE, DERR_TIMEOUT, DERR_NONFINITE, DERR_ZEROSUM = 1, 2, 4, 8

_STATUS_NAMES = {0: "PCSIR_OK", -1: "PCSIR_EINVAL", -2: "PCSIR_ENOMEM", -3: "PCSIR_ECUDA",
                 -4: "PCSIR_ETIMEDOUT", -5: "PCSIR_ESTATE", -6: "PCSIR_ENOTSUP", -7: "PCSIR_ERANGE"}


class pcsir_config(ctypes.Structure):
    _fields_ = [("state_dtype", ctypes.c_int32), ("lik_kind", ctypes.c_int32), ("patch", ctypes.c_int32),
                ("keep", ctypes.c_int32), ("psf_sigma", ctypes.c_double), ("bg", ctypes.c_double),
                ("sigma_xi", ctypes.c_double), ("max_particles", ctypes.c_int64), ("dummy", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class pcsir_result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double * 5), ("ess", ctypes.c_double), ("max_loglik", ctypes.c_double),
                ("sum_wtilde", ctypes.c_double), ("n_particles", ctypes.c_int64), ("n_bins", ctypes.c_int64),
                ("device_error", ctypes.c_int32), ("kind", ctypes.c_int32), ("resampled", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class pcsir_outputs(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_bins", ctypes.c_int64), ("bin_stride", ctypes.c_int64),
                ("prop_state", ctypes.c_void_p), ("bin_xy", ctypes.c_void_p), ("bin_count", ctypes.c_void_p),
                ("dummy", ctypes.c_void_p), ("bin_loglik", ctypes.c_void_p), ("loglik", ctypes.c_void_p),
                ("particle_bin", ctypes.c_void_p), ("ancestor", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("qweight", ctypes.c_void_p)]


class pcsir_target(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("h", ctypes.c_double), ("psf_sigma", ctypes.c_double),
                ("bg", ctypes.c_double), ("patch", ctypes.c_int32), ("pad", ctypes.c_int32)]


class pcsir_surrogate_config(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("batch", ctypes.c_int32), ("geometry", ctypes.c_int32),
                ("i0_ref", ctypes.c_double), ("sigma_ref", ctypes.c_double), ("max_pixels", ctypes.c_int64)]


class pcsir_surrogate_check(ctypes.Structure):
    _fields_ = [("n_dummies", ctypes.c_int64), ("n_exact", ctypes.c_int64), ("n_holdout", ctypes.c_int64),
                ("n_significant", ctypes.c_int64), ("n_clipped", ctypes.c_int64), ("max_abs_err", ctypes.c_double),
                ("rms_err", ctypes.c_double), ("fallback", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# sizes of pcsir_surrogate.h
SUR_PATCH, SUR_INPUTS, SUR_HIDDEN = 21, 445, 256
SUR_NPARAMS = 256 * 445 + 256 + 256 * 256 + 256 + 256 + 1
SUR_ROW = 448  # stored inputs per dataset row
SUR3_NPARAMS = 256 * 852 + 256 + 256 * 256 + 256 + 256 + 1
SUR3_ROW = 896


class pcsir3_config(ctypes.Structure):
    _fields_ = [("patch_xy", ctypes.c_int32), ("patch_z", ctypes.c_int32), ("keep", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("psf_sigma_xy", ctypes.c_double), ("psf_sigma_z", ctypes.c_double),
                ("bg", ctypes.c_double), ("max_particles", ctypes.c_int64)]


class pcsir3_result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double * 7), ("ess", ctypes.c_double), ("max_loglik", ctypes.c_double),
                ("sum_wtilde", ctypes.c_double), ("n_particles", ctypes.c_int64), ("n_bins", ctypes.c_int64),
                ("device_error", ctypes.c_int32), ("kind", ctypes.c_int32)]


class pcsir3_outputs(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_bins", ctypes.c_int64), ("bin_stride", ctypes.c_int64),
                ("prop_state", ctypes.c_void_p), ("bin_xyz", ctypes.c_void_p), ("bin_count", ctypes.c_void_p),
                ("dummy", ctypes.c_void_p), ("bin_loglik", ctypes.c_void_p), ("loglik", ctypes.c_void_p),
                ("particle_bin", ctypes.c_void_p), ("ancestor", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("qweight", ctypes.c_void_p)]


class pcsir3_target(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("hx", ctypes.c_double), ("hy", ctypes.c_double),
                ("hz", ctypes.c_double), ("psf_sigma_xy", ctypes.c_double), ("psf_sigma_z", ctypes.c_double),
                ("bg", ctypes.c_double), ("patch_xy", ctypes.c_int32), ("patch_z", ctypes.c_int32)]


class pcsir3_batch_outputs(ctypes.Structure):
    _fields_ = [("n_total", ctypes.c_int64), ("n_bins", ctypes.c_int64), ("bin_stride", ctypes.c_int64),
                ("prop_state", ctypes.c_void_p), ("bin_key", ctypes.c_void_p), ("bin_count", ctypes.c_void_p),
                ("dummy", ctypes.c_void_p), ("bin_loglik", ctypes.c_void_p), ("particle_slot", ctypes.c_void_p),
                ("ancestor", ctypes.c_void_p), ("qweight", ctypes.c_void_p)]


class PcsirError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, status), msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpcsir.so is not built (expected at %s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    U64 = ctypes.c_uint64
    sig = {
        "pcsir_create": ([ctypes.POINTER(pcsir_config), ctypes.POINTER(ctypes.c_void_p)], I32),
        "pcsir_destroy": ([P], I32),
        "pcsir_step": ([P, P, I64, P, I32, I32, D, P, D, P, P], I32),
        "pcsir_deferred_begin": ([P, P, I64, P], I32),
        "pcsir_deferred_step": ([P, P, I32, I32, D, P, D, P, P], I32),
        "pcsir_deferred_state": ([P, P, P], I32),
        "pcsir_step_philox": ([P, P, I64, P, I32, I32, D, P, U64, U64, D, P, P], I32),
        "pcsir_deferred_step_philox": ([P, P, I32, I32, D, P, U64, U64, D, P, P], I32),
        "sir_step": ([P, P, I64, P, I32, I32, P, D, P, P], I32),
        "pcsir_step_ess": ([P, P, P, I64, P, I32, I32, D, P, D, D, P, P], I32),
        "sir_step_ess": ([P, P, P, I64, P, I32, I32, P, D, D, P, P], I32),
        "pcsir_loglik": ([P, P, P, P, I64, P, I32, I32, P, P], I32),
        "pcsir_resample": ([P, P, I64, D, P, P], I32),
        "pcsir_get_outputs": ([P, ctypes.POINTER(pcsir_outputs)], I32),
        "pcsir_last_result": ([P, ctypes.POINTER(pcsir_result)], I32),
        "pcsir_last_error": ([P], ctypes.c_char_p),
        "pcsir_version": ([], ctypes.c_char_p),
        "pcsir_resample_noalloc": ([P, I64, D, P, P], I32),
        "pcsir_timing_enable": ([P, I32], I32),
        "pcsir_save": ([P, ctypes.c_char_p], I32),
        "pcsir_load": ([P, ctypes.c_char_p], I32),
        "pcsir_batch_create": ([ctypes.POINTER(pcsir_target), I32, ctypes.POINTER(ctypes.c_void_p)], I32),
        "pcsir_batch_destroy": ([P], I32),
        "pcsir_batch_set_grid": ([P, I32], I32),
        "pcsir_batched_step": ([P, P, P, I32, I32, P, P, P], I32),
        "pcsir_batch_deferred_begin": ([P, P, P], I32),
        "pcsir_batched_deferred_step": ([P, P, I32, I32, P, P, P], I32),
        "pcsir_batch_deferred_state": ([P, P, P], I32),
        "pcsir_batch_results": ([P, ctypes.POINTER(pcsir_result), I32, ctypes.POINTER(ctypes.c_int32)], I32),
        "pcsir_batch_outputs": ([P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)], I32),
        "pcsir_batch_bins": ([P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                              ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)], I32),
        "pcsir_batch_last_error": ([P], ctypes.c_char_p),
        "pcsir_batch_phase_times": ([P, ctypes.POINTER(ctypes.c_double), I32], I32),
        "pcsir_batch_set_wait": ([P, I32, I32], I32),
        "pcsir_batch_set_table": ([P, I32], I32),
        "pcsir_batch_keep": ([P, I32], I32),
        "pcsir_batch_kept": ([P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p)], I32),
        "pcsir_gemm_bf16": ([P, I64, I64, P, I64, I64, P, I64, I32, I32, I32, I32, P], I32),
        "pcsir_timing_read": ([P, ctypes.POINTER(ctypes.c_float), I32, ctypes.POINTER(ctypes.c_int32)], I32),
        "pcsir_surrogate_create": ([ctypes.POINTER(pcsir_surrogate_config), ctypes.POINTER(ctypes.c_void_p)], I32),
        "pcsir_surrogate_destroy": ([P], I32),
        "pcsir_surrogate_last_error": ([P], ctypes.c_char_p),
        "pcsir_surrogate_init": ([P, ctypes.c_uint64, P], I32),
        "pcsir_surrogate_set_params": ([P, P, D, D], I32),
        "pcsir_surrogate_get_params": ([P, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], I32),
        "pcsir_surrogate_add": ([P, P, I64, I64, P, D, P, I32, I32, D, D, P], I32),
        "pcsir_surrogate_rows": ([P, ctypes.POINTER(ctypes.c_int64)], I32),
        "pcsir_surrogate_clear": ([P, P], I32),
        "pcsir_surrogate_dataset": ([P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.POINTER(ctypes.c_void_p)], I32),
        "pcsir_surrogate_fit_scale": ([P, I64, I64], I32),
        "pcsir_surrogate_train": ([P, I64, I64, I32, D, ctypes.c_uint64, P, P], I32),
        "pcsir_surrogate_grads": ([P, I64, I32, P, ctypes.POINTER(ctypes.c_double)], I32),
        "pcsir_surrogate_predict_rows": ([P, I64, I64, P, P], I32),
        "pcsir_surrogate_predict": ([P, P, I64, I64, P, I32, I32, D, D, P, P], I32),
        "pcsir_attach_surrogate": ([P, P, D, I32, D, D], I32),
        "pcsir3_create": ([ctypes.POINTER(pcsir3_config), ctypes.POINTER(ctypes.c_void_p)], I32),
        "pcsir3_destroy": ([P], I32),
        "pcsir3_last_error": ([P], ctypes.c_char_p),
        "pcsir3_step": ([P, P, I64, P, I32, I32, I32, D, D, D, P, D, P, P], I32),
        "sir3_step": ([P, P, I64, P, I32, I32, I32, P, D, P, P], I32),
        "pcsir3_get_outputs": ([P, ctypes.POINTER(pcsir3_outputs)], I32),
        "pcsir3_last_result": ([P, ctypes.POINTER(pcsir3_result)], I32),
        "pcsir_surrogate_last_check": ([P, ctypes.POINTER(pcsir_surrogate_check)], I32),
        "pcsir_surrogate_add3": ([P, P, I64, I64, P, D, P, I32, I32, I32, D, D, P], I32),
        "pcsir_surrogate_predict3": ([P, P, I64, I64, P, I32, I32, I32, D, D, P, P], I32),
        "pcsir_surrogate_nparams": ([P, ctypes.POINTER(ctypes.c_int64)], I32),
        "pcsir3_attach_surrogate": ([P, P, D, I32, D, D], I32),
        "pcsir3_surrogate_last_check": ([P, ctypes.POINTER(pcsir_surrogate_check)], I32),
        "pcsir3_batch_create": ([ctypes.POINTER(pcsir3_target), I32, I32, ctypes.POINTER(ctypes.c_void_p)], I32),
        "pcsir3_batch_destroy": ([P], I32),
        "pcsir3_batch_last_error": ([P], ctypes.c_char_p),
        "pcsir3_batched_step": ([P, P, P, I32, I32, I32, P, P, P], I32),
        "pcsir3_batch_results": ([P, ctypes.POINTER(pcsir3_result), I32, ctypes.POINTER(ctypes.c_int32)], I32),
        "pcsir3_batch_get_outputs": ([P, ctypes.POINTER(pcsir3_batch_outputs)], I32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_cuda(t, name, dtype=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))


class Context:
    """Owns one ``pcsir_ctx`` (workspace for up to ``max_particles`` particles)."""

    def __init__(self, max_particles, state_dtype=torch.float32, lik="poisson", patch=9, psf_sigma=1.5,
                 bg=10.0, sigma_xi=20.0, keep=0, dummy="com"):
        self.torch_dtype = state_dtype
        cfg = pcsir_config(state_dtype=F32 if state_dtype == torch.float32 else F64,
                           lik_kind=LIK_POISSON if lik == "poisson" else LIK_SSE, patch=int(patch), keep=int(keep),
                           psf_sigma=float(psf_sigma), bg=float(bg), sigma_xi=float(sigma_xi),
                           max_particles=int(max_particles), dummy=DUMMY_COC if dummy == "coc" else DUMMY_COM,
                           reserved=0)
        h = ctypes.c_void_p()
        st = lib.pcsir_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise PcsirError(st, "pcsir_create failed")
        self.handle = h
        self.cfg = cfg

    def close(self):
        if getattr(self, "handle", None):
            lib.pcsir_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st):
        raise PcsirError(st, lib.pcsir_last_error(self.handle).decode())

    def last_result(self):
        """The last step's pcsir_result as a dict (synchronise the step's stream first)."""
        r = pcsir_result()
        lib.pcsir_last_result(self.handle, ctypes.byref(r))
        return dict(estimate=list(r.estimate), ess=r.ess, max_loglik=r.max_loglik, sum_wtilde=r.sum_wtilde,
                    n_particles=r.n_particles, n_bins=r.n_bins, device_error=r.device_error, kind=r.kind,
                    resampled=bool(r.resampled))

    def save(self, path):
        """Checkpoint of the context's state between steps (see pcsir_save)."""
        st = lib.pcsir_save(self.handle, os.fsencode(path))
        if st != OK:
            self._raise(st)

    def load(self, path):
        """Restore a checkpoint written by ``save`` (attach the surrogate first if it holds one)."""
        st = lib.pcsir_load(self.handle, os.fsencode(path))
        if st != OK:
            self._raise(st)

    def timing_enable(self, max_steps):
        st = lib.pcsir_timing_enable(self.handle, int(max_steps))
        if st != OK:
            self._raise(st)

    def timing_read(self, max_steps):
        """Per-step stage durations in ms, shape [n_steps, 4] (waits for the recorded steps)."""
        buf = (ctypes.c_float * (4 * max_steps))()
        n = ctypes.c_int32()
        st = lib.pcsir_timing_read(self.handle, buf, 4 * max_steps, ctypes.byref(n))
        if st != OK:
            self._raise(st)
        return [list(buf[4 * k:4 * k + 4]) for k in range(n.value)]

    def outputs(self):
        """Intermediates of the last step as torch tensors (views, valid until the next step)."""
        o = pcsir_outputs()
        st = lib.pcsir_get_outputs(self.handle, ctypes.byref(o))
        if st != OK:
            self._raise(st)
        N, B, S = o.n_particles, o.n_bins, o.bin_stride
        sd = self.torch_dtype

        def view(ptr, shape, dtype):
            if not ptr:
                return None
            return _from_ptr(ptr, shape, dtype)

        out = dict(n_particles=N, n_bins=B,
                   prop_state=view(o.prop_state, (5, N), sd),
                   ancestor=view(o.ancestor, (N,), torch.int32),
                   weight=view(o.weight, (N,), torch.float64),
                   qweight=view(o.qweight, (N,), torch.int64))
        if B > 0:
            out.update(bin_xy=view(o.bin_xy, (2, S), torch.int32)[:, :B],
                       bin_count=view(o.bin_count, (B,), torch.int32),
                       dummy=view(o.dummy, (5, S), torch.float64)[:, :B],
                       bin_loglik=view(o.bin_loglik, (B,), torch.float64),
                       particle_bin=view(o.particle_bin, (N,), torch.int32))
        if o.loglik:
            out["loglik"] = view(o.loglik, (N,), torch.float64)
        return out


class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 2, "strides": None}


_TYPESTR = {torch.float32: "<f4", torch.float64: "<f8", torch.int32: "<i4", torch.int64: "<i8",
            torch.int16: "<i2", torch.uint8: "|u1"}


def _from_ptr(ptr, shape, dtype):
    return torch.as_tensor(_CudaArray(ptr, shape, _TYPESTR[dtype]), device="cuda")


def pcsir_step(ctx, state, image, h, noise, u0, stream=None):
    """One pcSIR step (Algorithm 2) on ``state`` [5, N] in place."""
    _check_cuda(state, "state", ctx.torch_dtype)
    _check_cuda(noise, "noise", ctx.torch_dtype)
    _check_cuda(image, "image", torch.float32)
    N = state.shape[1]
    H, W = image.shape
    st = lib.pcsir_step(ctx.handle, _ptr(state), N, _ptr(image), W, H, float(h), _ptr(noise), float(u0),
                        _stream_ptr(stream), None)
    if st != OK:
        ctx._raise(st)


def pcsir_deferred_begin(ctx, state, stream=None):
    """Start a deferred-resampling run from the states ``state`` [5, N] (copied into the context)."""
    _check_cuda(state, "state", ctx.torch_dtype)
    st = lib.pcsir_deferred_begin(ctx.handle, _ptr(state), state.shape[1], _stream_ptr(stream))
    if st != OK:
        ctx._raise(st)


def pcsir_deferred_step(ctx, image, h, noise, u0, stream=None):
    """One pcSIR step of the context's deferred run (Algorithm 2; resampling recorded as ancestors)."""
    _check_cuda(noise, "noise", ctx.torch_dtype)
    _check_cuda(image, "image", torch.float32)
    H, W = image.shape
    st = lib.pcsir_deferred_step(ctx.handle, _ptr(image), W, H, float(h), _ptr(noise), float(u0),
                                 _stream_ptr(stream), None)
    if st != OK:
        ctx._raise(st)


def _q5(q):
    q = [float(x) for x in q]
    if len(q) != 5:
        raise ValueError("q holds the five standard deviations of the increments")
    return (ctypes.c_double * 5)(*q)  # ctypes passes the array as a pointer to its first element


def pcsir_step_philox(ctx, state, image, h, q, seed, frame, u0, stream=None):
    """One pcSIR step (Algorithm 2) on ``state`` [5, N] in place, the process noise drawn in the kernel."""
    _check_cuda(state, "state", ctx.torch_dtype)
    _check_cuda(image, "image", torch.float32)
    N = state.shape[1]
    H, W = image.shape
    st = lib.pcsir_step_philox(ctx.handle, _ptr(state), N, _ptr(image), W, H, float(h), _q5(q), int(seed),
                               int(frame), float(u0), _stream_ptr(stream), None)
    if st != OK:
        ctx._raise(st)


def pcsir_deferred_step_philox(ctx, image, h, q, seed, frame, u0, stream=None):
    """One step of the context's deferred run with the process noise drawn in the kernel."""
    _check_cuda(image, "image", torch.float32)
    H, W = image.shape
    st = lib.pcsir_deferred_step_philox(ctx.handle, _ptr(image), W, H, float(h), _q5(q), int(seed), int(frame),
                                        float(u0), _stream_ptr(stream), None)
    if st != OK:
        ctx._raise(st)


def pcsir_deferred_state(ctx, state, stream=None):
    """Write the deferred run's current resampled states into ``state`` [5, N]."""
    _check_cuda(state, "state", ctx.torch_dtype)
    st = lib.pcsir_deferred_state(ctx.handle, _ptr(state), _stream_ptr(stream))
    if st != OK:
        ctx._raise(st)


def sir_step(ctx, state, image, noise, u0, stream=None):
    """One SIR step (Algorithm 1) on ``state`` [5, N] in place."""
    _check_cuda(state, "state", ctx.torch_dtype)
    _check_cuda(noise, "noise", ctx.torch_dtype)
    _check_cuda(image, "image", torch.float32)
    N = state.shape[1]
    H, W = image.shape
    st = lib.sir_step(ctx.handle, _ptr(state), N, _ptr(image), W, H, _ptr(noise), float(u0),
                      _stream_ptr(stream), None)
    if st != OK:
        ctx._raise(st)


# carried log-weights of the ESS-thresholded steps: int64, log w = logw * 2^-32
LOGW_SCALE = 4294967296.0


def pcsir_step_ess(ctx, state, logw, image, h, noise, u0, ess_min, stream=None):
    """One ESS-thresholded pcSIR step on ``state`` [5, N] (FP32) and the carried fixed-point
    log-weights ``logw`` [N] (int64) in place; resamples only when N_eff < ess_min."""
    _check_cuda(state, "state", torch.float32)
    _check_cuda(noise, "noise", torch.float32)
    _check_cuda(image, "image", torch.float32)
    _check_cuda(logw, "logw", torch.int64)
    N = state.shape[1]
    H, W = image.shape
    st = lib.pcsir_step_ess(ctx.handle, _ptr(state), _ptr(logw), N, _ptr(image), W, H, float(h), _ptr(noise),
                            float(u0), float(ess_min), _stream_ptr(stream), None)
    if st != OK:
        ctx._raise(st)


def sir_step_ess(ctx, state, logw, image, noise, u0, ess_min, stream=None):
    """One ESS-thresholded SIR step (Algorithm 1 with its resampling test), in place."""
    _check_cuda(state, "state", torch.float32)
    _check_cuda(noise, "noise", torch.float32)
    _check_cuda(image, "image", torch.float32)
    _check_cuda(logw, "logw", torch.int64)
    N = state.shape[1]
    H, W = image.shape
    st = lib.sir_step_ess(ctx.handle, _ptr(state), _ptr(logw), N, _ptr(image), W, H, _ptr(noise), float(u0),
                          float(ess_min), _stream_ptr(stream), None)
    if st != OK:
        ctx._raise(st)


def pcsir_loglik(ctx, x, y, i0, image, out=None, stream=None):
    """Log-likelihood of positions (float64 CUDA tensors) against ``image``."""
    for t, n in ((x, "x"), (y, "y"), (i0, "I0")):
        _check_cuda(t, n, torch.float64)
    _check_cuda(image, "image", torch.float32)
    if out is None:
        out = torch.empty_like(x)
    H, W = image.shape
    st = lib.pcsir_loglik(ctx.handle, _ptr(x), _ptr(y), _ptr(i0), x.numel(), _ptr(image), W, H, _ptr(out),
                          _stream_ptr(stream))
    if st != OK:
        ctx._raise(st)
    return out


def pcsir_resample(ctx, logw, u0, out=None, stream=None):
    """Systematic-resampling ancestors (int32) of ``logw`` (float64 CUDA tensor)."""
    _check_cuda(logw, "logw", torch.float64)
    if out is None:
        out = torch.empty(logw.numel(), dtype=torch.int32, device=logw.device)
    st = lib.pcsir_resample(ctx.handle, _ptr(logw), logw.numel(), float(u0), _ptr(out), _stream_ptr(stream))
    if st != OK:
        ctx._raise(st)
    return out


def pcsir_resample_noalloc(logw, u0, out=None, stream=None):
    """Systematic-resampling ancestors without a context and without device allocation
    (scratch in a fixed library-owned device array; N <= 2^22; calls must not overlap)."""
    _check_cuda(logw, "logw", torch.float64)
    if out is None:
        out = torch.empty(logw.numel(), dtype=torch.int32, device=logw.device)
    _check_cuda(out, "ancestors", torch.int32)
    # the library takes its scratch from the current device: every operand must live there
    dev = torch.cuda.current_device()
    if logw.device.index != dev or out.device.index != dev:
        raise ValueError("logw and out must be on the current CUDA device (cuda:%d)" % dev)
    if stream is not None and stream.device.index != dev:
        raise ValueError("the stream must belong to the current CUDA device (cuda:%d)" % dev)
    st = lib.pcsir_resample_noalloc(_ptr(logw), logw.numel(), float(u0), _ptr(out), _stream_ptr(stream))
    if st != OK:
        raise PcsirError(st, "pcsir_resample_noalloc failed")
    return out


class Batch:
    """Owns one ``pcsir_batch``: T targets filtered together (FP32 state, Poisson likelihood)."""

    def __init__(self, n, h, psf_sigma, bg, patch):
        T = len(n)
        arr = (pcsir_target * T)()
        for t in range(T):
            arr[t] = pcsir_target(int(n[t]), float(h[t]), float(psf_sigma[t]), float(bg if np.isscalar(bg) else bg[t]),
                                  int(patch[t]), 0)
        hdl = ctypes.c_void_p()
        st = lib.pcsir_batch_create(arr, T, ctypes.byref(hdl))
        if st != OK:
            raise PcsirError(st, "pcsir_batch_create failed")
        self.handle = hdl
        self.T = T
        self.n_total = int(sum(int(x) for x in n))

    def close(self):
        if getattr(self, "handle", None):
            lib.pcsir_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, state, image, noise, u0, stream=None):
        """One step of every target (state [5, sum N] float32 in place; u0 float64 [T] on the device)."""
        _check_cuda(state, "state", torch.float32)
        _check_cuda(noise, "noise", torch.float32)
        _check_cuda(image, "image", torch.float32)
        _check_cuda(u0, "u0", torch.float64)
        H, W = image.shape
        st = lib.pcsir_batched_step(self.handle, _ptr(state), _ptr(image), W, H, _ptr(noise), _ptr(u0),
                                    _stream_ptr(stream))
        if st != OK:
            raise PcsirError(st, lib.pcsir_batch_last_error(self.handle).decode())

    def deferred_begin(self, state, stream=None):
        """Start a deferred-resampling run from state [5, sum N] float32 (copied)."""
        _check_cuda(state, "state", torch.float32)
        st = lib.pcsir_batch_deferred_begin(self.handle, _ptr(state), _stream_ptr(stream))
        if st != OK:
            raise PcsirError(st, lib.pcsir_batch_last_error(self.handle).decode())

    def deferred_step(self, image, noise, u0, stream=None):
        """One step of every target of the run (the resampling records ancestors; the next step gathers)."""
        _check_cuda(noise, "noise", torch.float32)
        _check_cuda(image, "image", torch.float32)
        _check_cuda(u0, "u0", torch.float64)
        H, W = image.shape
        st = lib.pcsir_batched_deferred_step(self.handle, _ptr(image), W, H, _ptr(noise), _ptr(u0),
                                             _stream_ptr(stream))
        if st != OK:
            raise PcsirError(st, lib.pcsir_batch_last_error(self.handle).decode())

    def deferred_state(self, out, stream=None):
        """Write the run's current resampled states into out [5, sum N] float32."""
        _check_cuda(out, "out", torch.float32)
        st = lib.pcsir_batch_deferred_state(self.handle, _ptr(out), _stream_ptr(stream))
        if st != OK:
            raise PcsirError(st, lib.pcsir_batch_last_error(self.handle).decode())

    def phase_times(self):
        """Durations (ms) of the last step's seven phases (synchronises)."""
        buf = (ctypes.c_double * 7)()
        st = lib.pcsir_batch_phase_times(self.handle, buf, 7)
        if st != OK:
            raise PcsirError(st, "pcsir_batch_phase_times failed")
        return list(buf)

    def set_grid(self, blocks_per_sm):
        st = lib.pcsir_batch_set_grid(self.handle, int(blocks_per_sm))
        if st != OK:
            raise PcsirError(st, "pcsir_batch_set_grid failed")

    def set_table(self, table_bits):
        """2^table_bits slots in each block's cell table (9 .. 11; results do not depend on it)."""
        st = lib.pcsir_batch_set_table(self.handle, int(table_bits))
        if st != OK:
            raise PcsirError(st, "pcsir_batch_set_table failed")

    def set_wait(self, max_polls=1 << 22, unreachable_barrier=-1):
        """Bound of each grid-barrier wait, and a barrier made unreachable (tests of the timeout)."""
        st = lib.pcsir_batch_set_wait(self.handle, int(max_polls), int(unreachable_barrier))
        if st != OK:
            raise PcsirError(st, "pcsir_batch_set_wait failed")

    def keep(self, flags):
        """Keep per-particle ancestors (KEEP_ANCESTORS) and integer weights (KEEP_QWEIGHTS) of later steps."""
        st = lib.pcsir_batch_keep(self.handle, int(flags))
        if st != OK:
            raise PcsirError(st, "pcsir_batch_keep failed")

    def kept(self):
        """The kept per-particle arrays of the last step (None where not kept)."""
        anc, q = ctypes.c_void_p(), ctypes.c_void_p()
        st = lib.pcsir_batch_kept(self.handle, ctypes.byref(anc), ctypes.byref(q))
        if st != OK:
            raise PcsirError(st, "pcsir_batch_kept failed")
        n = self.n_total
        return dict(ancestor=_from_ptr(anc.value, (n,), torch.int32) if anc.value else None,
                    qweight=_from_ptr(q.value, (n,), torch.int64) if q.value else None)

    def results(self):
        """Per-target results of the last step and the step's device error flags (synchronises).
        A step whose barrier wait gave up returns its flags (with DERR_TIMEOUT) rather than raising."""
        arr = (pcsir_result * self.T)()
        err = ctypes.c_int32()
        st = lib.pcsir_batch_results(self.handle, arr, self.T, ctypes.byref(err))
        if st not in (OK, ETIMEDOUT):
            raise PcsirError(st, "pcsir_batch_results failed")
        out = [dict(estimate=list(r.estimate), ess=r.ess, n_bins=r.n_bins, n_particles=r.n_particles,
                    device_error=r.device_error) for r in arr]
        return out, err.value

    def outputs(self):
        prop, stride, slot, n = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_int64()
        lib.pcsir_batch_outputs(self.handle, ctypes.byref(prop), ctypes.byref(stride), ctypes.byref(slot),
                                ctypes.byref(n))
        keys, cnts, ll, nb = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        lib.pcsir_batch_bins(self.handle, ctypes.byref(keys), ctypes.byref(cnts), ctypes.byref(ll), ctypes.byref(nb))
        B = nb.value
        return dict(prop_state=_from_ptr(prop.value, (5, stride.value), torch.float32)[:, :n.value],
                    bin_key=_from_ptr(keys.value, (B,), torch.int64) if B else None,
                    bin_count=_from_ptr(cnts.value, (B,), torch.int32) if B else None,
                    bin_loglik=_from_ptr(ll.value, (B,), torch.float64) if B else None)


def gemm_bf16(A, B, C=None, accumulate=False, stream=None):
    """C (+)= A @ B.T on the tensor cores (A [M, K], B [N, K] bfloat16 views with any strides;
    C [M, N] float32)."""
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_cuda and B.is_cuda
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    st = lib.pcsir_gemm_bf16(_ptr(A), A.stride(0), A.stride(1), _ptr(B), B.stride(0), B.stride(1), _ptr(C),
                             C.stride(0), M, N, K, int(bool(accumulate)), _stream_ptr(stream))
    if st != OK:
        raise PcsirError(st, "pcsir_gemm_bf16 failed")
    return C


def version():
    return lib.pcsir_version().decode()


class Surrogate:
    """Owns one ``pcsir_surrogate``: the likelihood network, its training state and its dataset."""

    def __init__(self, capacity, batch=4096, i0_ref=128.0, sigma_ref=1.5, max_pixels=1 << 20, geometry=2):
        self.geometry = int(geometry)
        self.nparams = SUR3_NPARAMS if self.geometry == 3 else SUR_NPARAMS
        self.row = SUR3_ROW if self.geometry == 3 else SUR_ROW
        cfg = pcsir_surrogate_config(capacity=int(capacity), batch=int(batch), geometry=self.geometry,
                                     i0_ref=float(i0_ref),
                                     sigma_ref=float(sigma_ref), max_pixels=int(max_pixels))
        h = ctypes.c_void_p()
        st = lib.pcsir_surrogate_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise PcsirError(st, "pcsir_surrogate_create failed")
        self.handle = h
        self.cfg = cfg

    def close(self):
        if getattr(self, "handle", None):
            lib.pcsir_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise PcsirError(st, lib.pcsir_surrogate_last_error(self.handle).decode())

    def init(self, seed, stream=None):
        self._check(lib.pcsir_surrogate_init(self.handle, int(seed), _stream_ptr(stream)))

    def set_params(self, flat, label_mean=0.0, label_scale=1.0):
        a = np.ascontiguousarray(np.asarray(flat, np.float32))
        assert a.size == self.nparams
        self._check(lib.pcsir_surrogate_set_params(self.handle, a.ctypes.data, float(label_mean), float(label_scale)))

    def get_params(self):
        a = np.empty(self.nparams, np.float32)
        m, s = ctypes.c_double(), ctypes.c_double()
        self._check(lib.pcsir_surrogate_get_params(self.handle, a.ctypes.data, ctypes.byref(m), ctypes.byref(s)))
        return a, m.value, s.value

    def add(self, dummy, ll, image, bg, psf_sigma, label_floor=-math.inf, stream=None):
        """Append rows for the states ``dummy`` [5, n] (float64 view with unit column stride) with labels
        max(``ll``, ``label_floor``)."""
        assert dummy.dtype == torch.float64 and dummy.is_cuda and dummy.stride(1) == 1
        _check_cuda(ll, "ll", torch.float64)
        _check_cuda(image, "image", torch.float32)
        n = dummy.shape[1]
        H, W = image.shape
        self._check(lib.pcsir_surrogate_add(self.handle, _ptr(dummy), dummy.stride(0), n, _ptr(ll),
                                            float(label_floor), _ptr(image), W, H, float(bg), float(psf_sigma),
                                            _stream_ptr(stream)))

    def rows(self):
        n = ctypes.c_int64()
        self._check(lib.pcsir_surrogate_rows(self.handle, ctypes.byref(n)))
        return n.value

    def clear(self, stream=None):
        self._check(lib.pcsir_surrogate_clear(self.handle, _stream_ptr(stream)))

    def dataset(self):
        """(inputs [rows, 448] as int16 bit patterns of bf16, labels [rows] float32, censored [rows] uint8) views."""
        xp, yp, cp = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self._check(lib.pcsir_surrogate_dataset(self.handle, ctypes.byref(xp), ctypes.byref(yp), ctypes.byref(cp)))
        n = self.rows()
        if n == 0:
            return None, None, None
        return (_from_ptr(xp.value, (n, self.row), torch.int16), _from_ptr(yp.value, (n,), torch.float32),
                _from_ptr(cp.value, (n,), torch.uint8))

    def fit_scale(self, begin, end):
        self._check(lib.pcsir_surrogate_fit_scale(self.handle, int(begin), int(end)))

    def train(self, begin, end, steps, lr, seed, loss=None, stream=None):
        if loss is not None:
            _check_cuda(loss, "loss", torch.float32)
            assert loss.numel() >= steps
        self._check(lib.pcsir_surrogate_train(self.handle, int(begin), int(end), int(steps), float(lr), int(seed),
                                              _ptr(loss), _stream_ptr(stream)))

    def grads(self, begin, n):
        g = np.empty(self.nparams, np.float32)
        loss = ctypes.c_double()
        self._check(lib.pcsir_surrogate_grads(self.handle, int(begin), int(n), g.ctypes.data, ctypes.byref(loss)))
        return g, loss.value

    def predict_rows(self, begin, end, out=None, stream=None):
        """Predictions of dataset rows in label units (the residual, without the window term)."""
        if out is None:
            out = torch.empty(end - begin, dtype=torch.float64, device="cuda")
        self._check(lib.pcsir_surrogate_predict_rows(self.handle, int(begin), int(end), _ptr(out), _stream_ptr(stream)))
        return out

    def predict(self, dummy, image, bg, psf_sigma, out=None, stream=None):
        assert dummy.dtype == torch.float64 and dummy.is_cuda and dummy.stride(1) == 1
        _check_cuda(image, "image", torch.float32)
        n = dummy.shape[1]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=dummy.device)
        H, W = image.shape
        self._check(lib.pcsir_surrogate_predict(self.handle, _ptr(dummy), dummy.stride(0), n, _ptr(image), W, H,
                                                float(bg), float(psf_sigma), _ptr(out), _stream_ptr(stream)))
        return out


def _surrogate_add3(self, dummy, ll, volume, bg, psf_sigma_xy, label_floor=-math.inf, stream=None):
    """Append rows for the 3D states ``dummy`` [7, n] (float64 view with unit column stride)."""
    assert dummy.dtype == torch.float64 and dummy.is_cuda and dummy.stride(1) == 1
    _check_cuda(ll, "ll", torch.float64)
    _check_cuda(volume, "volume", torch.float32)
    n = dummy.shape[1]
    D, H, W = volume.shape
    self._check(lib.pcsir_surrogate_add3(self.handle, _ptr(dummy), dummy.stride(0), n, _ptr(ll), float(label_floor),
                                         _ptr(volume), W, H, D, float(bg), float(psf_sigma_xy), _stream_ptr(stream)))


def _surrogate_predict3(self, dummy, volume, bg, psf_sigma_xy, out=None, stream=None):
    assert dummy.dtype == torch.float64 and dummy.is_cuda and dummy.stride(1) == 1
    _check_cuda(volume, "volume", torch.float32)
    n = dummy.shape[1]
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=dummy.device)
    D, H, W = volume.shape
    self._check(lib.pcsir_surrogate_predict3(self.handle, _ptr(dummy), dummy.stride(0), n, _ptr(volume), W, H, D,
                                             float(bg), float(psf_sigma_xy), _ptr(out), _stream_ptr(stream)))
    return out


Surrogate.add3 = _surrogate_add3
Surrogate.predict3 = _surrogate_predict3


def attach_surrogate3(ctx3, sur, holdout_frac=0.02, min_holdout=32, window=20.0, max_err=1.0):
    """Let the 3D step of ``ctx3`` use the 3D surrogate ``sur`` (``sur=None`` detaches)."""
    st = lib.pcsir3_attach_surrogate(ctx3.handle, sur.handle if sur is not None else None, float(holdout_frac),
                                     int(min_holdout), float(window), float(max_err))
    if st != OK:
        ctx3._raise(st)
    ctx3.surrogate = sur


def surrogate_last_check3(ctx3):
    c = pcsir_surrogate_check()
    st = lib.pcsir3_surrogate_last_check(ctx3.handle, ctypes.byref(c))
    if st != OK:
        ctx3._raise(st)
    return {k: getattr(c, k) for k, _ in pcsir_surrogate_check._fields_ if k != "reserved"}


def attach_surrogate(ctx, sur, holdout_frac=0.02, min_holdout=32, window=20.0, max_err=1.0):
    """Let ``pcsir_step`` on ``ctx`` use ``sur`` for the dummies' log-likelihoods (``sur=None`` detaches)."""
    st = lib.pcsir_attach_surrogate(ctx.handle, sur.handle if sur is not None else None, float(holdout_frac),
                                    int(min_holdout), float(window), float(max_err))
    if st != OK:
        ctx._raise(st)
    ctx.surrogate = sur


def surrogate_last_check(ctx):
    c = pcsir_surrogate_check()
    st = lib.pcsir_surrogate_last_check(ctx.handle, ctypes.byref(c))
    if st != OK:
        ctx._raise(st)
    return {k: getattr(c, k) for k, _ in pcsir_surrogate_check._fields_ if k != "reserved"}


class Context3:
    """Owns one ``pcsir3_ctx``: 3D tracking, state (x, y, z, vx, vy, vz, I0) float32 [7, N]."""

    def __init__(self, max_particles, patch_xy=11, patch_z=7, psf_sigma_xy=1.5, psf_sigma_z=3.0, bg=10.0, keep=0):
        cfg = pcsir3_config(patch_xy=int(patch_xy), patch_z=int(patch_z), keep=int(keep), reserved=0,
                            psf_sigma_xy=float(psf_sigma_xy), psf_sigma_z=float(psf_sigma_z), bg=float(bg),
                            max_particles=int(max_particles))
        h = ctypes.c_void_p()
        st = lib.pcsir3_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise PcsirError(st, "pcsir3_create failed")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib.pcsir3_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st):
        raise PcsirError(st, lib.pcsir3_last_error(self.handle).decode())

    def step(self, state, volume, h, noise, u0, stream=None):
        """One 3D pcSIR step on ``state`` [7, N] in place; ``volume`` float32 [D, H, W]; h = (hx, hy, hz)."""
        _check_cuda(state, "state", torch.float32)
        _check_cuda(noise, "noise", torch.float32)
        _check_cuda(volume, "volume", torch.float32)
        D, H, W = volume.shape
        st = lib.pcsir3_step(self.handle, _ptr(state), state.shape[1], _ptr(volume), W, H, D, float(h[0]), float(h[1]),
                             float(h[2]), _ptr(noise), float(u0), _stream_ptr(stream), None)
        if st != OK:
            self._raise(st)

    def sir_step(self, state, volume, noise, u0, stream=None):
        _check_cuda(state, "state", torch.float32)
        _check_cuda(noise, "noise", torch.float32)
        _check_cuda(volume, "volume", torch.float32)
        D, H, W = volume.shape
        st = lib.sir3_step(self.handle, _ptr(state), state.shape[1], _ptr(volume), W, H, D, _ptr(noise), float(u0),
                           _stream_ptr(stream), None)
        if st != OK:
            self._raise(st)

    def last_result(self):
        r = pcsir3_result()
        lib.pcsir3_last_result(self.handle, ctypes.byref(r))
        return dict(estimate=list(r.estimate), ess=r.ess, max_loglik=r.max_loglik, sum_wtilde=r.sum_wtilde,
                    n_particles=r.n_particles, n_bins=r.n_bins, device_error=r.device_error, kind=r.kind)

    def outputs(self):
        o = pcsir3_outputs()
        st = lib.pcsir3_get_outputs(self.handle, ctypes.byref(o))
        if st != OK:
            self._raise(st)
        N, B, S = o.n_particles, o.n_bins, o.bin_stride

        def view(ptr, shape, dtype):
            return _from_ptr(ptr, shape, dtype) if ptr else None

        out = dict(n_particles=N, n_bins=B, prop_state=view(o.prop_state, (7, N), torch.float32),
                   ancestor=view(o.ancestor, (N,), torch.int32), weight=view(o.weight, (N,), torch.float64),
                   qweight=view(o.qweight, (N,), torch.int64))
        if B > 0:
            out.update(bin_xyz=view(o.bin_xyz, (3, S), torch.int32)[:, :B],
                       bin_count=view(o.bin_count, (B,), torch.int32),
                       dummy=view(o.dummy, (7, S), torch.float64)[:, :B],
                       bin_loglik=view(o.bin_loglik, (B,), torch.float64),
                       particle_bin=view(o.particle_bin, (N,), torch.int32))
        if o.loglik:
            out["loglik"] = view(o.loglik, (N,), torch.float64)
        return out


class Batch3:
    """Owns one ``pcsir3_batch``: T targets in one 3D volume (state [7, sum N] float32)."""

    def __init__(self, n, h, psf_sigma_xy, psf_sigma_z, bg, patch_xy, patch_z, keep=0):
        T = len(n)
        arr = (pcsir3_target * T)()
        for t in range(T):
            hx, hy, hz = (float(v) for v in h[t])
            arr[t] = pcsir3_target(int(n[t]), hx, hy, hz, float(psf_sigma_xy[t]), float(psf_sigma_z[t]),
                                   float(bg[t]), int(patch_xy[t]), int(patch_z[t]))
        hdl = ctypes.c_void_p()
        st = lib.pcsir3_batch_create(arr, T, int(keep), ctypes.byref(hdl))
        if st != OK:
            raise PcsirError(st, "pcsir3_batch_create failed")
        self.handle = hdl
        self.T = T
        self.n_total = int(sum(int(x) for x in n))

    def close(self):
        if getattr(self, "handle", None):
            lib.pcsir3_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, state, volume, noise, u0, stream=None):
        """One step of every target (state [7, sum N] float32 in place; u0 float64 [T] on the device)."""
        _check_cuda(state, "state", torch.float32)
        _check_cuda(noise, "noise", torch.float32)
        _check_cuda(volume, "volume", torch.float32)
        _check_cuda(u0, "u0", torch.float64)
        D, H, W = volume.shape
        st = lib.pcsir3_batched_step(self.handle, _ptr(state), _ptr(volume), W, H, D, _ptr(noise), _ptr(u0),
                                     _stream_ptr(stream))
        if st != OK:
            raise PcsirError(st, lib.pcsir3_batch_last_error(self.handle).decode())

    def results(self):
        """Per-target results of the last step and the step's device error flags (synchronises)."""
        arr = (pcsir3_result * self.T)()
        err = ctypes.c_int32()
        st = lib.pcsir3_batch_results(self.handle, arr, self.T, ctypes.byref(err))
        if st != OK:
            raise PcsirError(st, "pcsir3_batch_results failed")
        return [dict(estimate=list(r.estimate), ess=r.ess, n_bins=r.n_bins, n_particles=r.n_particles,
                     max_loglik=r.max_loglik, device_error=r.device_error) for r in arr], err.value

    def outputs(self):
        o = pcsir3_batch_outputs()
        st = lib.pcsir3_batch_get_outputs(self.handle, ctypes.byref(o))
        if st != OK:
            raise PcsirError(st, "pcsir3_batch_get_outputs failed")
        N, B, S = o.n_total, o.n_bins, o.bin_stride

        def view(ptr, shape, dtype):
            return _from_ptr(ptr, shape, dtype) if ptr else None

        return dict(prop_state=view(o.prop_state, (7, N), torch.float32), n_bins=B,
                    bin_key=view(o.bin_key, (B,), torch.int64) if B else None,
                    bin_count=view(o.bin_count, (B,), torch.int32) if B else None,
                    dummy=view(o.dummy, (7, S), torch.float64)[:, :B] if B else None,
                    bin_loglik=view(o.bin_loglik, (B,), torch.float64) if B else None,
                    ancestor=view(o.ancestor, (N,), torch.int32), qweight=view(o.qweight, (N,), torch.int64))
