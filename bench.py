#!/usr/bin/env python
"""Throughput of one pcSIR filter step on GB300 (one JSON line on stdout).

Workload: single-target tracking in 512 x 512 Poisson images (Gaussian PSF
sigma 1.5 px, I0 100, background 10, nearly-constant-velocity motion with
process std 0.5 px), 21 x 21 likelihood patch, N = 2^24 FP32 particles,
cells of h = 0.5 px (pcSIR-2x2).  A step is one full pass of the hot path:
propagate, cells, dummies (centre of mass), dummy likelihood, weight copy,
normalisation, systematic resampling.  Inputs are synthetic and seeded; the
state and noise arrays (335 MB each) are larger than L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent filter (replicas; no data-path
collective); the value is all ranks' particle-steps over the slowest rank's
time.  ``--impl reference`` times the CPU oracle instead, on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s & steps/s: SIR vs pcSIR vs surrogate-pcSIR at matched RMSE, %roofline"
UNIT = "particles/s"
W_IMG = H_IMG = 512
PATCH = 21
SIGMA, I0, BG = 1.5, 100.0, 10.0
Q = (0.5, 0.5, 0.1, 0.1, 1.0)
N_DEFAULT = 1 << 24
H_DEFAULT = 0.5
NOISE_POOL = 3
SEED = 1310554100 + 200
# algorithmic bytes per particle of the propagate + cell + centre-of-mass kernel (FP32 state):
# read state 20 + noise 20, write propagated state 20 + cell slot 4
PROP_BIN_BYTES = 64
# tile sums + resample kernels: read cell slot 4 (twice), gather one propagated state 20 and write it 20
# per output
RESAMPLE_BYTES = 48
KERNELS_PER_STEP = 5
# deferred resampling: the propagate kernel reads the last step's ancestor 4 and gathers that state 20,
# reads noise 20, writes the propagated state 20 and the slot 4; tile sums + resample read the slot 4
# (twice) and write the ancestor 4
DEFERRED_PROP_BIN_BYTES = 68
DEFERRED_RESAMPLE_BYTES = 12
# noise drawn in the kernel: no noise array is read (plain: 64 - 20; deferred: 68 - 20)
DRAWN_PROP_BIN_BYTES = 44
DRAWN_DEFERRED_PROP_BIN_BYTES = 48
DRAWN_SEED = 0x5EED_1310_5541
# batched step (all targets, one launch): propagate/cells as above (64) + resampling (48); with
# deferred resampling 68 + 12, as for one target
BATCHED_BYTES = PROP_BIN_BYTES + RESAMPLE_BYTES
BATCHED_DEFERRED_BYTES = DEFERRED_PROP_BIN_BYTES + DEFERRED_RESAMPLE_BYTES


# SIR's likelihood (Eq. likelihood, Poisson): per pixel term the algorithmic work is
# lambda = I0 gx gy + bg (2), d = lambda - z (1), u = d / z (1), log(1 + u) (1, on the XU),
# z (u - log(1 + u)) (2) and the accumulation (1): 8 FP32 lane operations, one of them on the XU
SIR_OPS_PER_TERM = 8
FP32_LANES_PER_SM = 128  # FP32 lanes per SM (4 sub-partitions x 32)
XU_LANES_PER_SM = 16     # transcendental (XU) results per SM and clock


def sir_roofline(N, ms, num_sms, clocks):
    """FP32 roofline of a SIR step on the workload: its N P^2 pixel terms (all patches lie inside
    the image) at SIR_OPS_PER_TERM lane operations each, over the step's device time, against
    SMs x 128 lanes x the SM clock (the median sampled while SIR ran, else the maximum 2070 MHz);
    and its one logarithm per term against SMs x 16 XU results per clock."""
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    terms = N * PATCH * PATCH
    fp32_peak = num_sms * FP32_LANES_PER_SM * mhz * 1e6 / 1e12
    xu_peak = num_sms * XU_LANES_PER_SM * mhz * 1e6 / 1e12
    achieved = terms * SIR_OPS_PER_TERM / (ms * 1e-3) / 1e12
    xu = terms / (ms * 1e-3) / 1e12
    return {"kernel": "k_sir_prop_lik", "bound": "fp32", "achieved": achieved, "peak": fp32_peak,
            "unit": "Tops/s (FP32 lane operations)", "frac": achieved / fp32_peak,
            "peak_source": "derived: %d SMs x %d FP32 lanes x %.0f MHz" % (num_sms, FP32_LANES_PER_SM, mhz),
            "xu": {"achieved": xu, "peak": xu_peak, "unit": "T results/s", "frac": xu / xu_peak},
            "pixel_terms_per_step": terms, "ops_per_term": SIR_OPS_PER_TERM, "traffic": None}


def workload_name(N, h):
    return "single-target pcSIR, 512x512 Poisson images, 21x21 patch, N=%d FP32, h=%g px" % (N, h)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the propagate/bin kernel's source: its file, the device helpers, and the structures of
    pcsir_internal.h that its launches pass (declarations elsewhere in that header do not count)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1310_5541_gb300", "csrc")
    for f in ("pcsir_kernels.cu", "pcsir_device.cuh", "pcsir_philox.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "pcsir_internal.h"), "rb") as fh:
        txt = fh.read()
    h.update(txt[txt.index(b"struct Control {"):txt.index(b"struct ModelParams")])
    return h.hexdigest()[:16]


def profiled_traffic(N, label="dram bytes per particle"):
    """dram bytes per launch of the propagate/bin kernel from the committed ncu summary (``label``:
    the plain or the gathering variant's line), scaled to N particles; None if absent or taken on a
    different kernel source."""
    path = os.path.join(ROOT, "profiles", "k_prop_bin_512x512_h0.5.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel source hash:\s*([0-9a-f]+)", txt)
    m_bpp = re.search(r"^" + re.escape(label) + r":\s*([0-9.]+)", txt, re.M)
    if not (m_hash and m_bpp) or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_bpp.group(1)) * N


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", uuid, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_cpu_affinity(gpu_index):
    """CPUs local to the GPU, from `nvidia-smi topo -m` ("CPU Affinity" column), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True, timeout=30).stdout
    except Exception:
        return None
    lines = [l for l in out.splitlines() if l.strip()]
    head = next((l for l in lines if "CPU Affinity" in l), None)
    row = next((l for l in lines if l.split("\t")[0].strip() == "GPU%d" % gpu_index), None)
    if head is None or row is None:
        return None
    cols = [c.strip() for c in head.split("\t")]
    vals = [c.strip() for c in row.split("\t")]
    try:
        field = vals[cols.index("CPU Affinity")]
        cpus = set()
        for part in field.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return cpus & set(range(os.cpu_count() or 1)) or None
    except (ValueError, IndexError):
        return None


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_rate(n_sample, budget_s, seed, h, steps=None, warmup=0):
    """Time the oracle's pcSIR step on a bounded sample of the workload (host cores)."""
    import numpy as np

    from oracle import pcsir_oracle as O
    from paper_1310_5541_gb300 import synth

    model = synth.Model(sigma_psf=SIGMA, I0=I0, bg=BG, patch=PATCH, q=Q)
    nfr = (steps or 64) + warmup + 1
    seq = synth.make_sequence(W_IMG, H_IMG, min(nfr, 64), model, seed)
    st = synth.initial_state(seq.gt[0], n_sample, np.float32)
    times = []
    k = 0
    t_start = time.perf_counter()
    while True:
        nz = synth.make_noise(n_sample, Q, seed, k, np.float32)
        u0 = synth.make_u0(seed, k)
        img = seq.images[k % seq.images.shape[0]]
        t0 = time.perf_counter()
        st = O.pcsir_step(st, img, nz, u0, h, model)["new_state"]
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
        k += 1
        if steps is not None:
            if len(times) >= steps:
                break
        elif time.perf_counter() - t_start > budget_s and len(times) >= 2:
            break
    return n_sample * len(times) / sum(times), len(times), sum(times)


def _oracle_worker(args):
    n_sample, budget_s, seed, h = args
    return cpu_oracle_rate(n_sample, budget_s, seed, h)


def cpu_oracle_rate_all_cores(n_sample, budget_s, seed, h, procs):
    """The oracle on every host core at once: ``procs`` spawned processes (one thread each), each
    timing oracle pcSIR steps on its own sample of the workload for about ``budget_s`` seconds.
    Returns (particle-steps per second over all processes, total steps, seconds of the busiest)."""
    import multiprocessing as mp

    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(n_sample, budget_s, seed + j, h) for j in range(procs)])
    total = sum(n_sample * steps for _, steps, _ in res)
    busiest = max(tot for _, _, tot in res)
    return total / busiest, sum(steps for _, steps, _ in res), busiest


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of the ranks' values (the slowest rank's time); on one rank the value itself."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(n_particles, steps, world, slowest_ms):
    """Whole-job particle-steps per second of `world` independent replicas of n_particles each
    (weak scaling): every rank's particles over the slowest rank's time."""
    return n_particles * steps * world / (slowest_ms / 1e3)


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    n_s = 1 << 18
    rate, steps, tot = cpu_oracle_rate(n_s, 0, SEED, args.h, steps=args.steps, warmup=args.warmup)
    sample = "oracle pcSIR steps on N=2^18 particles of the same workload (h=%g), %d timed steps" % (args.h, steps)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args.n, args.h), "sample_particles": n_s},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(n_targets, steps, warmup, seed, world=1):
    """Multi-target workload: n_targets spots in 1024 x 1024 frames, log-uniform particle counts in
    [10^3, 10^5] (about 2.1e7 in total for 1000 targets), PSF std U[1.2, 2.0], SNR U[2, 8], patch
    2 ceil(3 sigma) + 1, cell edges from the autotuner cache (else sigma / 3); one persistent launch
    per step, replayed from CUDA graphs."""
    import numpy as np
    import torch

    from paper_1310_5541_gb300 import autotune, pcsir, synth

    frames = warmup + steps
    table = autotune.load()
    if "c" not in table:
        table = autotune.tune()
    batch = synth.make_batch(n_targets, 1024, 1024, frames, seed)
    batch.h[:] = autotune.cell_edges(batch.sigma, table)
    T = len(batch.n)
    ntot = int(batch.n.sum())
    dev = torch.device("cuda", torch.cuda.current_device())
    images = torch.from_numpy(batch.images).to(dev)
    noise = [torch.from_numpy(synth.batch_noise(batch, Q, seed, j)).to(dev) for j in range(NOISE_POOL)]
    u0 = torch.from_numpy(np.stack([synth.batch_u0(T, seed, k) for k in range(frames)])).to(dev)
    state = torch.from_numpy(synth.batch_initial_state(batch, np.float32)).to(dev)
    bt = pcsir.Batch(batch.n, batch.h, batch.sigma, batch.bg, batch.patch)
    bt.set_table(int(table.get("table_bits", 10)))
    bt.set_grid(int(table.get("blocks_per_sm", 2)))
    s = torch.cuda.Stream()
    graphs = []
    with torch.cuda.stream(s):
        bt.step(state, images[0], noise[0], u0[0], stream=s)  # load and warm outside capture
    torch.cuda.synchronize()
    state.copy_(torch.from_numpy(synth.batch_initial_state(batch, np.float32)).to(dev))
    for k in range(frames):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bt.step(state, images[k], noise[k % NOISE_POOL], u0[k], stream=s)
        graphs.append(g)
    torch.cuda.synchronize()
    for k in range(warmup):
        graphs[k].replay()
    torch.cuda.synchronize()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        a.record(s)
        for k in range(warmup, frames):
            graphs[k].replay()
        b_.record(s)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b_) / steps
    phases = bt.phase_times()
    res, derr = bt.results()
    est = np.array([r["estimate"][:2] for r in res])
    rmse = float(np.sqrt(np.mean(np.sum((est - batch.gt[frames, :, :2]) ** 2, axis=1))))
    # the same steps with deferred resampling: each step records ancestors and the next step's
    # propagation gathers through them; one graph per step, replayed once each in capture order
    # (the two state buffers alternate at capture), and the resampled states written out once at
    # the end of the timed region
    state.copy_(torch.from_numpy(synth.batch_initial_state(batch, np.float32)).to(dev))
    with torch.cuda.stream(s):
        bt.deferred_begin(state, stream=s)
    torch.cuda.synchronize()
    dgraphs = []
    for k in range(frames):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bt.deferred_step(images[k], noise[k % NOISE_POOL], u0[k], stream=s)
        dgraphs.append(g)
    torch.cuda.synchronize()
    for k in range(warmup):
        dgraphs[k].replay()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        a.record(s)
        for k in range(warmup, frames):
            dgraphs[k].replay()
        bt.deferred_state(state, stream=s)
        b_.record(s)
    torch.cuda.synchronize()
    dms = a.elapsed_time(b_) / steps
    dphases = bt.phase_times()
    dres, dderr = bt.results()
    dest = np.array([r["estimate"][:2] for r in dres])
    drmse = float(np.sqrt(np.mean(np.sum((dest - batch.gt[frames, :, :2]) ** 2, axis=1))))
    bt.close()
    hbm, kind = peaks()
    dgbs = BATCHED_DEFERRED_BYTES * ntot / (dms * 1e-3) / 1e9
    deferred = {"value": ntot * world / (dms / 1e3), "unit": UNIT, "ms_per_step": dms, "rmse_px": drmse,
                "device_error": dderr, "step_bytes_per_particle": BATCHED_DEFERRED_BYTES, "step_gbs": dgbs,
                "step_frac_of_hbm": dgbs / hbm,
                "phase_ms_last_step": dict(zip(("setup", "prop_bin", "bins_lik", "weights", "tile_sums",
                                                "target_scan", "resample"), dphases))}
    return {"workload": "batched pcSIR, %d targets, 1024x1024, %d particles FP32" % (T, ntot),
            "value": ntot * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "targets": T, "particles": ntot, "cells_last_step": int(sum(r["n_bins"] for r in res)),
            "launches_per_step": 1, "graph": True, "rmse_px": rmse,
            "device_error": derr, "step_bytes_per_particle": BATCHED_BYTES,
            "step_gbs": BATCHED_BYTES * ntot / (ms * 1e-3) / 1e9,
            "step_frac_of_hbm": BATCHED_BYTES * ntot / (ms * 1e-3) / 1e9 / hbm, "peak_source": kind,
            "autotune": {k: table.get(k) for k in ("c", "blocks_per_sm", "table_bits", "rmse", "rmse_limit",
                                                   "first_c_over_limit", "step_ms")},
            "phase_ms_last_step": dict(zip(("setup", "prop_bin", "bins_lik", "weights", "tile_sums", "target_scan",
                                            "resample"), phases)),
            "deferred": deferred}


def run_matched(N, rows_target, train_steps, n_seq, n_frames, seed, sir_steps_cap=None):
    """SIR vs pcSIR vs surrogate-pcSIR on the single-target workload at matched tracking RMSE.

    The surrogate is trained first on pairs its own method generates: exact pcSIR
    steps (N = 2^20, cells h in {0.02, 0.05, 0.1, 0.2, 0.5} px) over further
    512 x 512 sequences of the same model, until ``rows_target`` (dummy inputs,
    exact log-likelihood) rows are stored.  Then every method filters the same
    ``n_seq`` sequences of ``n_frames`` frames with N particles and identical
    noise and resampling uniforms; per method the tracking RMSE against the
    ground truth and the device time per step (CUDA events around each step)
    are reported.  At matched RMSE (within 5% of SIR's) the fastest cell size of
    each pcSIR variant is picked.
    """
    import numpy as np
    import torch

    from paper_1310_5541_gb300 import pcsir, surrogate, synth

    dev = torch.device("cuda", torch.cuda.current_device())
    model = synth.Model(sigma_psf=SIGMA, I0=I0, bg=BG, patch=PATCH, q=Q)
    out = {}
    # training pairs from exact pcSIR runs
    t0 = time.perf_counter()
    Nc = 1 << 20
    hs_c = (0.02, 0.05, 0.1, 0.2, 0.5)
    pool_c = [torch.from_numpy(synth.make_noise(Nc, Q, seed + 9, j, np.float32)).to(dev) for j in range(4)]
    sur = pcsir.Surrogate(capacity=rows_target + (1 << 20), batch=4096, i0_ref=128.0, sigma_ref=SIGMA,
                          max_pixels=W_IMG * H_IMG)
    ctx_c = pcsir.Context(Nc, torch.float32, patch=PATCH, psf_sigma=SIGMA, bg=BG)
    i = 0
    while sur.rows() < rows_target and i < 100000:
        sq = synth.make_sequence(W_IMG, H_IMG, 10, model, seed + 500 + i)
        st = torch.from_numpy(synth.initial_state(sq.gt[0], Nc, np.float32)).to(dev)
        frames = ((torch.from_numpy(sq.images[k]).to(dev), pool_c[(i + k) % 4], synth.make_u0(seed + 500 + i, k))
                  for k in range(sq.images.shape[0]))
        surrogate.collect(ctx_c, sur, st, frames, hs_c[i % len(hs_c)], BG, SIGMA)
        i += 1
    ctx_c.close()
    rows = sur.rows()
    t1 = time.perf_counter()
    sur.init(seed)
    fit = surrogate.fit(sur, steps=train_steps, lr=2e-3, seed=3, val_frac=0.02, chunk=2000)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out["surrogate_training"] = {
        "rows": rows, "sequences": i, "train_steps": train_steps, "batch": 4096, "collect_s": t1 - t0,
        "train_s": t2 - t1, "val_rmse_nats": fit["val_rmse"], "val_max_nats": fit["val_max"],
        "val_label_std_nats": fit["val_label_std"], "val_censored_above": fit["val_censored_above"],
        "final_loss": float(fit["loss"][-500:].mean())}

    # the comparison sequences
    seqs = [synth.make_sequence(W_IMG, H_IMG, n_frames, model, seed + 90000 + r) for r in range(n_seq)]
    imgs = [torch.from_numpy(sq.images).to(dev) for sq in seqs]
    pool = [torch.from_numpy(synth.make_noise(N, Q, seed + 7, j, np.float32)).to(dev) for j in range(NOISE_POOL)]
    ctx = pcsir.Context(N, torch.float32, patch=PATCH, psf_sigma=SIGMA, bg=BG)
    ctx_s = pcsir.Context(N, torch.float32, patch=PATCH, psf_sigma=SIGMA, bg=BG)
    pcsir.attach_surrogate(ctx_s, sur, holdout_frac=0.02, min_holdout=32, window=20.0, max_err=3.0)
    stream = torch.cuda.current_stream()

    def run(kind, h, frames_cap=None):
        errs, ms, exact, dummies, fallbacks = [], [], 0, 0, 0
        c = ctx_s if kind == "surrogate" else ctx
        c.timing_enable(n_seq * n_frames)
        for r, sq in enumerate(seqs):
            st = torch.from_numpy(synth.initial_state(sq.gt[0], N, np.float32)).to(dev)
            K = n_frames if frames_cap is None else min(n_frames, frames_cap)
            for k in range(K):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                u0 = synth.make_u0(seed + 90000 + r, k)
                a.record(stream)
                if kind == "sir":
                    pcsir.sir_step(c, st, imgs[r][k], pool[k % NOISE_POOL], u0, stream)
                else:
                    pcsir.pcsir_step(c, st, imgs[r][k], h, pool[k % NOISE_POOL], u0, stream)
                b.record(stream)
                torch.cuda.synchronize()
                res = c.last_result()
                if res["device_error"]:
                    raise RuntimeError("device error %d in %s h=%s" % (res["device_error"], kind, h))
                if k >= 2:  # the first steps include one-time work
                    ms.append(a.elapsed_time(b))
                errs.append(np.array(res["estimate"][:2]) - sq.gt[k + 1, :2])
                if kind == "surrogate":
                    chk = pcsir.surrogate_last_check(c)
                    exact += chk["n_exact"]
                    dummies += chk["n_dummies"]
                    fallbacks += chk["fallback"]
        stages = np.array(c.timing_read(n_seq * n_frames))[2:].mean(axis=0)
        c.timing_enable(0)
        e = np.array(errs)
        d = {"method": kind, "h": h, "rmse_px": float(np.sqrt(np.mean(np.sum(e ** 2, axis=1)))),
             "ms_per_step": float(np.mean(ms)), "steps_per_s": 1e3 / float(np.mean(ms)),
             "particles_per_s": N * 1e3 / float(np.mean(ms)), "frames": len(errs),
             "stages_ms": [float(x) for x in stages]}
        if kind == "surrogate":
            d.update(exact_fraction=exact / max(1, dummies), fallbacks=fallbacks, mean_dummies=dummies / len(errs))
        return d

    results = [run("sir", None, sir_steps_cap)]
    for h in (0.5, 0.2, 0.1, 0.05, 0.02):
        results.append(run("pcsir", h))
    for h in (0.2, 0.1, 0.05, 0.02):
        results.append(run("surrogate", h))
    ctx.close()
    ctx_s.close()
    sur.close()
    target = 1.05 * results[0]["rmse_px"]

    def best(kind):
        ok = [r for r in results if r["method"] == kind and r["rmse_px"] <= target]
        return max(ok, key=lambda r: r["steps_per_s"]) if ok else None

    out.update(N=N, sequences=n_seq, frames=n_frames, target_rmse_px=target, runs=results,
               matched={"sir": results[0], "pcsir": best("pcsir"), "surrogate_pcsir": best("surrogate")})
    return out


def matched_summary(m):
    """The metric's comparison in compact form: per method the cell size, tracking RMSE and
    throughput of every run, and the fastest run of each method within 5% of SIR's RMSE."""
    if not m:
        return None

    def row(r):
        return None if r is None else [r["method"], r["h"], round(r["rmse_px"], 5), round(r["steps_per_s"], 2),
                                       float("%.4g" % r["particles_per_s"])]

    return {"N": m["N"], "target_rmse_px": round(m["target_rmse_px"], 5),
            "columns": ["method", "h_px", "rmse_px", "steps_per_s", "particles_per_s"],
            "at_matched_rmse": {k: row(v) for k, v in m["matched"].items()},
            "runs": [row(r) for r in m["runs"]]}


def run_ess(N, n_frames, frac, seed):
    """ESS-thresholded pcSIR (Algorithm 2 with Algorithm 1's test: resample only when
    N_eff < frac N, weights carried otherwise) against pcSIR resampling every step, on the
    single-target workload (512 x 512, Poisson, 21 x 21 patch, h = 0.5 px) with the same
    sequence, noise and uniforms; per method the device time per step (CUDA events), the
    tracking RMSE and the fraction of steps that resampled."""
    import numpy as np
    import torch

    from paper_1310_5541_gb300 import pcsir, synth

    dev = torch.device("cuda", torch.cuda.current_device())
    model = synth.Model(sigma_psf=SIGMA, I0=I0, bg=BG, patch=PATCH, q=Q)
    seq = synth.make_sequence(W_IMG, H_IMG, n_frames, model, seed)
    imgs = torch.from_numpy(seq.images).to(dev)
    pool = [torch.from_numpy(synth.make_noise(N, Q, seed + 3, j, np.float32)).to(dev) for j in range(NOISE_POOL)]
    ctx = pcsir.Context(N, torch.float32, patch=PATCH, psf_sigma=SIGMA, bg=BG, keep=0)
    stream = torch.cuda.current_stream()
    rows = []
    for name in ("pcsir", "pcsir-ess"):
        st = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).to(dev)
        lw = torch.zeros(N, dtype=torch.int64, device=dev)
        ms, ms_res, ms_keep, errs, ess = [], [], [], [], []
        for k in range(n_frames):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            u0 = synth.make_u0(seed + 5, k)
            a.record(stream)
            if name == "pcsir":
                pcsir.pcsir_step(ctx, st, imgs[k], H_DEFAULT, pool[k % NOISE_POOL], u0, stream)
            else:
                pcsir.pcsir_step_ess(ctx, st, lw, imgs[k], H_DEFAULT, pool[k % NOISE_POOL], u0, frac * N, stream)
            b.record(stream)
            torch.cuda.synchronize()
            r = ctx.last_result()
            if k >= 2:
                t = a.elapsed_time(b)
                ms.append(t)
                (ms_res if r["resampled"] else ms_keep).append(t)
            errs.append(np.array(r["estimate"][:2]) - seq.gt[k + 1, :2])
            ess.append(r["ess"] / N)
        e = np.array(errs)
        rows.append({"method": name, "ms_per_step": float(np.mean(ms)), "value": N / (np.mean(ms) / 1e3),
                     "unit": UNIT, "rmse_px": float(np.sqrt(np.mean(np.sum(e ** 2, axis=1)))),
                     "resampled_fraction": len(ms_res) / max(1, len(ms)),
                     "ms_resampled_steps": float(np.mean(ms_res)) if ms_res else None,
                     "ms_carried_steps": float(np.mean(ms_keep)) if ms_keep else None,
                     "mean_ess_fraction": float(np.mean(ess))})
    ctx.close()
    return {"workload": "ESS-thresholded pcSIR (N_thr = %.2f N) vs every-step pcSIR, N=%d, 512x512, 21x21, h=%.2f"
                        % (frac, N, H_DEFAULT), "frames": n_frames, "rows": rows}


def run_large_object(counts, n_frames, seed):
    """The paper's large-object regime (Section 5.3): 512 x 512 frames, PSF sigma 13 px, SNR 2, speed
    U[2, 7] px/frame, Gaussian (SSE) likelihood over a 65 x 65 kernel.  SIR, pcSIR-1x1 (h = 1) and
    pcSIR-2x2 (h = 0.5) filter the same sequence with the same noise; per method and particle count
    the device time per step (CUDA events around each step) and the tracking RMSE."""
    import numpy as np
    import torch

    from paper_1310_5541_gb300 import pcsir, synth

    dev = torch.device("cuda", torch.cuda.current_device())
    m = synth.large_object_model()
    seq = synth.large_object_sequence(n_frames, seed)
    imgs = torch.from_numpy(seq.images).to(dev)
    stream = torch.cuda.current_stream()
    rows = []
    for N in counts:
        pool = [torch.from_numpy(synth.make_noise(N, m.q, seed + 3, j, np.float32)).to(dev) for j in range(NOISE_POOL)]
        ctx = pcsir.Context(N, torch.float32, lik="sse", patch=m.patch, psf_sigma=m.sigma_psf, bg=m.bg,
                            sigma_xi=m.sigma_xi)
        for name, h in (("sir", None), ("pcsir-1x1", 1.0), ("pcsir-2x2", 0.5)):
            st = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).to(dev)
            ms, errs = [], []
            for k in range(n_frames):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                u0 = synth.make_u0(seed + 5, k)
                a.record(stream)
                if h is None:
                    pcsir.sir_step(ctx, st, imgs[k], pool[k % NOISE_POOL], u0, stream)
                else:
                    pcsir.pcsir_step(ctx, st, imgs[k], h, pool[k % NOISE_POOL], u0, stream)
                b.record(stream)
                torch.cuda.synchronize()
                if k >= 2:
                    ms.append(a.elapsed_time(b))
                r = ctx.last_result()
                errs.append(np.array(r["estimate"][:2]) - seq.gt[k + 1, :2])
            e = np.array(errs)
            rows.append({"method": name, "N": N, "ms_per_step": float(np.mean(ms)),
                         "rmse_px": float(np.sqrt(np.mean(np.sum(e ** 2, axis=1))))})
        ctx.close()
    for r in rows:
        sir = next(x for x in rows if x["N"] == r["N"] and x["method"] == "sir")
        r["speedup_vs_sir"] = sir["ms_per_step"] / r["ms_per_step"]
        r["rmse_vs_sir"] = r["rmse_px"] / sir["rmse_px"] - 1.0
    return {"workload": "large object: 512x512, PSF sigma 13 px, SNR 2, SSE likelihood sigma_xi 30, 65x65 kernel",
            "frames": n_frames, "rows": rows}


def run_3d(counts, n_frames, seed, sur_seqs=0, sur_steps=0):
    """3D tracking: 256 x 256 x 64 Poisson volumes (PSF sigma 1.5 / 3 voxels, I0 100, bg 10), state
    (x, y, z, vx, vy, vz, I0), 11 x 11 x 7 likelihood patch; SIR and pcSIR with 0.5 x 0.5 x 1 and
    0.1 x 0.1 x 0.2 voxel cells filter the same sequence with the same noise: device time per step and
    tracking RMSE."""
    import numpy as np
    import torch

    from paper_1310_5541_gb300 import pcsir, synth

    dev = torch.device("cuda", torch.cuda.current_device())
    seq = synth.make_sequence3(256, 256, 64, n_frames, seed)
    vols = torch.from_numpy(seq.images).to(dev)
    stream = torch.cuda.current_stream()
    rows = []
    sur, training = None, None
    if sur_steps > 0:
        sur, training = train_surrogate3(sur_seqs, sur_steps, seed + 11)
    for N in counts:
        pool = [torch.from_numpy(synth.make_noise(N, synth.Q3, seed + 3, j, np.float32)).to(dev)
                for j in range(NOISE_POOL)]
        ctx = pcsir.Context3(N)
        methods = [("sir", None), ("pcsir", (0.5, 0.5, 1.0)), ("pcsir-fine", (0.1, 0.1, 0.2))]
        if sur is not None:
            # checked: the held-out test falls back to the exact likelihood; unchecked: never (the
            # surrogate path's own cost, whatever the network's error)
            methods += [("surrogate-fine", (0.1, 0.1, 0.2)), ("surrogate-fine-unchecked", (0.1, 0.1, 0.2))]
        for name, h in methods:
            use_sur = name.startswith("surrogate")
            pcsir.attach_surrogate3(ctx, sur if use_sur else None, holdout_frac=0.02, min_holdout=32, window=20.0,
                                    max_err=1e300 if name.endswith("unchecked") else 3.0)
            exact, dummies, fallbacks = 0, 0, 0
            st = torch.from_numpy(synth.initial_state3(seq.gt[0], N, np.float32)).to(dev)
            ms, errs = [], []
            for k in range(n_frames):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                u0 = synth.make_u0(seed + 5, k)
                a.record(stream)
                if h is None:
                    ctx.sir_step(st, vols[k], pool[k % NOISE_POOL], u0, stream)
                else:
                    ctx.step(st, vols[k], h, pool[k % NOISE_POOL], u0, stream)
                b.record(stream)
                torch.cuda.synchronize()
                if k >= 2:
                    ms.append(a.elapsed_time(b))
                r = ctx.last_result()
                if r["device_error"]:
                    raise RuntimeError("device error %d in 3D %s" % (r["device_error"], name))
                errs.append(np.array(r["estimate"][:3]) - seq.gt[k + 1, :3])
                if use_sur:
                    c = pcsir.surrogate_last_check3(ctx)
                    exact += c["n_exact"]
                    dummies += c["n_dummies"]
                    fallbacks += c["fallback"]
            e = np.array(errs)
            row = {"method": name, "N": N, "ms_per_step": float(np.mean(ms)),
                   "particles_per_s": N * 1e3 / float(np.mean(ms)),
                   "rmse_voxel": float(np.sqrt(np.mean(np.sum(e ** 2, axis=1))))}
            if use_sur:
                row.update(exact_fraction=exact / max(1, dummies), fallbacks=fallbacks,
                           mean_dummies=dummies / max(1, len(errs)))
            rows.append(row)
        ctx.close()
    if sur is not None:
        sur.close()
    return {"workload": "3D: 256x256x64 volumes, 11x11x7 patch, cells 0.5x0.5x1 and 0.1x0.1x0.2 voxel",
            "frames": n_frames, "surrogate_training": training,
            "rows": rows}


def train_surrogate3(n_seq, steps, seed):
    """The 3D surrogate trained on pairs its own method generates: exact 3D pcSIR steps (N = 2^16) over
    ``n_seq`` four-frame 64 x 64 x 32 sequences of the same model, at the model's process noise with
    0.1 x 0.1 x 0.2 voxel cells and at scaled-down noise with finer cells (``surrogate.COLLECT3``); then
    ``steps`` Adam updates."""
    import torch

    from paper_1310_5541_gb300 import pcsir, surrogate

    t0 = time.perf_counter()
    sur = pcsir.Surrogate(capacity=max(1 << 20, 1600 * n_seq), batch=4096, i0_ref=128.0, sigma_ref=1.5,
                          max_pixels=256 * 256 * 64, geometry=3)
    surrogate.collect3_sequences(sur, n_seq, 4, 1 << 16, seed + 500)
    t1 = time.perf_counter()
    sur.init(seed)
    fit = surrogate.fit(sur, steps=steps, lr=2e-3, seed=3, val_frac=0.02, chunk=2000)
    torch.cuda.synchronize()
    return sur, {"rows": sur.rows(), "sequences": n_seq, "train_steps": steps, "collect_s": t1 - t0,
                 "train_s": time.perf_counter() - t1, "val_rmse_nats": fit["val_rmse"],
                 "val_max_nats": fit["val_max"], "val_label_std_nats": fit["val_label_std"]}


def run_batched3(n_targets, n_per, steps, warmup, seed, world=1):
    """3D multi-target workload: n_targets spots in 256 x 256 x 64 Poisson volumes (PSF sigma 1.5 / 3
    voxels, I0 100, bg 10), n_per particles each, 11 x 11 x 7 patches, 0.5 x 0.5 x 1 voxel cells; one
    step is the fixed kernel sequence of pcsir3_batched_step over all targets, replayed from CUDA
    graphs.  Algorithmic bytes per particle and step: propagate/cell 88 (state and noise 28 + 28 read,
    propagated state 28 + slot 4 written), tile sums 8 (slot, integer weight), resampling 60 (slot 4,
    gathered state 28, written state 28)."""
    import numpy as np
    import torch

    from paper_1310_5541_gb300 import pcsir, synth

    frames = warmup + steps
    batch = synth.make_batch3(n_targets, 256, 256, 64, frames, seed, n_particles=n_per)
    T = len(batch.n)
    ntot = int(batch.n.sum())
    dev = torch.device("cuda", torch.cuda.current_device())
    vols = torch.from_numpy(batch.images).to(dev)
    noise = [torch.from_numpy(synth.make_noise(ntot, synth.Q3, seed, j, np.float32)).to(dev) for j in range(2)]
    u0 = torch.from_numpy(np.stack([synth.batch_u0(T, seed, k) for k in range(frames)])).to(dev)
    st0 = torch.from_numpy(synth.batch3_initial_state(batch)).to(dev)
    state = st0.clone()
    bt = pcsir.Batch3(batch.n, batch.h, batch.sigma_xy, batch.sigma_z, batch.bg, batch.patch_xy, batch.patch_z)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bt.step(state, vols[0], noise[0], u0[0], stream=s)  # load the kernels outside capture
    torch.cuda.synchronize()
    state.copy_(st0)
    graphs = []
    for k in range(frames):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bt.step(state, vols[k], noise[k % 2], u0[k], stream=s)
        graphs.append(g)
    torch.cuda.synchronize()
    for k in range(warmup):
        graphs[k].replay()
    torch.cuda.synchronize()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        a.record(s)
        for k in range(warmup, frames):
            graphs[k].replay()
        b_.record(s)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b_) / steps
    res, derr = bt.results()
    est = np.array([r["estimate"][:3] for r in res])
    rmse = float(np.sqrt(np.mean(np.sum((est - batch.gt[frames, :, :3]) ** 2, axis=1))))
    bt.close()
    hbm, kind = peaks()
    bpp = 88 + 8 + 60
    gbs = bpp * ntot / (ms * 1e-3) / 1e9
    return {"workload": "batched 3D pcSIR, %d targets x %d particles, 256x256x64, 11x11x7, cells 0.5x0.5x1"
                        % (T, n_per), "value": ntot * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "steps": steps, "particles": ntot, "cells_last_step": int(sum(r["n_bins"] for r in res)),
            "kernels_per_step": 8, "graph": True, "rmse_voxel": rmse, "device_error": derr,
            "step_bytes_per_particle": bpp, "step_gbs": gbs, "step_frac_of_hbm": gbs / hbm, "peak_source": kind}


def run_gemm(shapes, reps=10):
    """The surrogate training's tcgen05 GEMM (pcsir_gemm_bf16: TMA tiles, FP32 accumulation in
    tensor memory) on K-contiguous bf16 operands: CUDA-event time per product and TFLOP/s against the
    measured bf16 peak."""
    import torch

    from paper_1310_5541_gb300 import pcsir

    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak = json.load(fh).get("bf16_tflops")
    except (OSError, ValueError):
        pass
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    rows = []
    for (M, N, K) in shapes:
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        C = torch.empty(M, N, device="cuda")
        for _ in range(3):
            pcsir.gemm_bf16(A, B, C)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            pcsir.gemm_bf16(A, B, C)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        rows.append({"M": M, "N": N, "K": K, "ms": ms, "tflops": tf,
                     "frac_of_measured_bf16": (tf / peak) if peak else None})
    return {"kernel": "k_gemm_bf16_tma", "peak_tflops": peak, "rows": rows}


def run_drawn(ctx, pcsir, state0, images, img_host, u0s, N, h, K, Wm, stream, seq, pg, dev, hbm, peak_kind,
              deferred):
    """The headline's steps with the process noise drawn in the kernel (pcsir_step_philox, or a
    deferred run of pcsir_deferred_step_philox): device-resident timing of K steps, and an end-to-end
    run through the same C ABI in which every step copies its image from page-locked host memory and
    reads its result back (the noise no longer crosses the host link).  The deferred run writes its
    resampled states out once at the end of each timed region."""
    import numpy as np
    import torch

    q = Q
    state = state0.clone()
    out = torch.empty_like(state0)
    res1 = pcsir.pcsir_result()

    def step(k, img):
        if deferred:
            r = pcsir.lib.pcsir_deferred_step_philox(ctx.handle, pcsir._ptr(img), W_IMG, H_IMG, float(h),
                                                     pcsir._q5(q), DRAWN_SEED, k, float(u0s[k]),
                                                     pcsir._stream_ptr(stream), None)
        else:
            r = pcsir.lib.pcsir_step_philox(ctx.handle, pcsir._ptr(state), N, pcsir._ptr(img), W_IMG, H_IMG,
                                            float(h), pcsir._q5(q), DRAWN_SEED, k, float(u0s[k]),
                                            pcsir._stream_ptr(stream), None)
        if r != 0:
            ctx._raise(r)

    def begin():
        state.copy_(state0)
        if deferred:
            pcsir.pcsir_deferred_begin(ctx, state0, stream=stream)

    begin()
    for k in range(Wm):
        step(k, images[k])
    torch.cuda.synchronize()
    ctx.timing_enable(K)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(Wm, Wm + K):
        step(k, images[k])
    if deferred:
        pcsir.pcsir_deferred_state(ctx, out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed = e0.elapsed_time(e1)
    r = ctx.last_result()
    stages = np.array(ctx.timing_read(K)).mean(axis=0)
    if pg:
        elapsed = max_over_ranks(elapsed, pg, dev)
    bytes_pb = DRAWN_DEFERRED_PROP_BIN_BYTES if deferred else DRAWN_PROP_BIN_BYTES
    achieved = bytes_pb * N / (stages[0] * 1e-3) / 1e9

    # end to end: image in, result out, every step (one stream; the image is 1 MB)
    img_dev = torch.empty((H_IMG, W_IMG), dtype=torch.float32, device=dev)
    K_e2e = max(3, K // 2)
    begin()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K_e2e):
        img_dev.copy_(img_host[k], non_blocking=True)
        step(k, img_dev)
        stream.synchronize()
        pcsir.lib.pcsir_last_result(ctx.handle, pcsir.ctypes.byref(res1))
    if deferred:
        pcsir.pcsir_deferred_state(ctx, out, stream=stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    return {"value": N * K * 1e3 / elapsed, "unit": "particles/s", "ms_per_step": elapsed / K, "steps": K,
            "api": ("pcsir_deferred_begin / pcsir_deferred_step_philox x K / pcsir_deferred_state (timed)"
                    if deferred else "pcsir_step_philox"),
            "noise": "Philox4x32-10 + Box-Muller in the propagation kernel, seed %#x, counter (i, frame)" % DRAWN_SEED,
            "stages_ms": {"prop_bin": float(stages[0]), "dummies_lik": float(stages[1]), "weights": float(stages[2]),
                          "scan_resample": float(stages[3])},
            "roofline": {"kernel": "k_prop_bin (drawn noise%s)" % (", gathering" if deferred else ""), "bound": "hbm",
                         "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "peak_source": peak_kind, "algorithmic_bytes": bytes_pb * N},
            "e2e": {"value": N * K_e2e / e2e_s, "unit": "particles/s", "h2d_bytes_per_step": 4 * H_IMG * W_IMG,
                    "d2h_bytes_per_step": pcsir.ctypes.sizeof(pcsir.pcsir_result), "steps": K_e2e, "copies": "serial"},
            "device_error": int(r["device_error"])}


def run_deferred(ctx, pcsir, state0, images, noise, u0s, N, h, K, Wm, stream, seq, pg, dev, hbm, peak_kind):
    """The same steps as a deferred-resampling run (pcsir_deferred_*): each resampling recorded as
    ancestors, gathered by the next step's propagation.  Timed: K steps and, once at the end, the
    resampled states written out to a caller buffer (pcsir_deferred_state)."""
    import numpy as np
    import torch

    out = torch.empty_like(state0)
    pcsir.pcsir_deferred_begin(ctx, state0, stream=stream)
    for k in range(Wm):
        pcsir.pcsir_deferred_step(ctx, images[k], h, noise[k % NOISE_POOL], u0s[k], stream=stream)
    torch.cuda.synchronize()
    ctx.timing_enable(K)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(Wm, Wm + K):
        pcsir.pcsir_deferred_step(ctx, images[k], h, noise[k % NOISE_POOL], u0s[k], stream=stream)
    pcsir.pcsir_deferred_state(ctx, out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed = e0.elapsed_time(e1)
    r = ctx.last_result()
    stages = np.array(ctx.timing_read(K)).mean(axis=0)
    if pg:
        elapsed = max_over_ranks(elapsed, pg, dev)
    achieved = DEFERRED_PROP_BIN_BYTES * N / (stages[0] * 1e-3) / 1e9
    return {"value": N * K * 1e3 / elapsed, "unit": "particles/s", "ms_per_step": elapsed / K,
            "steps": K, "api": "pcsir_deferred_begin / pcsir_deferred_step x K / pcsir_deferred_state (timed)",
            "stages_ms": {"prop_bin": float(stages[0]), "dummies_lik": float(stages[1]), "weights": float(stages[2]),
                          "scan_resample": float(stages[3])},
            "roofline": {"kernel": "k_prop_bin (gathering)", "bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": profiled_traffic(N, "gathering dram bytes per particle"), "peak_source": peak_kind,
                         "algorithmic_bytes": DEFERRED_PROP_BIN_BYTES * N},
            "scan_resample_gbs": DEFERRED_RESAMPLE_BYTES * N / (stages[3] * 1e-3) / 1e9,
            "last_estimate_err_px": float(np.hypot(*(np.array(r["estimate"][:2]) - seq.gt[Wm + K, :2]))),
            "device_error": int(r["device_error"])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--h", type=float, default=H_DEFAULT)
    ap.add_argument("--sir-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-targets", type=int, default=1000)
    ap.add_argument("--batched-steps", type=int, default=5)
    ap.add_argument("--matched-frames", type=int, default=30, help="frames per sequence of the matched-RMSE "
                    "comparison (0 skips it and the surrogate training)")
    ap.add_argument("--matched-seqs", type=int, default=2)
    ap.add_argument("--surrogate-rows", type=int, default=10_000_000)
    ap.add_argument("--surrogate-steps", type=int, default=100_000)
    ap.add_argument("--pseudo-reps", type=int, default=100, help="repetitions of the pseudo-tracking experiment "
                    "(Section 5.4; 0 skips it)")
    ap.add_argument("--large-frames", type=int, default=50, help="frames of the large-object comparison "
                    "(Section 5.3; 0 skips it)")
    ap.add_argument("--frames-3d", type=int, default=20, help="frames of the 3D comparison (0 skips it)")
    ap.add_argument("--batched3-steps", type=int, default=5, help="timed steps of the batched 3D workload (0 skips it)")
    ap.add_argument("--batched3-targets", type=int, default=200)
    ap.add_argument("--surrogate3-sequences", type=int, default=1200,
                    help="four-frame training sequences of the 3D surrogate")
    ap.add_argument("--surrogate3-steps", type=int, default=10_000, help="Adam steps of the 3D surrogate (0: none)")
    ap.add_argument("--gemm", type=int, default=1, help="time the training GEMM at two shapes (0 skips it)")
    ap.add_argument("--ess-frames", type=int, default=20, help="frames of the ESS-threshold comparison (0 skips it)")
    ap.add_argument("--ess-frac", type=float, default=0.5, help="N_thr / N of the ESS-threshold comparison")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    # host threads (and so the page-locked buffers they first touch) on the CPU attached to the GPU
    cpus = gpu_cpu_affinity(local)
    if cpus:
        try:
            os.sched_setaffinity(0, cpus)
        except OSError:
            cpus = None
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if pg:
        pg.barrier()
    from paper_1310_5541_gb300 import pcsir, synth

    N, h, K, Wm = args.n, args.h, args.steps, args.warmup
    seed = SEED + 1000 * rank
    model = synth.Model(sigma_psf=SIGMA, I0=I0, bg=BG, patch=PATCH, q=Q)
    n_frames = Wm + K + max(args.sir_steps, 2) + 4
    seq = synth.make_sequence(W_IMG, H_IMG, n_frames, model, seed)
    dev = torch.device("cuda", local)
    images = torch.from_numpy(seq.images).to(dev)
    noise_host = [torch.from_numpy(synth.make_noise(N, Q, seed, j, np.float32)).pin_memory()
                  for j in range(NOISE_POOL)]
    noise = [t.to(dev) for t in noise_host]
    u0s = [synth.make_u0(seed, k) for k in range(n_frames)]
    state0 = torch.from_numpy(synth.initial_state(seq.gt[0], N, np.float32)).to(dev)
    state = state0.clone()
    ctx = pcsir.Context(N, torch.float32, patch=PATCH, psf_sigma=SIGMA, bg=BG, keep=0)
    stream = torch.cuda.current_stream()
    res_bytes = pcsir.ctypes.sizeof(pcsir.pcsir_result)
    assert res_bytes % 8 == 0
    res_host = torch.zeros((n_frames, res_bytes // 8), dtype=torch.float64).pin_memory()  # one pcsir_result each

    def step(k, st):
        r = pcsir.lib.pcsir_step(ctx.handle, pcsir._ptr(st), N, pcsir._ptr(images[k]), W_IMG, H_IMG, float(h),
                                 pcsir._ptr(noise[k % NOISE_POOL]), float(u0s[k]), pcsir._stream_ptr(stream),
                                 pcsir.ctypes.c_void_p(res_host[k].data_ptr()))
        if r != 0:
            ctx._raise(r)

    for k in range(Wm):
        step(k, state)
    torch.cuda.synchronize()
    ctx.timing_enable(K)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    sampler = ClockSampler(uuid)
    time.sleep(0.4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(Wm, Wm + K):
        step(k, state)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed_ms = e0.elapsed_time(e1)
    stages = np.array(ctx.timing_read(K))
    if pg:
        elapsed_ms = max_over_ranks(elapsed_ms, pg, dev)
        pg.barrier()
    res = np.frombuffer(res_host.numpy().tobytes(), dtype=np.dtype([
        ("est", "f8", 5), ("ess", "f8"), ("maxll", "f8"), ("sumw", "f8"), ("n", "i8"), ("nb", "i8"),
        ("err", "i4"), ("kind", "i4"), ("resampled", "i4"), ("reserved", "i4")]))
    timed = res[Wm:Wm + K]
    derr = int(np.bitwise_or.reduce(timed["err"]))
    est = timed["est"][:, :2]
    gt = seq.gt[1 + Wm:1 + Wm + K, :2]
    rmse = float(np.sqrt(np.mean(np.sum((est - gt) ** 2, axis=1))))
    value = replica_rate(N, K, world, elapsed_ms)

    # roofline of the dominant kernel (propagate + cells + centre-of-mass sums)
    hbm, peak_kind = peaks()
    st_mean = stages.mean(axis=0)
    share = st_mean / st_mean.sum()
    dom = int(np.argmax(st_mean))
    bytes_pb = PROP_BIN_BYTES * N
    achieved = bytes_pb / (st_mean[0] * 1e-3) / 1e9
    traffic = profiled_traffic(N)
    roofline = {"kernel": "k_prop_bin", "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_kind,
                "algorithmic_bytes": bytes_pb}
    resample_gbs = RESAMPLE_BYTES * N / (st_mean[3] * 1e-3) / 1e9
    deferred = run_deferred(ctx, pcsir, state0, images, noise, u0s, N, h, K, Wm, stream, seq, pg, dev, hbm,
                            peak_kind)

    # end to end through the C ABI: every step's image and noise copied in from page-locked host
    # memory and its result read back; the next step's inputs travel on a second stream into a
    # second pair of device buffers while the current step runs
    img_host = [torch.from_numpy(seq.images[k]).pin_memory() for k in range(n_frames)]
    img_dev = [torch.empty((H_IMG, W_IMG), dtype=torch.float32, device=dev) for _ in range(2)]
    nz_dev = [torch.empty((5, N), dtype=torch.float32, device=dev) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    res1 = pcsir.pcsir_result()
    K_e2e = max(3, K // 2)
    # each step's copies timed on the copy stream (the host link's rate during the loop)
    cp_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K_e2e)]

    def stage_in(k):
        j = k % 2
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(consumed[j])  # the step that read this buffer pair is done
            cp_ev[k][0].record(copy_stream)
            img_dev[j].copy_(img_host[k], non_blocking=True)
            nz_dev[j].copy_(noise_host[k % NOISE_POOL], non_blocking=True)
            cp_ev[k][1].record(copy_stream)
            copied[j].record(copy_stream)

    def run_e2e(overlap):
        """K_e2e steps end to end; with overlap the next step's copies run during the current step,
        without it each step copies, computes and reads back in turn (on one stream)."""
        state.copy_(state0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if overlap:
            stage_in(0)
        for k in range(K_e2e):
            j = k % 2
            if overlap:
                if k + 1 < K_e2e:
                    stage_in(k + 1)
                stream.wait_event(copied[j])
            else:
                img_dev[j].copy_(img_host[k], non_blocking=True)
                nz_dev[j].copy_(noise_host[k % NOISE_POOL], non_blocking=True)
            r = pcsir.lib.pcsir_step(ctx.handle, pcsir._ptr(state), N, pcsir._ptr(img_dev[j]), W_IMG, H_IMG,
                                     float(h), pcsir._ptr(nz_dev[j]), float(u0s[k]), pcsir._stream_ptr(stream),
                                     None)
            if r != 0:
                ctx._raise(r)
            consumed[j].record(stream)
            stream.synchronize()
            pcsir.lib.pcsir_last_result(ctx.handle, pcsir.ctypes.byref(res1))
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    e2e_overlap_s = run_e2e(True)
    copy_ms = sum(a.elapsed_time(b) for a, b in cp_ev)
    e2e_serial_s = run_e2e(False)
    e2e_s = min(e2e_overlap_s, e2e_serial_s)
    # the host link alone: one page-locked noise array to the device, timed with events
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    nz_dev[0].copy_(noise_host[0], non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = noise_host[0].numel() * 4 / (c0.elapsed_time(c1) * 1e-3) / 1e9
    e2e = {"value": N * K_e2e * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(4 * H_IMG * W_IMG + 5 * 4 * N), "d2h_bytes_per_step": res_bytes,
           "steps": K_e2e,
           "copies": "overlapped" if e2e_overlap_s <= e2e_serial_s else "serial",
           "overlapped_value": N * K_e2e * world / e2e_overlap_s, "serial_value": N * K_e2e * world / e2e_serial_s,
           "h2d_copy_gbs": h2d_gbs, "host_cpus": len(cpus) if cpus else None,
           "h2d_copy_gbs_overlapped": int(4 * H_IMG * W_IMG + 5 * 4 * N) * K_e2e / (copy_ms * 1e-3) / 1e9}

    drawn = {"plain": run_drawn(ctx, pcsir, state0, images, img_host, u0s, N, h, K, Wm, stream, seq, pg, dev, hbm,
                                peak_kind, False),
             "deferred": run_drawn(ctx, pcsir, state0, images, img_host, u0s, N, h, K, Wm, stream, seq, pg, dev,
                                   hbm, peak_kind, True)}

    # plain SIR on the same workload (the comparison path; likelihood for every particle)
    sir = None
    if args.sir_steps > 0:
        state.copy_(state0)
        for k in range(2):
            pcsir.sir_step(ctx, state, images[k], noise[k % NOISE_POOL], u0s[k], stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sir_sampler = ClockSampler(uuid)
        time.sleep(0.4)
        a.record(stream)
        for k in range(2, 2 + args.sir_steps):
            pcsir.sir_step(ctx, state, images[k], noise[k % NOISE_POOL], u0s[k], stream)
        b.record(stream)
        torch.cuda.synchronize()
        sir_clocks = sir_sampler.stop()
        ms = a.elapsed_time(b) / args.sir_steps
        sir = {"value": N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.sir_steps,
               "roofline": sir_roofline(N, ms, torch.cuda.get_device_properties(dev).multi_processor_count,
                                        sir_clocks),
               "clocks": sir_clocks}

    gemm = run_gemm(((8192, 8192, 8192), (4096, 256, 448))) if args.gemm else None

    batched = None
    if args.batched_steps > 0:
        batched = run_batched(args.batched_targets, args.batched_steps, 3, SEED + 77 + 1000 * rank, world)

    matched = None
    if args.matched_frames > 0:
        matched = run_matched(N, args.surrogate_rows, args.surrogate_steps, args.matched_seqs, args.matched_frames,
                              SEED + 31 + 1000 * rank)

    pseudo = None
    if args.pseudo_reps > 0:
        from paper_1310_5541_gb300 import pseudo_tracking

        t0 = time.perf_counter()
        pseudo = pseudo_tracking.run(counts=(1000, 10000, 100000), reps=args.pseudo_reps, seed=SEED + 41 + rank)
        pseudo["sir_slope"] = {p: pseudo_tracking.convergence_slope(pseudo["counts"], t["sir"])
                               for p, t in pseudo["rmse_px"].items()}
        pseudo["seconds"] = time.perf_counter() - t0

    large = None
    if args.large_frames > 0:
        large = run_large_object((12800, 1 << 17, 1 << 20), args.large_frames, SEED + 53 + 1000 * rank)

    ess_cmp = None
    if args.ess_frames > 0:
        ess_cmp = run_ess(N, args.ess_frames, args.ess_frac, SEED + 71 + 1000 * rank)

    track3d = None
    if args.frames_3d > 0:
        track3d = run_3d((200_000, 1 << 22), args.frames_3d, SEED + 61 + 1000 * rank, args.surrogate3_sequences,
                         args.surrogate3_steps)
    if args.batched3_steps > 0:
        track3d = track3d or {}
        track3d["batched"] = run_batched3(args.batched3_targets, 200_000, args.batched3_steps, 3,
                                          SEED + 63 + 1000 * rank, world)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_s = 1 << 18
        rate, steps, tot = cpu_oracle_rate(n_s, 12.0, SEED + 17, h)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "N=2^18 particles of the same workload, %d oracle pcSIR steps (%.1f s)" % (steps, tot)}
        procs = len(cpus) if cpus else (os.cpu_count() or 1)
        rate_all, steps_all, busiest = cpu_oracle_rate_all_cores(n_s, 12.0, SEED + 17, h, procs)
        cpu["all_cores"] = {"value": rate_all, "unit": UNIT, "cores": procs, "kind": "oracle",
                            "sample": "%d processes, each N=2^18 particles of the same workload, %d oracle pcSIR "
                                      "steps in all (busiest process %.1f s)" % (procs, steps_all, busiest)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
            "matched": matched_summary(matched),
            "ms_per_step": elapsed_ms / K, "steps_per_s": 1e3 * K / elapsed_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(N, h), "N": N, "h": h, "image": "512x512", "patch": PATCH,
                       "state": "f32 SoA", "noise_pool": NOISE_POOL,
                       "l2": "inputs larger than L2 (state and noise 335 MB each)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline,
            "stages_ms": {"prop_bin": st_mean[0], "dummies_lik": st_mean[1], "weights": st_mean[2],
                          "scan_resample": st_mean[3], "share": [float(s) for s in share],
                          "dominant": ["prop_bin", "dummies_lik", "weights", "scan_resample"][dom],
                          "scan_resample_gbs": resample_gbs},
            "deferred": deferred, "drawn_noise": drawn, "training_gemm": gemm,
            "e2e": e2e, "sir": sir, "batched": batched, "matched_rmse": matched, "pseudo_tracking": pseudo,
            "large_object": large, "tracking_3d": track3d, "ess_threshold": ess_cmp,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": KERNELS_PER_STEP * K, "rmse_px": rmse, "mean_bins": float(timed["nb"].mean()),
            "device_error": derr,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
