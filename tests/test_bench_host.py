"""Host-side pieces of bench.py, checked on the CPU: the compact matched-RMSE summary, the derived
FP32 / XU roofline of SIR's likelihood, and the all-core oracle baseline (spawned processes)."""
import pytest

import bench


def test_matched_summary_keeps_every_run_and_the_matched_ones():
    runs = [{"method": "sir", "h": None, "rmse_px": 0.0861, "steps_per_s": 27.9, "particles_per_s": 4.7e8},
            {"method": "pcsir", "h": 0.5, "rmse_px": 0.195, "steps_per_s": 1909.0, "particles_per_s": 3.2e10},
            {"method": "pcsir", "h": 0.1, "rmse_px": 0.0866, "steps_per_s": 1405.0, "particles_per_s": 2.36e10}]
    m = {"N": 1 << 24, "target_rmse_px": 1.05 * 0.0861, "runs": runs,
         "matched": {"sir": runs[0], "pcsir": runs[2], "surrogate_pcsir": None}}
    s = bench.matched_summary(m)
    assert s["columns"][0] == "method" and len(s["runs"]) == 3
    assert s["at_matched_rmse"]["pcsir"] == ["pcsir", 0.1, 0.0866, 1405.0, 2.36e10]
    assert s["at_matched_rmse"]["surrogate_pcsir"] is None
    assert bench.matched_summary(None) is None


def test_sir_roofline_arithmetic():
    r = bench.sir_roofline(1 << 24, 36.0, 152, {"sm_mhz": 2070.0})
    terms = (1 << 24) * 21 * 21
    assert r["pixel_terms_per_step"] == terms
    assert r["peak"] == pytest.approx(152 * 128 * 2070e6 / 1e12)
    assert r["achieved"] == pytest.approx(terms * 8 / 0.036 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["xu"]["peak"] == pytest.approx(152 * 16 * 2070e6 / 1e12)
    assert bench.sir_roofline(1 << 20, 2.0, 152, None)["peak"] == pytest.approx(152 * 128 * 2070e6 / 1e12)


def test_all_core_oracle_baseline_runs_in_spawned_processes():
    rate, steps, busiest = bench.cpu_oracle_rate_all_cores(2048, 0.3, 5, 0.5, 2)
    assert rate > 0 and steps >= 4 and busiest > 0


def test_algorithmic_bytes_follow_the_fp32_state_layout():
    """Per-particle bytes behind the reported HBM fractions: five FP32 state components (20 B), a
    4-byte cell slot, a 4-byte ancestor.  Propagate/bin reads state and noise and writes the
    propagated state and the slot; resampling reads the slot twice (tile sums, scan) and gathers and
    writes one state; the deferred form gathers through the ancestor and writes only the ancestor."""
    import bench

    state, slot, anc = 5 * 4, 4, 4
    assert bench.PROP_BIN_BYTES == 2 * state + state + slot
    assert bench.RESAMPLE_BYTES == 2 * slot + 2 * state
    assert bench.DEFERRED_PROP_BIN_BYTES == anc + 2 * state + state + slot
    assert bench.DEFERRED_RESAMPLE_BYTES == 2 * slot + anc
    assert bench.DRAWN_PROP_BIN_BYTES == bench.PROP_BIN_BYTES - state
    assert bench.DRAWN_DEFERRED_PROP_BIN_BYTES == bench.DEFERRED_PROP_BIN_BYTES - state
    assert bench.BATCHED_BYTES == 112 and bench.BATCHED_DEFERRED_BYTES == 80


def test_profiled_traffic_scales_the_committed_capture():
    """The ncu traffic of the committed propagate/bin summary is taken only for the kernel source it
    was captured on, per particle, scaled to the launch size; it stays within the algorithmic bytes
    (no re-reads) and above three quarters of them."""
    import bench

    n = 1 << 24
    t = bench.profiled_traffic(n)
    tg = bench.profiled_traffic(n, "gathering dram bytes per particle")
    assert t is not None and tg is not None
    assert 0.75 * bench.PROP_BIN_BYTES * n <= t <= bench.PROP_BIN_BYTES * n
    assert 0.75 * bench.DEFERRED_PROP_BIN_BYTES * n <= tg <= bench.DEFERRED_PROP_BIN_BYTES * n
    assert bench.profiled_traffic(2 * n) == 2 * t
