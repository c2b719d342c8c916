"""Host logic of bench.py that needs no GPU: the oracle's steady-state rate
(frames/s = 1 / (t_spatial per frame + t_window / S)), measured in spawned worker
processes on one core and on several, and the reference arm that repeats the
1-core procedure per step."""
import argparse
import importlib
import os

import numpy as np


def _bench():
    # a module importable by name: the spawned workers unpickle its functions
    import bench
    return importlib.reload(bench)


def _tiny(b):
    w = dict(b.WORKLOADS["tiny_asp_stft_256_t64"])
    w.update(N=32, T=8, S=4, band=(1, 3), moments=("M0", "M1", "M2"), desc="tiny host-test stream")
    return w


def test_steady_state_rule_and_worker_pools():
    b = _bench()
    w = _tiny(b)
    try:
        fps, t_sp, t_win = b.oracle_rate(w, 1, 8, 0.5)
        assert t_sp > 0 and t_win > 0
        assert np.isclose(fps, 1.0 / (t_sp + t_win / w["S"]))
        fps2, t_sp2, t_win2 = b.oracle_rate(w, 2, 8, 1.0)
        assert np.isclose(fps2, 1.0 / (t_sp2 + t_win2 / w["S"]))
    finally:
        b.close_oracle_pools()
    assert not b._POOLS and not b._WINDOWS


def test_cpu_baseline_reports_all_cores_and_one_core():
    b = _bench()
    w = _tiny(b)
    r = b.cpu_baseline(w, reps=1)
    ncpu = os.cpu_count() or 1
    assert r["kind"] == "oracle" and r["unit"] == "frames/s"
    assert r["cores"] == ncpu and r["value"] > 0
    assert r["one_core"]["cores"] == 1 and r["one_core"]["value"] > 0
    assert "t_window / S" in r["rule"]
    assert not b._POOLS  # pools closed after the measurement


def test_reference_arm_uses_the_one_core_procedure():
    b = _bench()
    w = _tiny(b)
    seen = []

    def fake_rate(w_, cores, n_sp, frac):
        seen.append((cores, n_sp, frac))
        return 100.0 + len(seen), 1e-3, 1e-2

    b.oracle_rate = fake_rate
    args = argparse.Namespace(warmup=2, steps=3)
    value, n = b.run_reference(args, w, 0)
    assert seen == [(1, b.ONE_CORE_SPATIAL_FRAMES, b.ONE_CORE_ROW_FRAC)] * 5
    assert value == np.median([103.0, 104.0, 105.0])  # warm-up samples dropped
    assert b.run_reference(args, w, 1) is None        # other ranks do no work


def test_roofline_names_the_dominant_kernel_and_takes_only_its_own_profile():
    """The roofline entry: the dominant stage from the live stage times, the STFT
    kernel named from the tuning record, and a committed profile's DRAM traffic only
    for the kernel that profile captured (scaled to the render's frames)."""
    b = _bench()
    b._ALU.update(fp32_tflops=76.5, fp64_tflops=1.25, source="test figures")
    peaks = {"hbm_gbs": 6784.8}
    walk = b.profiled_traffic("stft_warp_512_stream_fresnel_256.md", ["k_stft.cu", "fft_dev.cuh"])
    fused = b.profiled_traffic("spatial_fused_asp_256.md", ["k_spatial_pp.cu", "fft_dev.cuh"])
    assert walk and fused  # the committed summaries match the committed sources

    w = b.WORKLOADS["stream_fresnel_256_t512_s64"]
    prof = {"renders": 1, "frames": 4096, "spatial_ms": 1.0, "temporal_ms": 2.7}
    for sk in (1, 0):  # the walking kernel, or no STFT choice recorded (it then runs)
        r = b.roofline(w, {"prof": prof, "frames_per_step": 4096,
                           "tuning": {"stft_kernel": sk, "spatial_kernel": 4}}, peaks)
        assert r["kernel"].startswith("k_stft_warp")
        assert r["traffic"] == int(walk * (4096 + 448) / (1024 + 448))
    r = b.roofline(w, {"prof": prof, "frames_per_step": 4096,
                       "tuning": {"stft_kernel": 5, "spatial_kernel": 4}}, peaks)
    assert r["kernel"].startswith("k_stft_wt") and r["traffic"] is None

    w = b.WORKLOADS[b.DEFAULT]
    prof = {"renders": 1, "frames": 4096, "spatial_ms": 1.54, "temporal_ms": 0.39}
    r = b.roofline(w, {"prof": prof, "frames_per_step": 4096,
                       "tuning": {"stft_kernel": 5, "spatial_kernel": 4}}, peaks)
    assert r["kernel"].startswith("k_spatial_fused") and r["bound"] == "alu"
    assert r["traffic"] == int(fused * 4096 / 1024)
    assert r["frac"] > 0 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
