#!/usr/bin/env python
"""Benchmark of the hologram-rendering hot path through the C ABI.

Default workload (asp_stft_256_t512_s512, the shape of the paper's ASP + STFT
512/512 benchmark row): 256x256 12-bit frames at fs = 71.4 kHz, angular-spectrum
propagation at z = 0.30 m, STFT windows T = 512 with stride S = 512, moments
M0/M1/M2 over 1-35 kHz (bins 8..250). One step streams 102,400 raw frames (25
batches of 4,096 frames: hv_push_frames from a device-resident pool, whose frames
the spatial stage reads in place, then hv_render of every complete window). Metric: raw frames
rendered per second. Other workloads by --workload (the paper-scale Fresnel
stream with stride 64, PCA, batched uneven streams, learned autofocus).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hv|reference]
                    [--workload NAME]

Prints one JSON line (rank 0). Multi-GPU: one independent stream per rank
(replicas; the path needs no exchange), barrier and max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import shutil
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import re  # noqa: E402

import numpy as np  # noqa: E402

from paper_2508_03911_gb300 import synth  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2508_03911_gb300", "csrc")


def profiled_traffic(profile, sources, which=0):
    """DRAM bytes per launch recorded in profiles/<profile> from an ncu capture, or
    None when the profiled kernel's sources changed since (hash mismatch)."""
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        digest = hashlib.sha256(b"".join(open(os.path.join(CSRC, f), "rb").read()
                                         for f in sources)).hexdigest()[:16]
        h = re.search(r"source_sha256_16: ([0-9a-f]{16})", text).group(1)
        vals = re.search(r"traffic_bytes_per_launch: ([^\n]+)", text).group(1)
        nums = [int(v) for v in re.findall(r"(\d+)", vals)]
        return nums[which] if h == digest else None
    except Exception:
        return None

WORKLOADS = {
    "stream_fresnel_256_t512_s64": dict(
        desc="256x256 uint16 (12-bit) frames, fs=71.4 kHz, Fresnel z=0.25 m, STFT T=512 "
             "stride 64, M0/M1/M2 over 1-35 kHz (bins 8..250), 102,400-frame stream per step",
        N=256, bits=12, spatial="fresnel", z=0.25, T=512, S=64, fs=71400.0,
        band_hz=(1000.0, 35000.0), moments=("M0", "M1", "M2"), batch=4096, batches=25,
        pool=1024, scene="scene_stream_fresnel"),
    "asp_stft_256_t512_s512": dict(
        desc="256x256 uint16 (12-bit) frames, fs=71.4 kHz, ASP z=0.30 m, STFT T=512 stride 512, "
             "M0/M1/M2 over 1-35 kHz, 102,400-frame stream per step (the paper's Table IV ASP+STFT "
             "512/512 row shape)",
        N=256, bits=12, spatial="asp", z=0.30, T=512, S=512, fs=71400.0,
        band_hz=(1000.0, 35000.0), moments=("M0", "M1", "M2"), batch=4096, batches=25,
        pool=1024, scene="scene_stream_fresnel"),
    "tiny_asp_stft_256_t64": dict(
        desc="256x256 uint8 frames, fs=20 kHz, ASP z=0.30 m, STFT T=64 stride 64, M0 over bins "
             "4..28, 102,400-frame stream per step",
        N=256, bits=8, spatial="asp", z=0.30, T=64, S=64, fs=20000.0, band=(4, 28),
        moments=("M0",), batch=4096, batches=25, pool=1024, scene="scene_tiny_asp_stft"),
    "pca_fresnel_256_t32": dict(
        desc="256x256 uint16 (12-bit) frames, Fresnel z=0.25 m, PCA over windows of T=32 "
             "(stride 32, the paper's Table IV PCA 32/32 shape), energy over eigenvectors 2..16; "
             "102,400-frame stream per step (25 batches of 4,096)",
        N=256, bits=12, spatial="fresnel", z=0.25, T=32, S=32, fs=71400.0, band=(0, 0),
        moments=(), temporal="pca", pca=(2, 16), batch=4096, batches=25, pool=1024,
        scene="scene_stream_fresnel"),
    "pca_512_t256": dict(
        desc="512x512 uint16 (12-bit) frames, ASP z=0.40 m, PCA over windows of T=256 (stride 256): "
             "FP32 covariance, Jacobi eigensolver (FP32 sweeps, then refinement with FP64 diagonal and "
             "eigenvectors), energy of the projection on eigenvectors 2..64; "
             "1,024 frames (4 windows) per step",
        N=512, bits=12, spatial="asp", z=0.40, T=256, S=256, fs=20000.0, band=(0, 0),
        moments=(), temporal="pca", pca=(2, 64), batch=1024, batches=1, pool=256,
        scene="scene_pca"),
}
# Batched uneven streams: (side N, window T, spatial transform); u16 12-bit frames, S = T,
# STFT M0/M1/M2 over 1-35 kHz at fs = 71.4 kHz, 4 windows per member and batch.
GROUP_MEMBERS = [(128, 32, "fresnel"), (128, 128, "asp"), (256, 512, "asp"), (256, 32, "fresnel"),
                 (512, 128, "asp"), (512, 32, "fresnel"), (1024, 128, "asp"), (1024, 32, "fresnel")]
GROUP_WINDOWS = 4
WORKLOADS["group_uneven_8"] = dict(
    desc="8 streams stepped together by hv_render_group: 128^2/T32/Fresnel, 128^2/T128/ASP, "
         "256^2/T512/ASP, 256^2/T32/Fresnel, 512^2/T128/ASP, 512^2/T32/Fresnel, "
         "1024^2/T128/ASP, 1024^2/T32/Fresnel; uint16 12-bit frames (seeded uniform, 128-frame pool "
         "per stream tiled on the device), S = T, STFT M0/M1/M2 over 1-35 kHz at fs = 71.4 kHz, "
         "4 windows per stream per batch (4,096 frames, 1.95 GB raw); one batch per step",
    N=0, bits=12, spatial="mixed", z=0.0, T=0, S=0, fs=71400.0, band=(0, 0),
    moments=("M0", "M1", "M2"), batch=sum(GROUP_WINDOWS * t for _, t, _ in GROUP_MEMBERS), batches=1,
    pool=0, scene="random", group=True)
WORKLOADS["autofocus_256"] = dict(
    desc="learned autofocus on 256x256 uint16 (12-bit) holograms of point-scatterer objects at "
         "z ~ U[0.10, 0.60] m (seed 1005): network input (2x2-binned log-magnitude spectrum, "
         "128x128 bfloat16) and CNN inference (4 conv 3x3 stride 2, 16/32/64/64 channels, average "
         "pool, MLP 64-32-1; trained on the GPU on 50,000 holograms labelled by the sweep unless "
         "--af-train 0); the plain "
         "64-distance ASP + Tamura sweep timed beside it; 512 holograms per step",
    N=256, bits=12, spatial="asp", z=0.0, T=0, S=0, fs=0.0, band=(0, 0), moments=(), batch=512,
    batches=1, pool=512, scene="autofocus", autofocus=True)
# conv: 2 * CI * 9 * CO * HO * WO per layer; dense 2 * 64 * 32 + 2 * 32
AF_FLOPS = (2 * 1 * 9 * 16 * 64 * 64 + 2 * 16 * 9 * 32 * 32 * 32 + 2 * 32 * 9 * 64 * 16 * 16
            + 2 * 64 * 9 * 64 * 8 * 8 + 2 * 64 * 32 + 2 * 32)
DEFAULT = "asp_stft_256_t512_s512"
METRIC = "raw frames/s rendered"


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# FP32 ALU peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # derived from unit counts and the maximum clock
_ALU = {}


def alu_peaks():
    """FP32 and FP64 FMA throughput measured on this run's device (hv_probe_peaks),
    once per process: the roofline denominators of the ALU-bound kernels."""
    if not _ALU:
        from paper_2508_03911_gb300 import hv
        try:
            _ALU.update(hv.hv_probe_peaks(int(os.environ.get("LOCAL_RANK", "0"))))
            _ALU["source"] = "measured at run time: FMA probe (hv_probe_peaks)"
        except Exception as exc:  # the probe is a measurement aid: fall back to the derived figures
            _ALU.update(fp32_tflops=FP32_PEAK_TFLOPS, fp64_tflops=1.25,
                        source=f"derived (probe failed: {exc})")
    return _ALU


def band_bins(w):
    if "band_hz" in w:
        lo, hi = w["band_hz"]
        return (math.ceil(lo * w["T"] / w["fs"] - 1e-12), math.floor(hi * w["T"] / w["fs"] + 1e-12))
    return w["band"]


def oracle_params(w):
    klo, khi = band_bins(w)
    lo, hi = w.get("pca", (2, 64))
    return dict(spatial=w["spatial"], z_m=w["z"], lambda_m=852e-9, pitch_x_m=20e-6,
                pitch_y_m=20e-6, fftshift=1, temporal=w.get("temporal", "stft"), T=w["T"],
                stride=w["S"], fs_hz=w["fs"], band_lo_bin=klo, band_hi_bin=khi,
                moments=w["moments"], pca_lo=lo, pca_hi=hi)


def make_pool(w, n):
    sc = getattr(synth, w["scene"])(N=w["N"], bits=w["bits"])
    synth.build(sc)
    return synth.frames(sc, 0, n)


def algorithmic(w):
    """Algorithmic bytes and flops per raw frame (method dataflow, see the design notes)."""
    hw = w["N"] * w["N"]
    bpp = 1 if w["bits"] <= 8 else 2
    nmom = max(1, len(w["moments"]))
    T, S = w["T"], w["S"]
    frame_bytes = hw * (bpp + 16 + 4.0 * nmom / S)
    fft2 = 5.0 * hw * math.log2(hw)
    spatial_flops = 2 * fft2 + 6 * hw if w["spatial"] == "asp" else fft2 + 6 * hw
    stft_flops = hw * 5.0 * T * math.log2(T) / S
    stft_bytes = hw * (8 + 4.0 * nmom / S)
    return dict(frame_bytes=frame_bytes, spatial_flops=spatial_flops, stft_flops=stft_flops,
                stft_bytes=stft_bytes)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                     text=True)
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((ts, parts))
        inside = [r for ts, r in rows if self.t0 and self.t1 and self.t0 - 0.15 <= ts <= self.t1 + 0.15]
        use = inside or [r for _, r in rows]
        if not use:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in use if num(r[1]) is not None]
        mx = [num(r[2]) for r in use if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in use:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(use),
                "samples_in_timed_region": len(inside)}


# ------------------------------------------------------------- replicas

def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (the job ends when its slowest replica does);
    x itself without a process group."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, units_per_step: int, seconds: float) -> float:
    """Whole-job throughput: every replica processes units_per_step per step (weak
    scaling), the job takes the slowest replica's time."""
    return world * steps * units_per_step / seconds


# --------------------------------------------------------------- hv arm

def run_hv(args, w, rank, world, dist, tuned=1, quick=False):
    import torch

    from paper_2508_03911_gb300 import hv

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    # one explicit stream for the library and for every timing event
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    pool_np = make_pool(w, w["pool"])
    B = w["batch"]
    reps = B // w["pool"]
    pool_t = torch.from_numpy(pool_np.view(np.int16) if pool_np.dtype == np.uint16 else pool_np)
    pool_dev = pool_t.to(dev).repeat(reps, 1, 1).contiguous()
    klo, khi = band_bins(w)
    N = w["N"]

    def open_renderer():
        r = hv.Renderer(N, N, 8 if w["bits"] <= 8 else 16, 2 * B, stream=stream.cuda_stream,
                        time_queue_frames=args.tq_frames)
        if w.get("temporal") == "pca":
            r.set_params(N, N, spatial=w["spatial"], z=w["z"], temporal="pca", T=w["T"],
                         stride=w["S"], pca=w["pca"], tuned=tuned,
                         precision=w.get("precision", "fp32"), spatial_kernel=args.spatial_kernel,
                         spatial_chunk=args.spatial_chunk)
        else:
            r.set_params(N, N, spatial=w["spatial"], z=w["z"], T=w["T"], stride=w["S"],
                         fs=w["fs"], band=(klo, khi), moments=w["moments"], tuned=tuned,
                         spatial_kernel=args.spatial_kernel, spatial_chunk=args.spatial_chunk,
                         stft_kernel=args.stft_kernel if tuned else "auto")
        return r

    r = open_renderer()
    wf = r.window_floats()
    max_win = B // w["S"] + 2
    out = torch.empty(max_win * wf, dtype=torch.float32, device=dev)

    def step(events=None):
        for _ in range(w["batches"]):
            if events is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            # the pool is written once before the timed region and never changed:
            # its frames may be read in place by the spatial stage (HV_MEM_DEVICE_ASYNC)
            st = r.push(pool_dev, async_=True)
            assert st == hv.HV_OK, st
            while r.render(out) > 0:  # every complete window, as a caller would
                pass
            if events is not None:
                e1 = torch.cuda.Event(enable_timing=True)
                e1.record(stream)
                events.append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    gpu_idx = None
    try:
        gpu_idx = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_idx.startswith("GPU-"):
            gpu_idx = "GPU-" + gpu_idx
    except Exception:
        gpu_idx = None
    clocks = ClockSampler(gpu_idx) if (rank == 0 and not quick) else None
    if clocks:
        clocks.start()
        time.sleep(0.6)
    stats0 = r.stats()
    hv.hv_profile_enable(r.h, True)
    lat = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark("t0")
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step(lat)
    t_end.record(stream)
    torch.cuda.synchronize()
    if clocks:
        clocks.mark("t1")
    if dist:
        dist.barrier()
    prof = hv.hv_profile_read(r.h)
    hv.hv_profile_enable(r.h, False)
    tuning = hv.hv_get_tuning(r.h)
    stats1 = r.stats()
    elapsed_ms = t_start.elapsed_time(t_end)
    lat_ms = sorted(a.elapsed_time(b) for a, b in lat)
    clk = clocks.stop() if clocks else None
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    frames_per_step = B * w["batches"]
    value = job_value(world, args.steps, frames_per_step, elapsed_ms / 1e3)
    launches = stats1["kernel_launches"] - stats0["kernel_launches"]
    r.close()
    library = None
    if not quick and not args.no_library and rank == 0:
        library = run_library(w, args, pool_dev, stream)

    if args.no_e2e or quick:
        out = dict(value=value, elapsed_ms=elapsed_ms, lat_ms=lat_ms, prof=prof, launches=launches,
                   clocks=clk, e2e=None, frames_per_step=frames_per_step, tuning=tuning)
        if library:
            out["library"] = library
        return out
    # ----- end-to-end through host buffers (pinned frames in, images out)
    host_pool = pool_t.repeat(reps, 1, 1).contiguous().pin_memory()
    r2 = open_renderer()
    out_host = torch.empty(max_win * wf, dtype=torch.float32).pin_memory()
    h2d = d2h = 0

    def step_host(count):
        # pinned frames pushed and images read back with queued copies
        # (HV_MEM_HOST_ASYNC): the upload of one batch overlaps the rendering of the
        # previous one; the step ends when the handle's streams are idle
        nonlocal h2d, d2h
        for _ in range(w["batches"]):
            assert r2.push(host_pool, async_=True) == hv.HV_OK
            n = 0
            while True:
                k = r2.render(out_host, async_=True)
                n += k
                if k == 0:
                    break
            if count:
                h2d += host_pool.numel() * host_pool.element_size()
                d2h += n * wf * 4
        r2.synchronize()
    for _ in range(max(1, args.warmup // 2)):
        step_host(False)
    torch.cuda.synchronize()
    e2e_steps = max(1, args.steps // 2)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host(True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_value = job_value(world, e2e_steps, frames_per_step, e2e_s)
    r2.close()
    # the host link's own rate for comparison: plain pinned host-to-device copies of
    # the same pool (best of three, CUDA events), outside the timed region
    link = torch.empty(host_pool.shape, dtype=host_pool.dtype, device=dev)
    link_gbs = 0.0
    with torch.cuda.stream(stream):
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            link.copy_(host_pool, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            link_gbs = max(link_gbs, host_pool.numel() * host_pool.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del link

    out = dict(value=value, elapsed_ms=elapsed_ms, lat_ms=lat_ms, prof=prof, launches=launches,
                clocks=clk, e2e=dict(value=e2e_value, unit="frames/s",
                                     h2d_bytes_per_step=h2d // e2e_steps,
                                     d2h_bytes_per_step=d2h // e2e_steps,
                                     h2d_gbs=round(h2d / e2e_s / 1e9, 1),
                                     host_link_h2d_gbs=round(link_gbs, 1),
                                     what=("pinned frames pushed (HV_MEM_HOST_ASYNC), images read back; "
                                           "h2d_gbs is the frames' rate over the host link, "
                                           "host_link_h2d_gbs that of plain pinned copies of the same pool")),
                frames_per_step=frames_per_step, tuning=tuning)
    if library:
        out["library"] = library
    return out


def roofline_pca(w, res, peaks, force=None):
    """PCA: dominant sub-stage from the live event timing (covariance, Jacobi, projection)."""
    prof = res["prof"]
    nwin = max(1, prof["windows"])
    P, T = w["N"] ** 2, w["T"]
    M = w["pca"][1] - w["pca"][0] + 1
    hbm = (peaks or {}).get("hbm_gbs", 6800.0)
    st = {"spatial": prof["spatial_ms"] / nwin, "covariance": prof["pca_cov_ms"] / nwin,
          "jacobi_fp64": prof["pca_eig_ms"] / nwin, "projection": prof["pca_proj_ms"] / nwin}
    kern = force or max(st, key=st.get)
    t = st[kern] / 1e3
    if force is None and kern != "covariance" and st["covariance"] > 0:
        # also report the covariance against its own roof
        sub = roofline_pca(w, res, peaks, force="covariance")
        entry = roofline_pca(w, res, peaks, force=kern)
        entry["covariance"] = sub
        return entry
    if kern == "covariance" and w.get("precision", "fp32") != "fp32":
        # tensor cores: algorithmic flops of the symmetric half of the real Gram matrix
        # G = Y Y^T (2T x 2T, K = P), times the products per step (3 for split-BF16),
        # against the measured bf16 peak
        nprod = 3 if w["precision"] == "split_bf16" else 1
        flops = 1.0 * (2 * T) * (2 * T + 1) * P * nprod
        peak = (peaks or {}).get("bf16_tflops", 1906.8)
        tf = flops / t / 1e12
        return {"bound": "tensor", "achieved": round(tf, 2), "peak": peak, "unit": "TFLOP/s",
                "frac": round(tf / peak, 4),
                "traffic": (profiled_traffic("cov_tc_pca_512_t256_split_bf16.md", ["k_cov_tc.cu"])
                            if w["precision"] == "split_bf16" and w["N"] == 512 and T == 256 else None),
                "kernel": f"k_cov_tc (tcgen05 {w['precision']})",
                "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)",
                "stage_ms_per_window": {k: round(v, 4) for k, v in st.items()}}
    if kern == "covariance":
        # the Hermitian half (T (T + 1) / 2 entries, 8 flops per pixel each)
        flops, byts = 4.0 * P * T * (T + 1), 8.0 * P * T
    elif kern == "projection":
        flops, byts = 8.0 * P * T * M, 8.0 * P * T
    elif kern == "jacobi_fp64":
        sweeps = prof["pca_sweeps"] / nwin
        sweeps32 = prof.get("pca_sweeps_f32", 0) / nwin
        per_sweep32 = (T - 1) * (T // 2) ** 2 * 96.0 + (T - 1) * T * (T // 2) * 32.0
        # float64 work over the whole eigensolver time: the congruence C' = Vf^H C Vf
        # (M = C Vf, then the upper triangle for T <= 64 or all of it) and the rotations
        # of V in the refinement sweeps (20 flops per row and pair); the 2 x 2 blocks of
        # C' are float32 there, and the float32 sweeps before them are bound by barriers
        per_sweep = (T - 1) * (T // 2) * T * 20.0
        congruence = 8.0 * T ** 3 + (4.0 * T * T * (T + 1) if T <= 64 else 8.0 * T ** 3)
        flops = sweeps * per_sweep + congruence
        byts = 0.0
        fp64_peak = alu_peaks()["fp64_tflops"]
        return {"bound": "alu", "achieved": round(flops / t / 1e12, 4), "peak": round(fp64_peak, 3),
                "unit": "TFLOP/s (FP64)", "frac": round(flops / t / 1e12 / fp64_peak, 4),
                "traffic": None,
                "kernel": "eigensolver (FP32 cyclic Jacobi, then refinement: FP64 diagonal and V, FP32 off-diagonal)",
                "peak_source": alu_peaks()["source"] + "; nominal GB300 FP64 1.25 TFLOP/s",
                "sweeps_per_window": round(sweeps, 2), "fp32_sweeps_per_window": round(sweeps32, 2),
                "fp32_flops_per_window": round(sweeps32 * per_sweep32),
                "stage_ms_per_window": {k: round(v, 4) for k, v in st.items()}}
    else:  # spatial: the S new frames each window propagates
        alg = algorithmic(w)
        flops = alg["spatial_flops"] * w["S"]
        byts = P * ((1 if w["bits"] <= 8 else 2) + 8.0) * w["S"]
    fp32 = alu_peaks()["fp32_tflops"]
    return {"bound": "alu", "achieved": round(flops / t / 1e12, 3), "peak": round(fp32, 1),
            "unit": "TFLOP/s", "frac": round(flops / t / 1e12 / fp32, 4), "traffic": None,
            "kernel": kern, "hbm_achieved_gbs": round(byts / t / 1e9, 1),
            "hbm_frac_of_measured": round(byts / t / 1e9 / hbm, 4),
            "peak_source": alu_peaks()["source"],
            "stage_ms_per_window": {k: round(v, 4) for k, v in st.items()}}


def roofline(w, res, peaks):
    """Roofline entry of the dominant stage, from the live per-stage event timing."""
    if w.get("temporal") == "pca":
        return roofline_pca(w, res, peaks)
    prof = res["prof"]
    alg = algorithmic(w)
    renders = max(1, prof["renders"])
    frames = res["frames_per_step"] * 0 + prof["frames"]
    t_sp = prof["spatial_ms"] / renders
    t_tm = prof["temporal_ms"] / renders
    frames_per_render = frames / renders
    hbm = (peaks or {}).get("hbm_gbs", 6800.0)
    if t_tm >= t_sp:
        flops = alg["stft_flops"] * frames_per_render
        byts = alg["stft_bytes"] * frames_per_render
        names = {1: "k_stft_warp", 2: "k_stft_win", 3: "k_stft_win (wide)", 4: "k_stft_winp", 5: "k_stft_wt",
                 6: "k_stft_wtp"}
        sk = (res.get("tuning") or {}).get("stft_kernel")
        kern, t = f"{names.get(sk, 'k_stft_warp')} (time FFT + band moments)", t_tm
    else:
        flops = alg["spatial_flops"] * frames_per_render
        byts = (w["N"] ** 2) * ((1 if w["bits"] <= 8 else 2) + 8) * frames_per_render
        kern, t = "spatial passes (FFT2)", t_sp
    tflops = flops / (t / 1e3) / 1e12
    gbs = byts / (t / 1e3) / 1e9
    fp32 = alu_peaks()["fp32_tflops"]
    alu_frac = tflops / fp32
    hbm_frac = gbs / hbm
    traffic = None
    traffic_per = "launch of the STFT kernel" if t_tm >= t_sp else \
        "render (all spatial pass launches; cold-cache ncu capture, L2 flushed)"
    tun = res.get("tuning") or {}
    if t_tm >= t_sp and w["T"] == 512 and w["N"] == 256 and w["S"] == 64 and tun.get("stft_kernel") in (0, 1, None):
        # walking STFT: a launch over 1,024 new frames captured; a launch reads its
        # new frames and the T - S frames of overlap once, so traffic scales with both
        v = profiled_traffic("stft_warp_512_stream_fresnel_256.md", ["k_stft.cu", "fft_dev.cuh"])
        if v is not None:
            ov = w["T"] - w["S"]
            traffic = int(v * (frames_per_render + ov) / (1024 + ov))
            traffic_per = "launch of the STFT kernel (1,024-frame ncu capture scaled to the launch's frames)"
    if (t_tm >= t_sp and w["T"] == 512 and w["N"] == 256 and w["S"] == 512
            and tun.get("stft_kernel") in (2, 5)):
        # window STFT (window-per-CTA, or TMA-fed): a 1,024-frame launch captured,
        # traffic in proportion to the frames
        prof = "stft_wt_512_asp_256.md" if tun.get("stft_kernel") == 5 else "stft_win_512_asp_256.md"
        v = profiled_traffic(prof, ["k_stft.cu", "fft_dev.cuh"])
        if v is not None:
            traffic = int(v * frames_per_render / 1024)
            traffic_per = "render (the STFT launch; 1,024-frame ncu capture scaled to the render's frames)"
    if t_tm < t_sp and w["N"] == 256 and w["spatial"] == "asp":
        kern = "k_spatial_fused (every spatial pass, one launch per render)" if tun.get("spatial_kernel") == 4 \
            else kern
        if tun.get("spatial_kernel") == 3 and tun.get("spatial_chunk") == 512:
            # the three persistent passes of one 512-frame launch set, scaled to a render
            parts = [profiled_traffic("spatial_pp_asp_256.md", ["k_spatial_pp.cu", "fft_dev.cuh"], i)
                     for i in range(3)]
            if all(v is not None for v in parts):
                traffic = int(sum(parts) * frames_per_render / 512)
        elif tun.get("spatial_kernel") == 4 and w["bits"] > 8:
            v = profiled_traffic("spatial_fused_asp_256.md", ["k_spatial_pp.cu", "fft_dev.cuh"])
            if v is not None:
                traffic = int(v * frames_per_render / 1024)
                traffic_per = ("render (the fused launch; cold-cache 1,024-frame ncu capture scaled to "
                               "the render's frames)")
    if alu_frac >= hbm_frac:
        return {"bound": "alu", "achieved": round(tflops, 3), "peak": round(fp32, 1),
                "unit": "TFLOP/s", "frac": round(alu_frac, 4), "traffic": traffic, "kernel": kern,
                "traffic_per": traffic_per,
                "algorithmic_bytes_per_render": int(byts),
                "peak_source": alu_peaks()["source"] + "; derived 152 SMs x 128 FP32 lanes x 2 flop "
                               "x 2.07 GHz = 80.5",
                "hbm_achieved_gbs": round(gbs, 1), "hbm_frac_of_measured": round(hbm_frac, 4),
                "stage_ms_per_render": {"spatial": round(t_sp, 4), "temporal": round(t_tm, 4)}}
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(hbm_frac, 4), "traffic": None, "kernel": kern,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
            "alu_achieved_tflops": round(tflops, 3),
            "stage_ms_per_render": {"spatial": round(t_sp, 4), "temporal": round(t_tm, 4)}}


# -------------------------------------------------------- oracle timing
#
# The oracle's steady-state rate on a workload. In steady state every raw frame is
# propagated once and one window is analysed every S frames, so
#     frames/s = 1 / (t_spatial per frame + t_window / S).
# t_spatial is timed on a sample of frames, t_window on one window (or on a
# fraction of its pixel rows, scaled up: the STFT is per pixel). Both steps are
# the oracle's own functions (hv_oracle.spatial / stft_moments / pca), run in
# worker processes started with `spawn` (safe after CUDA is in use): frames are
# spread over the workers for the spatial step, pixel-row tiles of the window for
# the STFT; a PCA window runs in one worker whose BLAS may use every thread it is
# given. The propagated window sits in shared memory (no copies in the timed
# region). Worker threads: 1 per process for the 1-core figure, else 1 per worker
# (the PCA worker: all of them).

_POOLS = {}
_WINDOWS = {}
_FRAMES = {}


def _thread_env(n):
    return {k: str(n) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS")}


def _oracle_pool(workers, threads):
    """A spawned pool of `workers` processes with `threads` BLAS/OpenMP threads each."""
    import multiprocessing as mp
    key = (workers, threads)
    if key not in _POOLS:
        saved = {k: os.environ.get(k) for k in _thread_env(1)}
        os.environ.update(_thread_env(threads))
        try:
            pool = mp.get_context("spawn").Pool(workers)
            pool.map(_warm_job, range(workers))  # workers up and the oracle imported
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        _POOLS[key] = pool
    return _POOLS[key]


def close_oracle_pools():
    for pool in _POOLS.values():
        pool.terminate()
    _POOLS.clear()
    for shm, _ in _WINDOWS.values():
        shm.close()
        shm.unlink()
    _WINDOWS.clear()
    _FRAMES.clear()


def _warm_job(_):
    from oracle import hv_oracle  # noqa: F401
    return os.getpid()


def _shared_window(name, shape):
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)


def _spatial_job(args):
    """Propagate raw frames into slots of the shared window (oracle spatial step)."""
    from oracle import hv_oracle as O
    name, shape, slots, raw, p = args
    shm, U = _shared_window(name, shape)
    for s, fr in zip(slots, raw):
        U[s] = O.spatial(O.convert(fr), p)
    del U
    shm.close()
    return len(slots)


def _temporal_job(args):
    """Oracle temporal step on pixel rows r0..r1 of the shared window (STFT), or on
    the whole window (PCA)."""
    from oracle import hv_oracle as O
    name, shape, r0, r1, p = args
    shm, U = _shared_window(name, shape)
    if p["temporal"] == "pca":
        out = O.pca(U, p["pca_lo"], p["pca_hi"])["E"][None]
    else:
        m = O.stft_moments(U[:, r0:r1], p["fs_hz"], p["band_lo_bin"], p["band_hi_bin"])
        out = np.stack([m[k] for k in O.MOMENT_ORDER if k in p["moments"]])
    del U
    shm.close()
    return out.shape


def _raw_frames(w, n):
    key = (w["desc"], n)
    if key not in _FRAMES:
        _FRAMES.clear()
        _FRAMES[key] = make_pool(w, n)
    return _FRAMES[key]


def oracle_rate(w, cores, n_spatial, row_frac=1.0):
    """Steady-state oracle frames/s on `cores` cores: t_spatial per frame from n_spatial
    frames, t_window from a row_frac fraction of one window's pixel rows (STFT; PCA takes
    the whole window). Returns (frames/s, t_spatial per frame, t_window)."""
    from multiprocessing import shared_memory
    T, S, N = w["T"], w["S"], w["N"]
    p = oracle_params(w)
    pca = p["temporal"] == "pca"
    workers = 1 if (cores == 1) else cores
    pool = _oracle_pool(workers, 1 if cores == 1 else 1)
    shape = (T, N, N)
    key = (w["desc"], T, N)
    raw = _raw_frames(w, max(T, n_spatial))
    if key not in _WINDOWS:
        shm = shared_memory.SharedMemory(create=True, size=T * N * N * 16)
        _WINDOWS[key] = (shm, False)
    shm, filled = _WINDOWS[key]
    if not filled:  # the window the temporal step reads (untimed)
        per = -(-T // workers)
        pool.map(_spatial_job, [(shm.name, shape, list(range(i, min(T, i + per))), raw[i:i + per], p)
                                for i in range(0, T, per)])
        _WINDOWS[key] = (shm, True)
    # spatial step: n_spatial frames over the workers, into the window's slots (overwriting
    # them with the same values: the sample's first T frames are the window's frames)
    per = -(-n_spatial // workers)
    jobs = [(shm.name, shape, [f % T for f in range(i, min(n_spatial, i + per))], raw[i:i + per], p)
            for i in range(0, n_spatial, per)]
    t0 = time.perf_counter()
    pool.map(_spatial_job, jobs)
    t_sp = (time.perf_counter() - t0) / n_spatial
    # temporal step
    if pca:
        pool_t = _oracle_pool(1, cores)
        t0 = time.perf_counter()
        pool_t.map(_temporal_job, [(shm.name, shape, 0, N, p)])
        t_win = time.perf_counter() - t0
    else:
        rows = max(1, int(round(N * row_frac)))
        per = -(-rows // workers)
        jobs = [(shm.name, shape, r, min(rows, r + per), p) for r in range(0, rows, per)]
        t0 = time.perf_counter()
        pool.map(_temporal_job, jobs)
        t_win = (time.perf_counter() - t0) * N / rows
    return 1.0 / (t_sp + t_win / S), t_sp, t_win


def host_cpu():
    """Core count and CPU model of this host (lscpu when present)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return os.cpu_count() or 1, model


# 1-core sample (shared with the reference arm, so both report the same rate)
ONE_CORE_SPATIAL_FRAMES = 32
ONE_CORE_ROW_FRAC = 0.25


def cpu_baseline(w, reps=3):
    """The oracle's steady-state rate on all host cores (the reported value) and on one
    core (median of reps samples, the reference arm's procedure)."""
    T, S, N = w["T"], w["S"], w["N"]
    ncpu, model = host_cpu()
    one = [oracle_rate(w, 1, ONE_CORE_SPATIAL_FRAMES, ONE_CORE_ROW_FRAC) for _ in range(reps)]
    one_fps = float(np.median([r[0] for r in one]))
    n_sp = max(T, 4 * ncpu) if ncpu > 1 else T
    allc = oracle_rate(w, ncpu, n_sp, 1.0) if ncpu > 1 else one[0]
    close_oracle_pools()
    what = "PCA window" if w.get("temporal") == "pca" else "STFT + moments window"
    return {"value": round(allc[0], 3), "unit": "frames/s", "cores": ncpu, "kind": "oracle",
            "cpu_model": model,
            "rule": "steady state: frames/s = 1 / (t_spatial per frame + t_window / S)",
            "sample": (f"FP64 numpy oracle, {ncpu} spawned worker processes: spatial step timed on "
                       f"{n_sp} frames spread over the workers ({allc[1] * 1e3:.2f} ms per frame), one "
                       f"{what} of T = {T} frames on {N}x{N} pixels spread over them by pixel rows "
                       f"({allc[2]:.2f} s), S = {S}"),
            "one_core": {"value": round(one_fps, 3), "cores": 1,
                         "sample": (f"median of {reps}: spatial step on {ONE_CORE_SPATIAL_FRAMES} frames "
                                    f"({float(np.median([r[1] for r in one])) * 1e3:.2f} ms per frame), "
                                    f"{what} on {int(ONE_CORE_ROW_FRAC * 100)} % of the pixel rows scaled "
                                    f"to the window ({float(np.median([r[2] for r in one])):.2f} s), one "
                                    "worker process with one thread")}}


def group_oracle_sample():
    """FP64 oracle on one window of each group member with N <= 256 and T <= 128."""
    from oracle import hv_oracle as O
    n_tot, t_tot = 0, 0.0
    for i, (N, T, sp) in enumerate(GROUP_MEMBERS):
        if N > 256 or T > 128:
            continue
        q = group_member_params(N, T, sp)
        fr = synth.random_frames(T, N, N, 12, seed=1003 + i)
        p = dict(spatial=sp, z_m=q["z"], lambda_m=852e-9, pitch_x_m=20e-6, pitch_y_m=20e-6,
                 fftshift=1, temporal="stft", T=T, stride=T, fs_hz=q["fs"], band_lo_bin=q["band"][0],
                 band_hi_bin=q["band"][1], moments=q["moments"])
        t0 = time.perf_counter()
        O.render(fr, p)
        t_tot += time.perf_counter() - t0
        n_tot += T
    return n_tot / t_tot, n_tot, t_tot


def run_reference(args, w, rank):
    """The oracle as it stands on one host core, one steady-state sample per step (the
    procedure of cpu_baseline's 1-core figure)."""
    if rank != 0:
        return None
    if w.get("group"):
        vals = []
        for i in range(args.warmup + args.steps):
            fps, n, _ = group_oracle_sample()
            if i >= args.warmup:
                vals.append(fps)
        return float(np.median(vals)), n
    vals = []
    for i in range(args.warmup + args.steps):
        fps, _, _ = oracle_rate(w, 1, ONE_CORE_SPATIAL_FRAMES, ONE_CORE_ROW_FRAC)
        if i >= args.warmup:
            vals.append(fps)
    close_oracle_pools()
    return float(np.median(vals)), ONE_CORE_SPATIAL_FRAMES


# -------------------------------------------------- library comparison

def library_tables(w, dev):
    """Transfer function (ASP) or chirp (Fresnel, fftshift folded in as (-1)^(j+l)) of the
    workload on the device, built in float64 by torch ops for the library route."""
    import torch
    N, lam, d = w["N"], 852e-9, 20e-6
    if w["spatial"] == "asp":
        m = torch.arange(N, device=dev, dtype=torch.float64)
        m = torch.where(m < N // 2, m, m - N)
        kx = 2 * math.pi * m / (N * d)
        k = 2 * math.pi / lam
        kz2 = k * k - kx[None, :] ** 2 - kx[:, None] ** 2
        ph = w["z"] * torch.sqrt(torch.clamp(kz2, min=0.0))
        h = torch.polar(torch.ones_like(ph), ph) * (kz2 >= 0)
        return h.to(torch.complex64)
    x = (torch.arange(N, device=dev, dtype=torch.float64) - N / 2) * d
    j = torch.arange(N, device=dev)
    ph = math.pi * (x[None, :] ** 2 + x[:, None] ** 2) / (lam * w["z"]) + math.pi * ((j[None, :] + j[:, None]) % 2)
    return torch.polar(torch.ones_like(ph), ph).to(torch.complex64)


def run_library(w, args, pool_dev, stream):
    """The same batches through library calls, outside the library under test:
    torch.fft (cuFFT plan-many) for FFT2 x H IFFT2 (or chirp x FFT2) in complex64,
    then per window a time-axis FFT over the strided queue (STFT: |S|^2 band sums by
    torch reductions) or, for PCA, C = X^H X by torch.matmul (cuBLAS complex GEMM),
    torch.linalg.eigh (cuSOLVER) and the projection energy. CUDA events on `stream`."""
    import torch
    dev = pool_dev.device
    N, T, S = w["N"], w["T"], w["S"]
    B = pool_dev.shape[0]
    tab = library_tables(w, dev)
    q = torch.empty((B, N, N), dtype=torch.complex64, device=dev)
    klo, khi = band_bins(w)
    pca = w.get("temporal") == "pca"
    if not pca:
        kk = torch.arange(klo, khi + 1, device=dev, dtype=torch.float32)
        kk = torch.where(kk < (T + 1) // 2, kk, kk - T)
        fk = (kk * w["fs"] / T / 1000.0)[:, None, None]
    starts = list(range(0, B - T + 1, S))
    nmom = max(1, len(w["moments"]))
    img = torch.empty((len(starts), nmom, N, N), dtype=torch.float32, device=dev)
    chunk = 512

    def spatial():
        for c in range(0, B, chunk):
            raw = pool_dev[c:c + chunk]
            x = (raw.to(torch.int32) & 0xFFFF).to(torch.float32) if raw.dtype == torch.int16 else raw.to(torch.float32)
            x = torch.complex(x, torch.zeros_like(x))
            if w["spatial"] == "asp":
                q[c:c + chunk] = torch.fft.ifft2(torch.fft.fft2(x) * tab)
            else:
                q[c:c + chunk] = torch.fft.fft2(x * tab)

    def temporal():
        for i, s0 in enumerate(starts):
            X = q[s0:s0 + T]
            if pca:
                Xm = X.reshape(T, N * N).transpose(0, 1)
                C = Xm.conj().transpose(0, 1) @ Xm
                lam, V = torch.linalg.eigh(C.to(torch.complex128))
                lo, hi = w["pca"]
                Vs = V.flip(-1)[:, lo - 1:hi].to(torch.complex64)
                Y = Xm @ Vs
                img[i, 0] = (Y.real ** 2 + Y.imag ** 2).sum(1).reshape(N, N)
            else:
                F = torch.fft.fft(X, dim=0)[klo:khi + 1]
                P = F.real ** 2 + F.imag ** 2
                img[i, 0] = P.sum(0)
                if nmom > 1:
                    img[i, 1] = (fk * P).sum(0)
                    img[i, 2] = (fk * fk * P).sum(0)

    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            spatial()
            temporal()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        sp = tm = 0.0
        reps = max(2, min(args.steps, 5))
        for _ in range(reps):
            ev[0].record(stream)
            spatial()
            ev[1].record(stream)
            temporal()
            ev[2].record(stream)
            torch.cuda.synchronize()
            sp += ev[0].elapsed_time(ev[1])
            tm += ev[1].elapsed_time(ev[2])
    sp /= reps
    tm /= reps
    # steady state: every frame propagated once, one window per S frames
    frames = len(starts) * S
    t_ms = sp * frames / B + tm
    del q, img
    torch.cuda.empty_cache()
    return {"value": round(frames / (t_ms / 1e3), 1), "unit": "frames/s",
            "spatial_ms_per_frame": round(sp / B, 6), "temporal_ms_per_window": round(tm / len(starts), 5),
            "what": ("torch.fft (cuFFT plan-many) FFT2 x H IFFT2 (or chirp x FFT2) in complex64 over "
                     f"{B} frames in launches of {chunk}, then per window " +
                     ("C = X^H X by torch.matmul (cuBLAS complex GEMM), torch.linalg.eigh in complex128 "
                      "(cuSOLVER), projection energy" if pca else
                      "a time-axis FFT of the strided queue (cuFFT) and |S|^2 band sums by torch reductions") +
                     "; steady state 1 / (t_spatial + t_window / S); same frames, not the library under test")}


# ------------------------------------------------------- batched streams

def group_member_params(N, T, spatial):
    return dict(spatial=spatial, z=0.25 if spatial == "fresnel" else 0.30, T=T, S=T, fs=71400.0,
                band=(math.ceil(1000.0 * T / 71400.0 - 1e-12), math.floor(35000.0 * T / 71400.0 + 1e-12)),
                moments=("M0", "M1", "M2"))


def group_bytes_per_batch():
    """Algorithmic bytes of one batch: raw 2 B/px + 16 B/px through the time queue per
    frame, and the moment images once per window."""
    tot = 0.0
    for N, T, _ in GROUP_MEMBERS:
        hw = N * N
        tot += GROUP_WINDOWS * T * hw * (2 + 16) + GROUP_WINDOWS * 3 * hw * 4
    return tot


def run_group(args, use_graph, tuned, quick=False, dist=None):
    """K steps of one hv_render_group batch each (every member: 4 windows of frames
    pushed from a device pool, then rendered); with a process group, one replica
    per rank and the slowest rank's time."""
    import torch

    from paper_2508_03911_gb300 import hv

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    rs, pools, outs = [], [], []
    for i, (N, T, sp) in enumerate(GROUP_MEMBERS):
        q = group_member_params(N, T, sp)
        nb = GROUP_WINDOWS * T
        r = hv.Renderer(N, N, 16, 2 * nb)
        r.set_params(N, N, spatial=sp, z=q["z"], T=T, stride=T, fs=q["fs"], band=q["band"],
                     moments=q["moments"], tuned=tuned)
        base = synth.random_frames(min(nb, 128), N, N, 12, seed=1003 + i).view(np.int16)
        pool = torch.from_numpy(base).to(dev).repeat(max(1, nb // base.shape[0]), 1, 1)[:nb].contiguous()
        rs.append(r)
        pools.append(pool)
        outs.append(torch.empty(GROUP_WINDOWS * r.window_floats(), dtype=torch.float32, device=dev))
    g = hv.hv_group_open([r.h for r in rs], stream=stream.cuda_stream, use_graph=use_graph)
    frames_per_batch = sum(p.shape[0] for p in pools)

    def step(events=None):
        if events is not None:
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        nw = hv.hv_render_group(g, pools, outs)
        assert nw == [GROUP_WINDOWS] * len(rs), nw
        if events is not None:
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record(stream)
            events.append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(None) if not quick else None
    if clocks:
        clocks.start()
        time.sleep(0.6)
    st0 = hv.hv_group_get_stats(g)
    lat = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark("t0")
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step(lat)
    t_end.record(stream)
    torch.cuda.synchronize()
    if clocks:
        clocks.mark("t1")
    st1 = hv.hv_group_get_stats(g)
    elapsed_ms = t_start.elapsed_time(t_end)
    lat_ms = sorted(a.elapsed_time(b) for a, b in lat)
    clk = clocks.stop() if clocks else None
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    world = dist.get_world_size() if dist else 1
    value = job_value(world, args.steps, frames_per_batch, elapsed_ms / 1e3)
    e2e = None
    if not quick and not args.no_e2e:
        # end to end: every batch's frames copied from pinned host memory (two device
        # pool sets, the copy of batch k + 1 overlapping the render of batch k on a
        # copy stream), the images read back to pinned host memory, wall clock
        hpools = [p.cpu().pin_memory() for p in pools]
        bufs = [pools, [torch.empty_like(p) for p in pools]]
        outs_h = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
        cs = torch.cuda.Stream(device=dev)
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        used = [torch.cuda.Event(), torch.cuda.Event()]

        def upload(b):
            with torch.cuda.stream(cs):
                for d, h in zip(bufs[b], hpools):
                    d.copy_(h, non_blocking=True)
            copied[b].record(cs)

        def run_e2e(K):
            upload(0)
            for k in range(K):
                b = k & 1
                stream.wait_event(copied[b])
                if k + 1 < K:
                    if k >= 1:
                        cs.wait_event(used[1 - b])
                    upload(1 - b)
                nw = hv.hv_render_group(g, bufs[b], outs)
                assert nw == [GROUP_WINDOWS] * len(rs), nw
                used[b].record(stream)
                for oh, od in zip(outs_h, outs):
                    oh.copy_(od, non_blocking=True)
            stream.synchronize()
            cs.synchronize()

        run_e2e(2)  # untimed: first copies from the freshly pinned pools, graph updates
        K = args.steps
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        tt = time.perf_counter()
        run_e2e(K)
        e2e_s = max_over_ranks((time.perf_counter() - tt) / K, dist, dev)
        e2e = {"value": round(world * frames_per_batch / e2e_s, 1), "unit": "frames/s",
               "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hpools)),
               "d2h_bytes_per_step": int(sum(o.numel() * o.element_size() for o in outs_h))}
    hv.hv_group_close(g)
    for r in rs:
        r.close()
    return dict(value=value, elapsed_ms=elapsed_ms, lat_ms=lat_ms, clocks=clk,
                launches=st1["kernel_launches"] - st0["kernel_launches"], stats=st1,
                frames_per_batch=frames_per_batch, e2e=e2e)


def group_config(name, frames_per_batch):
    return {"workload": name, "description": WORKLOADS[name]["desc"],
            "members": [{"N": N, "T": T, "S": T, "spatial": sp} for N, T, sp in GROUP_MEMBERS],
            "frames_per_step": frames_per_batch,
            "l2": "inputs larger than L2: each batch reads 1.95 GB of raw frames",
            "parallelism": f"replicas x{int(os.environ.get('WORLD_SIZE', '1'))}"}


def main_group(args):
    """Batched uneven streams: tuned form (autotuned spatial kernels, one graph per
    batch) and plain form (multi-pass kernels, launches issued per member)."""
    w = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
        dist = td
    plain = run_group(args, use_graph=False, tuned=0, quick=True, dist=dist)
    res = run_group(args, use_graph=True, tuned=1, dist=dist)
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    peaks = load_peaks()
    hbm = (peaks or {}).get("hbm_gbs", 6800.0)
    lat = res["lat_ms"]
    gbs = group_bytes_per_batch() * args.steps / (res["elapsed_ms"] / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": round(res["value"], 1), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(res["elapsed_ms"] / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": group_config(args.workload, res["frames_per_batch"]),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "what": "per batch (all 8 streams): hv_render_group, CUDA events"},
        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(gbs / hbm, 4), "traffic": None,
                     "kernel": "whole batch (all members' kernels; algorithmic bytes 18 B/px/frame "
                               "+ 12 B/px/window)",
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
        "e2e": res["e2e"],
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "form": "tuned",
        "forms": {"plain": round(plain["value"], 1), "tuned": round(res["value"], 1),
                  "plain_p99_ms": float(np.percentile(plain["lat_ms"], 99))},
        "graph": {k: res["stats"][k] for k in ("graph_launches", "graph_instantiations",
                                               "graph_updates", "capture_us_last")},
    }
    if not args.no_cpu_baseline:
        fps, n, dt = group_oracle_sample()
        line["cpu_baseline"] = {"value": round(fps, 2), "unit": "frames/s", "cores": 1, "kind": "oracle",
                                "sample": f"one window of each member with N <= 256 and T <= 128 "
                                          f"({n} frames), FP64 numpy oracle, {dt:.1f} s on 1 host core"}
    print(json.dumps(line), flush=True)



# ------------------------------------------------------------- autofocus

def main_autofocus(args):
    """Features + network inference per hologram (the learned path), the plain sweep
    beside it, end to end from pinned host frames, and the oracle on a sample."""
    import torch

    from paper_2508_03911_gb300 import af, hv
    from paper_2508_03911_gb300 import autofocus as AF
    w = WORKLOADS[args.workload]
    B = w["batch"]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    # holograms first: the process pool starts before any CUDA call. The timed batch is
    # the first B holograms of the 1,000-hologram test set (seed 1005); the network is
    # trained on --af-train holograms of the training set (seed 1004)
    workers = min(16, os.cpu_count() or 1)
    te_frames, te_z = synth.autofocus_set(max(B, 1000), N=256, seed=1005, workers=workers)
    frames = te_frames[:B]
    tr_frames = (synth.autofocus_set(args.af_train, N=256, seed=1004, workers=workers)[0]
                 if args.af_train > 0 else None)
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
        dist = td
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    r = hv.Renderer(256, 256, 16, B, stream=stream.cuda_stream)
    r.set_params(256, 256, spatial="asp", z=0.3, T=16, stride=16, band=(1, 7))
    net = af.Autofocus(B, stream=stream.cuda_stream)
    net.set_params(AF.he_uniform(1))
    accuracy = None
    if tr_frames is not None:
        # train on the GPU (the library's forward, backward and Adam kernels), labels from
        # the plain sweep; then score the 1,000 test holograms against the sweep
        pl = AF.Pipeline(max_batch=256)
        try:
            _, tr_lab, _, tr_x = pl.label_and_features(tr_frames)
            _, te_lab, _, te_x = pl.label_and_features(te_frames)
            pl.net.set_params(AF.he_uniform(1))
            hist, t_train = AF.train(pl, tr_x, tr_lab, epochs=args.af_epochs, batch=256, lr=2e-3)
            pred = pl.predict(te_x)
            err = np.abs(pred - te_lab) / AF.STEP
            const = np.abs(np.mean(tr_lab) - te_lab) / AF.STEP
            accuracy = {"within_1_step_of_sweep": round(float(np.mean(err <= 1.0)), 4),
                        "mean_steps_vs_sweep": round(float(err.mean()), 3),
                        "median_steps_vs_sweep": round(float(np.median(err)), 3),
                        "p90_steps_vs_sweep": round(float(np.percentile(err, 90)), 3),
                        "sweep_within_1_step_of_recorded_z": round(float(np.mean(np.abs(te_lab - te_z) <= AF.STEP)), 4),
                        "constant_guess_mean_steps": round(float(const.mean()), 2),
                        "train": {"holograms": int(args.af_train), "epochs": args.af_epochs, "batch": 256,
                                  "seconds": round(t_train, 1), "final_loss": round(float(hist[-1]), 5)},
                        "test_holograms": int(te_frames.shape[0])}
            net.set_params(pl.net.get_params())
            del tr_x, te_x
        finally:
            pl.close()
        del tr_frames
    fr = torch.from_numpy(frames.view(np.int16)).to(dev)
    feats = torch.empty((B, 1, 128, 128), dtype=torch.bfloat16, device=dev)
    z = torch.empty(B, dtype=torch.float32, device=dev)
    metric = torch.empty((B, AF.NZ), dtype=torch.float32, device=dev)
    zs = AF.z_grid()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        hv.hv_af_features(r.h, fr, feats)
        if ev is not None:
            ev[1].record(stream)
        net.forward(feats, z)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
        hv.hv_focus_sweep(r.h, fr, zs, metric)
    torch.cuda.synchronize()
    clocks = ClockSampler(None)
    clocks.start()
    time.sleep(0.6)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    s0 = r.stats()["kernel_launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark("t0")
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    ms = max_over_ranks(t0.elapsed_time(t1), dist, dev)
    feat_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    net_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    launches = (r.stats()["kernel_launches"] - s0) + args.steps * 5  # network: 4 convolutions + head
    # the plain sweep on the same holograms
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(max(1, args.steps // 2)):
        hv.hv_focus_sweep(r.h, fr, zs, metric)
    e1.record(stream)
    torch.cuda.synchronize()
    sweep_ms = e0.elapsed_time(e1) / max(1, args.steps // 2)
    clk = clocks.stop()
    # end to end: pinned host holograms in, distances out, wall clock; two device
    # frame buffers, the copy of step k + 1 on a copy stream overlapping step k
    host = torch.from_numpy(frames.view(np.int16)).pin_memory()
    zh = torch.empty(B, dtype=torch.float32).pin_memory()
    bufs = [fr, torch.empty_like(fr)]
    cs = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(b):
        with torch.cuda.stream(cs):
            bufs[b].copy_(host, non_blocking=True)
        copied[b].record(cs)

    def step_from(buf):
        hv.hv_af_features(r.h, buf, feats)
        net.forward(feats, z)

    def run_e2e(K):
        upload(0)
        for k in range(K):
            b = k & 1
            stream.wait_event(copied[b])
            if k + 1 < K:
                if k >= 1:
                    cs.wait_event(used[1 - b])
                upload(1 - b)
            step_from(bufs[b])
            used[b].record(stream)
            zh.copy_(z, non_blocking=True)
        stream.synchronize()
        cs.synchronize()

    run_e2e(2)  # untimed: first copies from the freshly pinned buffer
    torch.cuda.synchronize()
    tt = time.perf_counter()
    run_e2e(args.steps)
    e2e_s = max_over_ranks((time.perf_counter() - tt) / args.steps, dist, dev)
    value = job_value(world, args.steps, B, ms / 1e3)
    tflops = AF_FLOPS * B / (net_ms / 1e3) / 1e12
    peaks = load_peaks()
    hbm = (peaks or {}).get("hbm_gbs", 6800.0)
    bf16_peak = (peaks or {}).get("bf16_tflops", 1906.8)
    # features: raw hologram read, its spectrum written and read once, the bf16 input written
    feat_bytes = 256 * 256 * (2 + 8 + 8) + 128 * 128 * 2
    feat_gbs = feat_bytes * B / (feat_ms / 1e3) / 1e9
    line = {
        "metric": "holograms/s focused", "value": round(value, 1), "unit": "holograms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"], "frame": [256, 256],
                   "pixel_bits": 12, "holograms_per_step": B, "network_input": [128, 128],
                   "l2": "inputs below L2 size (64 MB of frames): the same batch each step",
                   "parallelism": "replicas x1"},
        "roofline": {"bound": "hbm", "achieved": round(feat_gbs, 1), "peak": round(hbm, 1), "unit": "GB/s",
                     "frac": round(feat_gbs / hbm, 4), "traffic": None,
                     "kernel": "network input (column and row FFT passes, binned log-magnitude spectrum)",
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                     "bytes_per_hologram": feat_bytes},
        "network_roofline": {"bound": "tensor", "achieved": round(tflops, 3), "peak": round(bf16_peak, 1),
                             "unit": "TFLOP/s", "frac": round(tflops / bf16_peak, 4),
                             "kernel": "CNN forward: layer 1 on CUDA cores, layers 2-4 as tcgen05 implicit GEMMs "
                                       "(bf16, float32 accumulation) + head",
                             "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)",
                             "flops_per_hologram": AF_FLOPS},
        "stage_ms_per_step": {"features": round(feat_ms, 4), "network": round(net_ms, 4)},
        "sweep": {"holograms_per_s": round(B / (sweep_ms / 1e3), 1), "ms_per_step": round(sweep_ms, 4),
                  "distances": AF.NZ, "speedup_of_network": round(sweep_ms / (ms / args.steps), 2)},
        "e2e": {"value": round(world * B / e2e_s, 1), "unit": "holograms/s",
                "h2d_bytes_per_step": int(host.numel() * 2), "d2h_bytes_per_step": int(B * 4)},
        "gpu_launches": launches,
        "clocks": clk,
        "accuracy": accuracy,
    }
    net.close()
    r.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    line["config"]["parallelism"] = f"replicas x{world}"
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = autofocus_oracle_sample(frames[:8])
    print(json.dumps(line), flush=True)


def autofocus_oracle_sample(frames):
    """The FP64 oracle's network input and forward pass on a few holograms."""
    from oracle import af_oracle as A
    from paper_2508_03911_gb300 import autofocus as AF
    flat = AF.he_uniform(1).astype(np.float64)
    t0 = time.perf_counter()
    x = np.stack([A.features(f) for f in frames])[:, None]
    A.forward(flat, x)
    dt = time.perf_counter() - t0
    return {"value": round(len(frames) / dt, 2), "unit": "holograms/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(frames)} holograms: FP64 features + CNN forward, {dt:.1f} s on 1 host core"}



def main_autofocus_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    frames, _ = synth.autofocus_set(4, N=256, seed=1005)
    vals = []
    for i in range(args.warmup + args.steps):
        v = autofocus_oracle_sample(frames)
        if i >= args.warmup:
            vals.append(v["value"])
    value = float(np.median(vals))
    w = WORKLOADS[args.workload]
    line = {"impl": "reference", "metric": "holograms/s focused", "value": round(value, 3),
            "unit": "holograms/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": w["desc"], "frame": [256, 256],
                       "pixel_bits": 12, "holograms_per_step": w["batch"], "network_input": [128, 128],
                       "l2": "inputs below L2 size (64 MB of frames): the same batch each step",
                       "parallelism": "replicas x1"},
            "cpu_baseline": {"value": round(value, 3), "unit": "holograms/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: 4 holograms through the FP64 oracle's features and "
                                       "CNN forward on 1 host core"},
            "e2e": {"value": round(value, 3), "unit": "holograms/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



# ------------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hv", "reference"], default="hv")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass")
    ap.add_argument("--no-library", action="store_true",
                    help="skip the cuFFT / cuBLAS comparison of the same batches")
    ap.add_argument("--precision", choices=["fp32", "bf16", "split_bf16"], default=None,
                    help="PCA covariance arithmetic (PCA workloads)")
    ap.add_argument("--form", choices=["tuned", "plain", "both"], default="both",
                    help="tuned: spatial kernels chosen by the autotuner; plain: multi-pass kernels")
    ap.add_argument("--spatial-kernel", choices=["auto", "multipass", "persistent", "cluster", "fused"],
                    default="auto",
                    help="fix the spatial kernels instead of autotuning them (profiling runs: the "
                         "autotuner's timings are distorted under a profiler)")
    ap.add_argument("--spatial-chunk", type=int, default=0, help="frames per spatial launch (0: automatic)")
    ap.add_argument("--batch", type=int, default=0,
                    help="frames per push/render batch (0: the workload's; profiling runs use small ones)")
    ap.add_argument("--batches", type=int, default=0, help="batches per step (0: the workload's)")
    ap.add_argument("--tq-frames", type=int, default=0,
                    help="time-queue capacity in frames (0: automatic; small for profiling runs)")
    ap.add_argument("--stft-kernel", choices=["auto", "walk", "window", "window_wide", "window_pipelined",
                                               "window_tma", "window_tma_pipelined"], default="auto",
                    help="fix the STFT kernel for windows that do not overlap instead of autotuning it")
    ap.add_argument("--af-train", type=int, default=50000,
                    help="autofocus workload: training holograms (0: untrained weights, no accuracy block)")
    ap.add_argument("--af-epochs", type=int, default=40, help="autofocus workload: training epochs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if WORKLOADS[args.workload].get("group") and args.impl == "hv":
        main_group(args)
        return
    if WORKLOADS[args.workload].get("autofocus"):
        if args.impl == "hv":
            main_autofocus(args)
        else:
            main_autofocus_reference(args)
        return
    w = dict(WORKLOADS[args.workload])
    if args.precision:
        w["precision"] = args.precision
    if args.batch:
        w["batch"] = args.batch
        w["pool"] = min(w["pool"], args.batch)
    if args.batches:
        w["batches"] = args.batches
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    klo, khi = band_bins(w)
    config = {"workload": args.workload, "description": w["desc"], "frame": [w["N"], w["N"]],
              "pixel_bits": w["bits"], "spatial": w["spatial"], "z_m": w["z"], "T": w["T"],
              "stride": w["S"], "fs_hz": w["fs"], "band_bins": [klo, khi],
              "moments": list(w["moments"]), "frames_per_step": w["batch"] * w["batches"],
              "batch_frames": w["batch"], "precision": w.get("precision", "fp32"),
              "l2": "inputs larger than L2: each step streams >10 GB through the time queue",
              "parallelism": f"replicas x{args.gpus}"}
    if w.get("group"):
        config = group_config(args.workload, w["batch"])

    if args.impl == "reference":
        res = run_reference(args, w, rank)
        if rank == 0:
            value, n = res
            line = {"impl": "reference", "metric": METRIC, "value": round(value, 3),
                    "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
                    "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                    "cpu_baseline": {"value": round(value, 3), "unit": "frames/s", "cores": 1,
                                     "kind": "oracle",
                                     "sample": (f"each step: one window of each member with N <= 256 "
                                                f"and T <= 128 ({n} frames) through the FP64 numpy "
                                                "oracle on 1 host core") if w.get("group") else
                                               (f"each step: the oracle's steady-state rate 1 / (t_spatial "
                                                f"+ t_window / S), spatial step on {n} frames, one window's "
                                                f"temporal step on {int(ONE_CORE_ROW_FRAC * 100)} % of its "
                                                "pixel rows scaled to the window; one worker process, one "
                                                "thread, one host core")},
                    "e2e": {"value": round(value, 3), "unit": "frames/s", "h2d_bytes_per_step": 0,
                            "d2h_bytes_per_step": 0}}
            print(json.dumps(line), flush=True)
        return

    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
        dist = td
    plain = None
    if args.form == "both":
        plain = run_hv(args, w, rank, world, dist, tuned=0, quick=True)
    res = run_hv(args, w, rank, world, dist, tuned=0 if args.form == "plain" else 1)
    if rank == 0:
        peaks = load_peaks()
        lat = res["lat_ms"]
        p50 = float(np.percentile(lat, 50)) if lat else None
        p99 = float(np.percentile(lat, 99)) if lat else None
        alg = algorithmic(w)
        hbm = (peaks or {}).get("hbm_gbs", 6800.0)
        line = {
            "metric": METRIC, "value": round(res["value"], 1), "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(res["elapsed_ms"] / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config,
            "latency_ms": {"p50": p50, "p99": p99, "what": f"per {w['batch']}-frame batch: push + "
                                                          "render, CUDA events"},
            "hbm_pct_of_measured": round(100 * res["value"] / world * alg["frame_bytes"] / 1e9 / hbm, 2),
            "algorithmic_bytes_per_frame": alg["frame_bytes"],
            "roofline": roofline(w, res, peaks),
            "e2e": ({k: (round(v, 1) if isinstance(v, float) else v) for k, v in res["e2e"].items()}
                    if res["e2e"] else None),
            "gpu_launches": res["launches"],
            "clocks": res["clocks"],
            "form": "plain" if args.form == "plain" else "tuned",
            "tuning": {"spatial_kernel": {1: "multipass", 2: "cluster", 3: "persistent", 4: "fused"}.get(
                           res["tuning"]["spatial_kernel"], "multipass"),
                       "frames_per_launch": ("every frame of a render" if res["tuning"]["spatial_kernel"] in (2, 4)
                                             else res["tuning"]["spatial_chunk"]),
                       "candidates_us_per_frame": dict(zip(
                           ["mp16", "mp32", "mp64", "mp128", "mp256", "pp64", "pp128", "pp256",
                            "pp512", "cluster", "fused"],
                           [round(v, 4) for v in res["tuning"]["candidate_us_per_frame"][:11]])),
                       "stft_kernel": {1: "walk", 2: "window", 3: "window_wide", 4: "window_pipelined",
                                       5: "window_tma", 6: "window_tma_pipelined"}.get(
                           res["tuning"].get("stft_kernel"), "walk"),
                       "stft_candidates_us_per_window": dict(zip(
                           ["walk", "window", "window_wide", "window_pipelined", "window_tma",
                            "window_tma_pipelined"],
                           [round(v, 3) for v in res["tuning"]["stft_us_per_window"][:6]]))},
        }
        if plain is not None:
            line["forms"] = {"plain": round(plain["value"], 1), "tuned": round(res["value"], 1),
                             "plain_stage_ms_per_render": {
                                 "spatial": round(plain["prof"]["spatial_ms"] / max(1, plain["prof"]["renders"]), 4),
                                 "temporal": round(plain["prof"]["temporal_ms"] / max(1, plain["prof"]["renders"]), 4)}}
        if "library" in res:
            lib = res["library"]
            lib["hbm_pct_of_measured"] = round(100 * lib["value"] * alg["frame_bytes"] / 1e9 / hbm, 2)
            lib["library_over_hv"] = round(lib["value"] / (res["value"] / world), 4)
            line["comparison"] = {"cufft_cublas": lib}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
