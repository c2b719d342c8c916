"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle.

Tolerances: conversion bit-exact; FP32 complex fields relative L2 <= 1e-5;
rendered moment images relative L2 <= 1e-4 (per rendered image).
"""
import numpy as np
import pytest

from oracle import hv_oracle as O
from paper_2508_03911_gb300 import hv, synth
from tests._util import images_from, oracle_params, rel_l2, to_device, to_hv

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
IMAGE_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hv.lib()  # fails loudly when the extension is missing


def gpu_render(frames, p, packets=None, out_kind="device", extra=None, queue=None, tq=0, in_place=False):
    """Push `frames` (in packets) and render all complete windows through the C ABI
    (rendering repeatedly after each packet until no window is left). in_place:
    device packets pushed with HV_MEM_DEVICE_ASYNC, read in place."""
    import torch
    n, H, W = frames.shape
    bits = 8 if frames.dtype == np.uint8 else 16
    r = hv.Renderer(W, H, bits, queue or max(n, 1), time_queue_frames=tq)
    try:
        hv.hv_set_params(r.h, to_hv(p, **(extra or {})))
        wf = r.window_floats()
        nwin_max = max(n, 1)
        if out_kind == "device":
            out = torch.zeros(nwin_max * wf + 7, dtype=torch.float32, device="cuda")
        else:
            out = np.zeros(nwin_max * wf + 7, dtype=np.float32)
        dev = to_device(frames) if out_kind == "device" else frames
        packets = packets or [n]
        done, got = 0, 0
        for k in packets:
            assert r.push(dev[done:done + k], async_=in_place) == hv.HV_OK
            done += k
            while True:
                k_win = r.render(out[got * wf:])
                got += k_win
                if k_win == 0:
                    break
        torch.cuda.synchronize()
        host = out.cpu().numpy() if out_kind == "device" else out
        return images_from(host, got, p), r.stats()
    finally:
        r.close()


def oracle_fields(frames, p):
    return np.stack([O.spatial(O.convert(f), p) for f in frames])[:, None]


# ----------------------------------------------------------- conversion

@pytest.mark.parametrize("bits", [8, 16])
def test_conversion_bit_exact_exhaustive(bits):
    if bits == 8:
        fr = np.arange(256, dtype=np.uint8).reshape(1, 16, 16)
    else:
        fr = np.arange(65536, dtype=np.uint16).reshape(1, 256, 256)
    p = oracle_params(spatial="none", temporal="none", T=1, stride=1, H=fr.shape[1], W=fr.shape[2])
    img, _ = gpu_render(fr, p)
    assert img.shape == (1, 1) + fr.shape[1:]
    assert np.array_equal(img[:, 0].real, fr.astype(np.float64))
    assert np.all(img.imag == 0)


# ------------------------------------------------------- complex fields

SIZES = [(16, 16), (32, 64), (64, 32), (128, 128), (256, 256), (512, 512), (1024, 1024)]


@pytest.mark.parametrize("H,W", SIZES)
@pytest.mark.parametrize("spatial", ["asp", "fresnel"])
def test_spatial_field_parity(H, W, spatial):
    n = 3 if H * W <= 256 * 256 else 1
    fr = synth.random_frames(n, H, W, 12, seed=100 + H + W)
    p = oracle_params(spatial=spatial, z_m=0.25, pitch_y_m=17e-6, temporal="none", T=1, stride=1,
                      H=H, W=W)
    img, st = gpu_render(fr, p)
    ref = oracle_fields(fr, p)
    assert img.shape == ref.shape
    for i in range(n):
        assert rel_l2(img[i], ref[i]) <= FIELD_TOL, (i, rel_l2(img[i], ref[i]))
    assert st["frames_propagated"] == n


@pytest.mark.parametrize("N", [128, 256, 512])
@pytest.mark.parametrize("spatial", ["asp", "fresnel"])
@pytest.mark.parametrize("bits", [8, 12])
def test_cluster_spatial_field_parity(N, spatial, bits):
    """Tuned form: the whole-frame cluster kernel (frame in distributed shared memory)."""
    n = 5 if N < 512 else 2
    fr = synth.random_frames(n, N, N, bits, seed=7 * N + bits)
    p = oracle_params(spatial=spatial, z_m=0.3, pitch_y_m=17e-6, temporal="none", T=1, stride=1,
                      H=N, W=N)
    img, st = gpu_render(fr, p, extra=dict(spatial_kernel="cluster"), queue=3, packets=[1, 2, 2][:n] if n == 5 else None)
    ref = oracle_fields(fr, p)
    for i in range(n):
        assert rel_l2(img[i], ref[i]) <= FIELD_TOL, (i, rel_l2(img[i], ref[i]))


@pytest.mark.parametrize("H,W,spatial,bits", [(64, 128, "asp", 12), (256, 256, "fresnel", 12),
                                              (512, 256, "asp", 12), (128, 512, "fresnel", 12),
                                              (1024, 1024, "asp", 12), (256, 1024, "fresnel", 8),
                                              (1024, 64, "asp", 8), (256, 256, "asp", 12),
                                              (64, 256, "asp", 8), (128, 256, "asp", 12),
                                              (64, 256, "fresnel", 8), (128, 256, "fresnel", 12)])
def test_persistent_multipass_parity(H, W, spatial, bits):
    """Persistent prefetching multi-pass kernels (frames and strips looped per CTA;
    8-line strips at side 1024, 8-byte raw copies for uint8 there). Width 256 takes
    the warp-private row passes (Fresnel; ASP with the TMA column IFFT for H <= 256)."""
    n = 7
    fr = synth.random_frames(n, H, W, bits, seed=H + 3 * W)
    p = oracle_params(spatial=spatial, z_m=0.3, pitch_y_m=17e-6, temporal="none", T=1, stride=1,
                      H=H, W=W)
    img, _ = gpu_render(fr, p, extra=dict(spatial_kernel="persistent", spatial_chunk=3),
                        packets=[2, 5])
    ref = oracle_fields(fr, p)
    for i in range(n):
        assert rel_l2(img[i], ref[i]) <= FIELD_TOL, (i, rel_l2(img[i], ref[i]))


def test_cluster_many_frames_ring_wrap():
    """More frames than resident clusters, input and time-queue rings wrapping."""
    N, n = 256, 300
    fr = synth.random_frames(n, N, N, 12, seed=99)
    p = oracle_params(spatial="fresnel", T=64, stride=16, fs_hz=71400.0, band_lo_bin=2,
                      band_hi_bin=30, moments=ALL_MOMENTS, H=N, W=N)
    img, st = gpu_render(fr, p, extra=dict(spatial_kernel="cluster"), packets=[100, 100, 100],
                       queue=200, tq=100)
    assert st["windows_rendered"] == len(O.window_starts(n, 64, 16))
    check_images(img, O.render(fr, p))


def test_autotuned_form_matches_oracle():
    """tuned = 1: the autotuner times the candidates on the handle's buffers and
    keeps one; the rendered windows are the oracle's."""
    N = 256
    fr = synth.random_frames(200, N, N, 12, seed=5)
    p = oracle_params(spatial="asp", T=64, stride=32, band_lo_bin=3, band_hi_bin=20,
                      moments=("M0", "M1"), H=N, W=N)
    import torch
    r = hv.Renderer(N, N, 16, 256)
    try:
        hv.hv_set_params(r.h, to_hv(p, tuned=1))
        out = torch.zeros(8 * 2 * N * N, device="cuda")
        assert r.push(to_device(fr)) == hv.HV_OK
        n = r.render(out)
        t = hv.hv_get_tuning(r.h)
        torch.cuda.synchronize()
        assert t["tuned"] == 1 and t["spatial_kernel"] in (1, 2, 3, 4)
        assert all(v > 0 for v in t["candidate_us_per_frame"][:11])
        img = out.cpu().numpy()[: n * 2 * N * N].reshape(n, 2, N, N)
        check_images(img, O.render(fr, p))
    finally:
        r.close()


@pytest.mark.parametrize("cut", [0.02, 0.1])
def test_asp_highpass_filter(cut):
    """High-pass spatial filter after ASP (folded into H on the GPU, applied as an
    explicit FFT-mask-IFFT after propagation by the oracle)."""
    fr = synth.random_frames(3, 64, 128, 12, seed=31)
    p = oracle_params(spatial="asp", z_m=0.3, highpass=cut, temporal="none", T=1, stride=1,
                      H=64, W=128)
    img, _ = gpu_render(fr, p)
    assert rel_l2(img, oracle_fields(fr, p)) <= FIELD_TOL
    q = oracle_params(spatial="asp", z_m=0.3, highpass=cut, T=16, stride=8, band_lo_bin=1,
                      band_hi_bin=7, moments=ALL_MOMENTS, H=64, W=128)
    fr2 = synth.random_frames(40, 64, 128, 12, seed=32)
    img2, _ = gpu_render(fr2, q)
    check_images(img2, O.render(fr2, q))


def test_fresnel_without_fftshift_and_negative_z():
    fr = synth.random_frames(2, 64, 128, 8, seed=5)
    for shift, z in ((0, 0.2), (1, -0.3)):
        p = oracle_params(spatial="fresnel", fftshift=shift, z_m=z, temporal="none", T=1, stride=1,
                          H=64, W=128)
        img, _ = gpu_render(fr, p)
        assert rel_l2(img, oracle_fields(fr, p)) <= FIELD_TOL
    p = oracle_params(spatial="asp", z_m=-0.4, temporal="none", T=1, stride=1, H=64, W=128)
    img, _ = gpu_render(fr, p)
    assert rel_l2(img, oracle_fields(fr, p)) <= FIELD_TOL


# -------------------------------------------------------- STFT moments

def check_images(img, ref, tol=IMAGE_TOL):
    assert img.shape == ref.shape, (img.shape, ref.shape)
    for w in range(ref.shape[0]):
        for q in range(ref.shape[1]):
            e = rel_l2(img[w, q], ref[w, q])
            assert e <= tol, (w, q, e)


def test_tiny_asp_stft_scene():
    """64 frames of 256x256 uint8, ASP z=0.30 m, STFT T=64, M0 over bins 4..28."""
    sc = synth.build(synth.scene_tiny_asp_stft())
    fr = synth.frames(sc, 0, 64)
    p = oracle_params(H=256, W=256)
    img, st = gpu_render(fr, p)
    check_images(img, O.render(fr, p))
    assert st["windows_rendered"] == 1 and st["frames_dropped"] == 0


ALL_MOMENTS = ("M0", "M1", "M2", "M1N", "M2N")


@pytest.mark.parametrize("T,S,spatial", [(8, 8, "asp"), (16, 4, "asp"), (32, 5, "fresnel"),
                                         (64, 96, "fresnel"), (128, 32, "none"), (256, 64, "asp")])
def test_stft_windows_strides_and_moments(T, S, spatial):
    H, W = 32, 64
    n = T + 3 * S + 5  # ragged tail: frames after the last complete window stay queued
    fr = synth.random_frames(n, H, W, 12, seed=T * 7 + S)
    p = oracle_params(spatial=spatial, T=T, stride=S, fs_hz=71400.0, band_lo_bin=1,
                      band_hi_bin=T // 2 + 1, moments=ALL_MOMENTS, H=H, W=W)
    img, st = gpu_render(fr, p)
    ref = O.render(fr, p)
    check_images(img, ref)
    assert st["windows_rendered"] == len(O.window_starts(n, T, S))


@pytest.mark.parametrize("T,S,band", [(256, 3, (2, 100)), (512, 700, (8, 250)), (512, 64, (1, 255)),
                                      (1024, 1024, (10, 300)), (256, 256, (0, 127))])
def test_long_window_kernel_paths(T, S, band):
    """Long windows: S < T ring prefetch, S > T alternating halves, bands below
    T/2 (pruned last stage) and up to the half-spectrum edge."""
    H, W = 16, 32
    n = T + 4 * S + 3
    fr = synth.random_frames(n, H, W, 12, seed=T + S)
    p = oracle_params(spatial="fresnel", T=T, stride=S, fs_hz=71400.0, band_lo_bin=band[0],
                      band_hi_bin=band[1], moments=ALL_MOMENTS, H=H, W=W)
    img, _ = gpu_render(fr, p)
    check_images(img, O.render(fr, p))


@pytest.mark.parametrize("T,S,tq", [(512, 256, 0), (1024, 256, 0), (64, 16, 0), (128, 32, 256),
                                    (512, 64, 1000), (256, 48, 0)])
def test_staged_frame_paths(T, S, tq):
    """Overlapping windows stage the S new frames of the next window: one TMA tile
    load per CTA when S divides T, the queue capacity and the first slot (1, 2 or 4
    pixels per warp; a small queue that wraps between launches), else per-warp
    cp.async (queue capacity 1000 or S = 48 not dividing T)."""
    H, W = 16, 32
    n = T + 6 * S + 3
    fr = synth.random_frames(n, H, W, 12, seed=T + 3 * S + tq)
    p = oracle_params(spatial="fresnel", T=T, stride=S, fs_hz=71400.0, band_lo_bin=2,
                      band_hi_bin=T // 2 - 3, moments=ALL_MOMENTS, H=H, W=W)
    img, st = gpu_render(fr, p, tq=tq, packets=[T + S, 2 * S + 1, n - T - 3 * S - 1])
    ref = O.render(fr, p)
    check_images(img, ref)
    assert st["windows_rendered"] == ref.shape[0]


def test_streaming_packets_match_one_shot():
    """Ragged packets and renders interleaved give the windows of the whole stream."""
    H = W = 64
    T, S = 32, 8
    fr = synth.random_frames(150, H, W, 8, seed=77)
    p = oracle_params(spatial="asp", T=T, stride=S, band_lo_bin=2, band_hi_bin=12,
                      moments=("M0", "M2"), H=H, W=W)
    img, st = gpu_render(fr, p, packets=[1, 30, 7, 50, 3, 59])
    check_images(img, O.render(fr, p))
    assert st["frames_pushed"] == 150


def test_host_buffers_path():
    H = W = 64
    fr = synth.random_frames(40, H, W, 12, seed=3)
    p = oracle_params(spatial="fresnel", T=16, stride=8, band_lo_bin=1, band_hi_bin=7,
                      moments=ALL_MOMENTS, H=H, W=W)
    img, _ = gpu_render(fr, p, out_kind="host", packets=[13, 27])
    check_images(img, O.render(fr, p))


def test_async_host_push_and_render():
    """Host frames pushed and images read back asynchronously (HV_MEM_HOST_ASYNC)
    through a ring smaller than the stream: slot reuse is ordered on the device."""
    import torch
    H = W = 64
    T, S, n = 16, 8, 200
    fr = synth.random_frames(n, H, W, 12, seed=8)
    p = oracle_params(spatial="asp", T=T, stride=S, band_lo_bin=1, band_hi_bin=7, moments=("M0", "M2"),
                      H=H, W=W)
    src = torch.from_numpy(fr.view(np.int16)).pin_memory()
    r = hv.Renderer(W, H, 16, 48)
    try:
        hv.hv_set_params(r.h, to_hv(p))
        wf = r.window_floats()
        out = torch.zeros(n * wf, dtype=torch.float32).pin_memory()
        got = 0
        for a in range(0, n, 24):
            assert r.push(src[a:a + 24], async_=True) == hv.HV_OK
            while True:
                k = r.render(out[got * wf:], async_=True)
                got += k
                if k == 0:
                    break
        r.synchronize()
    finally:
        r.close()
    img = images_from(out.numpy(), got, p)
    check_images(img, O.render(fr, p))


@pytest.mark.parametrize("spatial", ["asp", "fresnel"])
def test_async_device_push(spatial):
    """Device frames pushed with HV_MEM_DEVICE_ASYNC: read in place by the spatial
    stage from aligned pointers, copied on the copy stream (after the ring slots
    they overwrite have been consumed) from a pointer 2 bytes off alignment, mixed
    with plain device and host pushes, ragged packets, through an input ring
    smaller than the stream; a render's frames come from several sources in turn.
    The images match the oracle."""
    import torch
    H = W = 64
    T, S, n = 16, 8, 203
    fr = synth.random_frames(n, H, W, 12, seed=9)
    p = oracle_params(spatial=spatial, T=T, stride=S, band_lo_bin=1, band_hi_bin=7, moments=("M0", "M1"),
                      H=H, W=W)
    src = to_device(fr)
    flat = torch.empty(n * H * W + 1, dtype=torch.int16, device="cuda")
    off = flat[1:].view(n, H, W)  # 2 bytes off 16-byte alignment
    off.copy_(src)
    torch.cuda.synchronize()
    assert off.data_ptr() % 16 == 2
    r = hv.Renderer(W, H, 16, 50)
    try:
        hv.hv_set_params(r.h, to_hv(p))
        wf = r.window_floats()
        out = torch.zeros(n * wf, dtype=torch.float32, device="cuda")
        got, a = 0, 0
        kinds = ["in place", "in place", "offset", "in place", "device", "in place", "host", "offset", "in place"]
        for k, kind in zip([21, 24, 24, 17, 24, 24, 24, 24, 21], kinds):
            if kind == "in place":
                st = r.push(src[a:a + k], async_=True)
            elif kind == "offset":
                st = r.push(off[a:a + k], async_=True)
            elif kind == "device":
                st = r.push(src[a:a + k])
            else:
                st = r.push(fr[a:a + k])
            assert st == hv.HV_OK
            a += k
            while True:
                m = r.render(out[got * wf:])
                got += m
                if m == 0:
                    break
        assert a == n
        r.synchronize()
    finally:
        r.close()
    img = images_from(out.cpu().numpy(), got, p)
    check_images(img, O.render(fr, p))


def test_max_window_length():
    H, W, T = 16, 32, 1024
    fr = synth.random_frames(T + 256, H, W, 12, seed=11)
    p = oracle_params(spatial="asp", T=T, stride=256, band_lo_bin=3, band_hi_bin=900,
                      moments=ALL_MOMENTS, H=H, W=W)
    img, _ = gpu_render(fr, p)
    check_images(img, O.render(fr, p))


@pytest.mark.slow
def test_paper_scale_stream_prefix():
    """256x256 12-bit, Fresnel z=0.25 m, T=512 S=64, M0/M1/M2 over 1..35 kHz at
    fs = 71.4 kHz (bins 8..250): the first 768 frames (5 windows), every pixel."""
    sc = synth.build(synth.scene_stream_fresnel())
    fr = synth.frames(sc, 0, 768)
    klo, khi = O.band_bins_from_hz(1000.0, 35000.0, 71400.0, 512)
    p = oracle_params(spatial="fresnel", z_m=0.25, T=512, stride=64, fs_hz=71400.0,
                      band_lo_bin=klo, band_hi_bin=khi, moments=("M0", "M1", "M2"), H=256, W=256)
    img, _ = gpu_render(fr, p)
    check_images(img, O.render(fr, p))


# --------------------------------------------------------- C-ABI edges

def test_queue_full_backpressure_and_empty_render():
    import torch
    r = hv.Renderer(32, 32, 16, 10)
    try:
        p = oracle_params(H=32, W=32, T=8, stride=8, band_lo_bin=1, band_hi_bin=3)
        hv.hv_set_params(r.h, to_hv(p))
        out = torch.zeros(10 * 32 * 32, device="cuda")
        assert r.render(out) == 0                              # nothing queued
        fr = to_device(synth.random_frames(12, 32, 32, 12, 1))
        assert r.push(fr[:11]) == hv.HV_ERR_QUEUE_FULL        # all-or-nothing
        assert r.stats()["frames_pushed"] == 0
        assert r.push(fr[:10]) == hv.HV_OK
        assert r.push(fr[10:12]) == hv.HV_ERR_QUEUE_FULL
        assert r.render(out[:100]) == 0                        # capacity below one window
        assert r.render(out) == 1
        assert r.push(fr[10:12]) == hv.HV_OK                   # space freed by the window
        s = r.stats()
        assert s["frames_rejected"] == 13 and s["frames_dropped"] == 0
    finally:
        r.close()


@pytest.mark.parametrize("async_", [False, True])
def test_set_params_is_delayed_to_the_next_window(async_):
    """A new z applies from the next window on; that window is computed wholly
    with the new settings. async_: the device frames are read in place
    (HV_MEM_DEVICE_ASYNC), so the frames the new settings transform again come
    from the caller's buffer once more."""
    import torch
    H = W = 32
    fr = synth.random_frames(48, H, W, 12, seed=21)
    p1 = oracle_params(H=H, W=W, T=16, stride=8, z_m=0.2, band_lo_bin=1, band_hi_bin=7)
    p2 = dict(p1, z_m=0.35)
    r = hv.Renderer(W, H, 16, 64)
    try:
        hv.hv_set_params(r.h, to_hv(p1))
        out = torch.zeros(8 * H * W, device="cuda")
        dev = to_device(fr)
        r.push(dev[:24], async_=async_)
        n1 = r.render(out)                      # windows at 0, 8
        hv.hv_set_params(r.h, to_hv(p2))
        r.push(dev[24:], async_=async_)
        n2 = r.render(out[n1 * H * W:])          # windows at 16, 24, 32 with z = 0.35
        torch.cuda.synchronize()
        img = out.cpu().numpy()[: (n1 + n2) * H * W].reshape(n1 + n2, 1, H, W)
        assert (n1, n2) == (2, 3)
        ref1 = O.render(fr[:24], p1)
        ref2 = O.render(fr[16:], p2)
        check_images(img[:2], ref1)
        check_images(img[2:], ref2)
    finally:
        r.close()


def test_invalid_settings_are_rejected_and_previous_kept():
    r = hv.Renderer(64, 64, 8, 8)
    try:
        bad = [dict(W=48), dict(W=128), dict(T=12), dict(T=2048), dict(band_hi_bin=64),
               dict(moments=()), dict(spatial="fresnel", z_m=0.0)]
        for b in bad:
            p = oracle_params(H=64, W=64, T=16, stride=16, band_lo_bin=1, band_hi_bin=5)
            p.update(b)
            with pytest.raises(hv.HvError) as ei:
                hv.hv_set_params(r.h, to_hv(p))
            assert ei.value.status == hv.HV_ERR_ARG
    finally:
        r.close()


def test_probe_peaks_are_plausible():
    """The FMA probe behind the ALU rooflines: FP32 within the unit-count bound
    (152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s, a little slack for the
    clock) and FP64 well below it."""
    p = hv.hv_probe_peaks(0)
    assert p["sm_count"] > 0 and p["sm_clock_khz"] > 0
    bound = p["sm_count"] * 128 * 2 * p["sm_clock_khz"] * 1e3 / 1e12
    assert 0.3 * bound < p["fp32_tflops"] <= 1.05 * bound, (p, bound)
    assert 0.0 < p["fp64_tflops"] < 0.2 * p["fp32_tflops"], p


@pytest.mark.parametrize("spatial,T,S", [("asp", 64, 64), ("asp", 32, 8), ("fresnel", 64, 16)])
def test_persistent_passes_through_stft(spatial, T, S):
    """The tuned path's spatial passes at 256 x 256 feeding the STFT: moments against
    the oracle (u8 frames, several windows, chunks smaller than the stream)."""
    H = W = 256
    n = T + 3 * S
    fr = synth.random_frames(n, H, W, 8, seed=T + S + (1 if spatial == "asp" else 2))
    p = oracle_params(spatial=spatial, z_m=0.3, T=T, stride=S, fs_hz=20000.0, band_lo_bin=2,
                      band_hi_bin=T // 2 - 2, moments=ALL_MOMENTS, H=H, W=W)
    img, st = gpu_render(fr, p, extra=dict(spatial_kernel="persistent", spatial_chunk=48))
    ref = O.render(fr, p)
    check_images(img, ref)
    assert st["windows_rendered"] == ref.shape[0]


# ------------------------------------------------- fused spatial transform

@pytest.mark.parametrize("spatial,bits", [("asp", 12), ("asp", 8), ("fresnel", 12), ("fresnel", 8)])
def test_fused_spatial_field_parity(spatial, bits):
    """The fused transform at 256 x 256: every pass of every frame in one persistent
    launch, intermediates in rings of 96 frames. 220 frames pushed as packets of 1,
    97 and 122 (launches of one frame and of more than two ring generations; input
    and time-queue rings wrapping), every field against the oracle."""
    N, n = 256, 220
    fr = synth.random_frames(n, N, N, bits, seed=400 + bits + (1 if spatial == "asp" else 2))
    p = oracle_params(spatial=spatial, z_m=0.27, pitch_y_m=17e-6, temporal="none", T=1, stride=1,
                      H=N, W=N)
    img, st = gpu_render(fr, p, extra=dict(spatial_kernel="fused"), packets=[1, 97, 122], queue=160,
                         tq=150)
    ref = oracle_fields(fr, p)
    assert img.shape == ref.shape
    for i in range(n):
        assert rel_l2(img[i], ref[i]) <= FIELD_TOL, (i, rel_l2(img[i], ref[i]))
    assert st["frames_propagated"] == n


def test_fused_reads_frames_in_place():
    """The fused transform reading device frames in place (HV_MEM_DEVICE_ASYNC):
    one launch per pushed packet (1, 97 and 122 frames), each over the caller's
    buffer; every field against the oracle."""
    N, n = 256, 220
    fr = synth.random_frames(n, N, N, 16, seed=431)
    p = oracle_params(spatial="asp", z_m=0.27, temporal="none", T=1, stride=1, H=N, W=N)
    img, st = gpu_render(fr, p, extra=dict(spatial_kernel="fused"), packets=[1, 97, 122], queue=160,
                         tq=150, in_place=True)
    ref = oracle_fields(fr, p)
    for i in range(n):
        assert rel_l2(img[i], ref[i]) <= FIELD_TOL, (i, rel_l2(img[i], ref[i]))
    assert st["frames_propagated"] == n


@pytest.mark.parametrize("spatial,T,S,highpass", [("asp", 64, 64, 0.0), ("asp", 32, 8, 0.03),
                                                  ("fresnel", 64, 16, 0.0)])
def test_fused_passes_through_stft(spatial, T, S, highpass):
    """The fused transform feeding the STFT: every moment against the oracle (u8
    frames, several windows, the high-pass filter folded into H)."""
    H = W = 256
    n = T + 5 * S + 3
    fr = synth.random_frames(n, H, W, 8, seed=T + S + 17)
    p = oracle_params(spatial=spatial, z_m=0.3, T=T, stride=S, fs_hz=20000.0, band_lo_bin=2,
                      band_hi_bin=T // 2 - 2, moments=ALL_MOMENTS, H=H, W=W, highpass=highpass)
    img, st = gpu_render(fr, p, extra=dict(spatial_kernel="fused"), packets=[T + S, n - T - S])
    ref = O.render(fr, p)
    check_images(img, ref)
    assert st["windows_rendered"] == ref.shape[0]


def test_fused_rejects_other_sizes():
    r = hv.Renderer(128, 128, 16, 8)
    try:
        p = oracle_params(H=128, W=128, T=8, stride=8, band_lo_bin=1, band_hi_bin=3)
        with pytest.raises(hv.HvError) as ei:
            hv.hv_set_params(r.h, to_hv(p, spatial_kernel="fused"))
        assert ei.value.status == hv.HV_ERR_UNSUPPORTED
    finally:
        r.close()


def test_fused_stall_is_reported_and_the_context_stays_usable():
    """Failure path of the fused transform's device waits, by fault injection (no
    GPU fault): the row items of one launch wait on a condition that nothing sets.
    The producers' bounded waits give up after about a second, every CTA returns,
    and hv_synchronize reports HV_ERR_CUDA. The launch before it on the same handle
    was exact, and a new handle on the same context renders exact fields after it."""
    import time
    import torch
    N, n = 256, 40
    fr = synth.random_frames(2 * n, N, N, 16, seed=437)
    p = oracle_params(spatial="asp", z_m=0.27, temporal="none", T=1, stride=1, H=N, W=N)
    dev = to_device(fr)
    ref = oracle_fields(fr, p)
    r = hv.Renderer(N, N, 16, 2 * n)
    try:
        hv.hv_set_params(r.h, to_hv(p, spatial_kernel="fused"))
        with pytest.raises(hv.HvError) as ei:
            hv.hv_debug_inject(r.h, 7)
        assert ei.value.status == hv.HV_ERR_ARG
        wf = r.window_floats()
        out = torch.zeros(2 * n * wf, dtype=torch.float32, device="cuda")
        assert r.push(dev[:n]) == hv.HV_OK
        got = 0
        while (k := r.render(out[got * wf:])) > 0:
            got += k
        r.synchronize()
        img = images_from(out.cpu().numpy(), got, p)
        for i in range(n):
            assert rel_l2(img[i], ref[i]) <= FIELD_TOL, (i, rel_l2(img[i], ref[i]))
        hv.hv_debug_inject(r.h, hv.HV_INJECT_FUSED_STALL)
        assert r.push(dev[n:]) == hv.HV_OK
        t0 = time.perf_counter()
        while (k := r.render(out[got * wf:])) > 0:
            got += k
        with pytest.raises(hv.HvError) as ei:
            r.synchronize()
        assert ei.value.status == hv.HV_ERR_CUDA and "bounded wait" in str(ei.value)
        assert time.perf_counter() - t0 < 30
    finally:
        r.close()
    img, _ = gpu_render(fr[n:], p, extra=dict(spatial_kernel="fused"))
    for i in range(n):
        assert rel_l2(img[i], ref[n + i]) <= FIELD_TOL, (i, rel_l2(img[i], ref[n + i]))


@pytest.mark.slow
@pytest.mark.parametrize("spatial", ["fresnel", "asp"])
def test_fused_paper_scale_stream_prefix(spatial):
    """The paper-scale stream's shape through the fused transform: 256x256 12-bit,
    T=512 S=64, M0/M1/M2 over 1..35 kHz at fs = 71.4 kHz, the first 768 frames."""
    sc = synth.build(synth.scene_stream_fresnel())
    fr = synth.frames(sc, 0, 768)
    klo, khi = O.band_bins_from_hz(1000.0, 35000.0, 71400.0, 512)
    p = oracle_params(spatial=spatial, z_m=0.25, T=512, stride=64, fs_hz=71400.0,
                      band_lo_bin=klo, band_hi_bin=khi, moments=("M0", "M1", "M2"), H=256, W=256)
    img, _ = gpu_render(fr, p, extra=dict(spatial_kernel="fused"))
    check_images(img, O.render(fr, p))


# ------------------------------------------- STFT: one CTA per (window, tile)

@pytest.mark.parametrize("T,S,band", [(8, 8, (1, 3)), (32, 40, (2, 20)), (64, 64, (4, 28)),
                                      (128, 128, (1, 63)), (256, 300, (0, 127)), (512, 512, (8, 250)),
                                      (512, 700, (3, 400)), (1024, 1024, (10, 300))])
def test_window_per_cta_stft(T, S, band):
    """Windows that do not overlap through the kernel with one CTA per (window, pixel
    tile), frames landing straight in padded rows and transformed in place: every
    moment against the oracle, bands below and across T/2, gaps between windows."""
    H, W = 16, 32
    n = T + 3 * S + 5
    fr = synth.random_frames(n, H, W, 12, seed=T + 5 * S)
    p = oracle_params(spatial="fresnel", T=T, stride=S, fs_hz=71400.0, band_lo_bin=band[0],
                      band_hi_bin=band[1], moments=ALL_MOMENTS, H=H, W=W)
    ref = O.render(fr, p)
    # window_tma*: kernels of their own at T = 512, the window-per-CTA kernel elsewhere
    for kern in ("window", "window_wide", "window_pipelined", "window_tma", "window_tma_pipelined"):
        img, st = gpu_render(fr, p, extra=dict(stft_kernel=kern), packets=[T + S, n - T - S])
        check_images(img, ref)
        assert st["windows_rendered"] == ref.shape[0]


def test_stft_autotuner_times_both_kernels():
    """tuned = 1 with S = T: both STFT kernels are timed on the handle's queue and the
    faster kept; the rendered windows are the oracle's either way."""
    import torch
    N, T = 64, 64
    fr = synth.random_frames(3 * T, N, N, 12, seed=55)
    p = oracle_params(spatial="asp", T=T, stride=T, band_lo_bin=3, band_hi_bin=40,
                      moments=("M0", "M1", "M2"), H=N, W=N)
    r = hv.Renderer(N, N, 16, 4 * T)
    try:
        hv.hv_set_params(r.h, to_hv(p, tuned=1))
        out = torch.zeros(3 * 3 * N * N, device="cuda")
        assert r.push(to_device(fr)) == hv.HV_OK
        n = r.render(out)  # the settings, and the autotuner, apply here
        torch.cuda.synchronize()
        t = hv.hv_get_tuning(r.h)
        assert t["stft_kernel"] in (1, 2, 3, 4) and min(t["stft_us_per_window"][:4]) > 0
        img = out.cpu().numpy()[: n * 3 * N * N].reshape(n, 3, N, N)
        check_images(img, O.render(fr, p))
    finally:
        r.close()


@pytest.mark.slow
def test_default_bench_configuration_every_pixel():
    """The default bench workload in the launch configuration bench.py times: its
    1,024-frame pool of 256x256 12-bit frames tiled to 4,096 on the device, ASP
    z = 0.30 m, STFT T = S = 512, M0/M1/M2 over 1-35 kHz; two batches pushed in
    place (HV_MEM_DEVICE_ASYNC) on an explicit stream, the autotuned kernels, every
    complete window rendered after each push. Each of the 16 windows is one of the
    pool's two windows: every pixel of every moment against the oracle."""
    import torch

    import bench
    w = bench.WORKLOADS[bench.DEFAULT]
    assert (w["N"], w["bits"], w["spatial"], w["T"], w["S"]) == (256, 12, "asp", 512, 512)
    pool = bench.make_pool(w, w["pool"])
    klo, khi = bench.band_bins(w)
    B = w["batch"]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    pool_dev = torch.from_numpy(pool.view(np.int16)).to(dev).repeat(B // w["pool"], 1, 1).contiguous()
    torch.cuda.synchronize()
    r = hv.Renderer(256, 256, 16, 2 * B, stream=stream.cuda_stream)
    try:
        r.set_params(256, 256, spatial=w["spatial"], z=w["z"], T=w["T"], stride=w["S"], fs=w["fs"],
                     band=(klo, khi), moments=w["moments"], tuned=1)
        wf = r.window_floats()
        out = torch.zeros((2 * B // w["S"] + 2) * wf, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        got = 0
        for _ in range(2):
            assert r.push(pool_dev, async_=True) == hv.HV_OK
            while (k := r.render(out[got * wf:])) > 0:
                got += k
        r.synchronize()
        tuning = hv.hv_get_tuning(r.h)
        host = out.cpu().numpy()
    finally:
        r.close()
    assert got == 2 * B // w["S"]
    assert tuning["tuned"] == 1
    p = oracle_params(spatial=w["spatial"], z_m=w["z"], T=w["T"], stride=w["S"], fs_hz=w["fs"],
                      band_lo_bin=klo, band_hi_bin=khi, moments=w["moments"], H=256, W=256)
    img = images_from(host, got, p)
    ref = O.render(pool, p)
    assert ref.shape[0] == 2
    for i in range(got):
        check_images(img[i:i + 1], ref[i % 2:i % 2 + 1])


@pytest.mark.slow
def test_paper_scale_stream_bench_configuration_every_pixel():
    """The paper-scale stream workload in the launch configuration bench.py times:
    its 1,024-frame pool of 256x256 12-bit frames tiled to 4,096 on the device,
    Fresnel z = 0.25 m, STFT T = 512, S = 64, M0/M1/M2 over 1-35 kHz; two batches
    pushed in place on an explicit stream, the autotuned kernels. The stream has
    period 1,024 frames, so window i equals window i mod 16 of the pool repeated:
    every pixel of every moment of all 121 windows against the oracle."""
    import torch

    import bench
    w = bench.WORKLOADS["stream_fresnel_256_t512_s64"]
    assert (w["N"], w["bits"], w["spatial"], w["T"], w["S"]) == (256, 12, "fresnel", 512, 64)
    pool = bench.make_pool(w, w["pool"])
    klo, khi = bench.band_bins(w)
    B, T, S = w["batch"], w["T"], w["S"]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    pool_dev = torch.from_numpy(pool.view(np.int16)).to(dev).repeat(B // w["pool"], 1, 1).contiguous()
    torch.cuda.synchronize()
    r = hv.Renderer(256, 256, 16, 2 * B, stream=stream.cuda_stream)
    try:
        r.set_params(256, 256, spatial=w["spatial"], z=w["z"], T=T, stride=S, fs=w["fs"],
                     band=(klo, khi), moments=w["moments"], tuned=1)
        wf = r.window_floats()
        nwin = (2 * B - T) // S + 1
        out = torch.zeros((nwin + 2) * wf, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        got = 0
        for _ in range(2):
            assert r.push(pool_dev, async_=True) == hv.HV_OK
            while (k := r.render(out[got * wf:])) > 0:
                got += k
        r.synchronize()
        host = out.cpu().numpy()
    finally:
        r.close()
    assert got == nwin
    p = oracle_params(spatial=w["spatial"], z_m=w["z"], T=T, stride=S, fs_hz=w["fs"],
                      band_lo_bin=klo, band_hi_bin=khi, moments=w["moments"], H=256, W=256)
    img = images_from(host, got, p)
    period = w["pool"] // S
    ref = O.render(np.concatenate([pool, pool[:T - S]]), p)
    assert ref.shape[0] == period
    for i in range(got):
        check_images(img[i:i + 1], ref[i % period:i % period + 1])


@pytest.mark.slow
def test_window_per_cta_stft_paper_asp_shape():
    """The paper's ASP + STFT 512/512 shape at 256 x 256 (12-bit, ASP z = 0.30 m,
    M0/M1/M2 over 1-35 kHz at 71.4 kHz) through the fused transform and the
    window-per-CTA STFT: two windows, every pixel."""
    sc = synth.build(synth.scene_stream_fresnel())
    fr = synth.frames(sc, 0, 1024)
    klo, khi = O.band_bins_from_hz(1000.0, 35000.0, 71400.0, 512)
    p = oracle_params(spatial="asp", z_m=0.30, T=512, stride=512, fs_hz=71400.0,
                      band_lo_bin=klo, band_hi_bin=khi, moments=("M0", "M1", "M2"), H=256, W=256)
    img, _ = gpu_render(fr, p, extra=dict(spatial_kernel="fused", stft_kernel="window"))
    check_images(img, O.render(fr, p))
