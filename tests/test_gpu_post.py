"""GPU parity of post-processing (periodic convolution, re-normalisation, moving
average over windows) against the FP64 oracle, across several renders so that
the accumulation history crosses calls."""
import numpy as np
import pytest

from oracle import hv_oracle as O
from paper_2508_03911_gb300 import hv, synth
from tests._util import oracle_params, rel_l2, to_device, to_hv

pytestmark = pytest.mark.gpu
IMAGE_TOL = 1e-4


def gpu_stream(frames, p, post, packets, post_at=0, **extra):
    """Render frames pushed in `packets`; post-processing set before packet post_at."""
    import torch
    n, H, W = frames.shape
    r = hv.Renderer(W, H, 16, n)
    try:
        hv.hv_set_params(r.h, to_hv(p, **extra))
        wf = r.window_floats()
        out = torch.zeros(n * wf, dtype=torch.float32, device="cuda")
        nw, a = 0, 0
        for i, k in enumerate(packets):
            if i == post_at and post is not None:
                hv.hv_set_postprocess(r.h, **post)
            assert r.push(to_device(frames[a:a + k])) == hv.HV_OK
            a += k
            while True:
                got = r.render(out[nw * wf:])
                nw += got
                if got == 0:
                    break
        torch.cuda.synchronize()
        n_img = len(p["moments"]) if p["temporal"] == "stft" else 1
        return out.cpu().numpy()[: nw * wf].reshape(nw, n_img, H, W)
    finally:
        r.close()


def check(img, ref):
    assert img.shape == ref.shape, (img.shape, ref.shape)
    for w in range(ref.shape[0]):
        for q in range(ref.shape[1]):
            e = rel_l2(img[w, q], ref[w, q])
            assert e <= IMAGE_TOL, (w, q, e)


def oracle_post(frames, p, kern, renorm, A, first=0):
    ref = O.render(frames, p)
    out = ref.copy()
    for q in range(ref.shape[1]):
        out[first:, q] = O.postprocess(ref[first:, q], kern, renorm, A)
    return out


def test_gaussian_renorm_accumulate_stft():
    H, W, T, S = 32, 64, 16, 8
    fr = synth.random_frames(T + 11 * S + 3, H, W, 12, seed=21)
    p = oracle_params(spatial="fresnel", z_m=0.25, T=T, stride=S, fs_hz=71400.0, band_lo_bin=1,
                      band_hi_bin=7, moments=("M0", "M1", "M2N"), H=H, W=W)
    post = dict(kernel_size=5, sigma=1.2, renormalize=True, accumulate=3)
    img = gpu_stream(fr, p, post, [T + 3 * S, 2 * S, 5, 4 * S + 3, 2 * S - 5 + 3])
    check(img, oracle_post(fr, p, O.gaussian_kernel(5, 1.2), True, 3))


@pytest.mark.parametrize("T,S,form", [(16, 16, dict(tuned=1)), (16, 16, dict(stft_kernel="window_wide")),
                                      (16, 16, dict(stft_kernel="window_pipelined")),
                                      (512, 512, dict(stft_kernel="window_tma")),
                                      (512, 512, dict(stft_kernel="window_tma_pipelined")),
                                      (16, 4, dict(tuned=1)), (16, 4, dict(tuned=0))])
def test_renorm_accumulate_fused_into_the_stft(T, S, form):
    """Without a convolution the STFT epilogue writes the image ring and adds each
    image's sum itself (window-per-CTA kernels for S >= T, the walking kernel for
    S < T, one launch per window in the plain form); every moment kind, history
    across renders and ring wrap-around."""
    H, W = 32, 64
    fr = synth.random_frames(T + 13 * S + 5, H, W, 12, seed=T + S)
    p = oracle_params(spatial="asp", T=T, stride=S, fs_hz=20000.0, band_lo_bin=1, band_hi_bin=6,
                      moments=("M0", "M1", "M2", "M1N", "M2N"), H=H, W=W)
    packets = [T + 2 * S, 3 * S + 1, 4 * S, 4 * S - 1 + 5]
    img = gpu_stream(fr, p, dict(renormalize=True, accumulate=4), packets, **form)
    check(img, oracle_post(fr, p, None, True, 4))


def test_user_kernel_pca():
    H = W = 64
    fr = synth.frames(synth.build(synth.scene_pca(N=64)), 0, 32 * 5)
    p = oracle_params(spatial="fresnel", z_m=0.3, temporal="pca", T=32, stride=32, pca_lo=2, pca_hi=3,
                      H=H, W=W)
    k = np.array([[0.0, 0.1, 0.0], [0.2, 0.5, 0.05], [0.0, 0.1, 0.05]])
    img = gpu_stream(fr, p, dict(kernel=k), [64, 32, 64])
    check(img, oracle_post(fr, p, k, False, 1))


@pytest.mark.parametrize("A", [2, 7])
def test_accumulate_only_and_history_restart(A):
    H, W, T, S = 16, 32, 8, 4
    fr = synth.random_frames(T + 14 * S, H, W, 12, seed=A)
    p = oracle_params(spatial="asp", T=T, stride=S, fs_hz=20000.0, band_lo_bin=1, band_hi_bin=3,
                      moments=("M0",), H=H, W=W)
    # post-processing set after the first packet: windows rendered before stay raw,
    # the history starts with the first window rendered after
    packets = [T + 2 * S, 3 * S, S, 8 * S]
    img = gpu_stream(fr, p, dict(accumulate=A), packets, post_at=1)
    first = len(O.window_starts(T + 2 * S, T, S))
    check(img, oracle_post(fr, p, None, False, A, first=first))


def test_invalid_post_settings_and_temporal_none():
    H = W = 32
    r = hv.Renderer(W, H, 16, 8)
    try:
        p = oracle_params(spatial="asp", temporal="none", T=1, stride=1, H=H, W=W)
        hv.hv_set_params(r.h, to_hv(p))
        for bad in [dict(kernel_size=4, sigma=1.0), dict(accumulate=0), dict(accumulate=65),
                    dict(kernel_size=3, sigma=0.0), dict(kernel_size=33, sigma=1.0)]:
            with pytest.raises(hv.HvError) as ei:
                hv.hv_set_postprocess(r.h, **bad)
            assert ei.value.status == hv.HV_ERR_ARG
        hv.hv_set_postprocess(r.h, accumulate=2)
        import torch
        out = torch.zeros(64 * H * W, device="cuda")
        assert r.push(to_device(synth.random_frames(2, H, W, 12, seed=1))) == hv.HV_OK
        with pytest.raises(hv.HvError) as ei:
            r.render(out)
        assert ei.value.status == hv.HV_ERR_UNSUPPORTED
    finally:
        r.close()
