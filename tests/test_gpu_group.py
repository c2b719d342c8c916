"""Groups of handles stepped together (hv_render_group): uneven frame sizes,
window lengths, transforms and temporal analyses in one batch, with and
without CUDA-graph capture, against the FP64 oracle on every member's stream."""
import numpy as np
import pytest

from oracle import hv_oracle as O
from paper_2508_03911_gb300 import hv, synth
from tests._util import oracle_params, rel_l2, to_device, to_hv

pytestmark = pytest.mark.gpu

IMAGE_TOL = 1e-4


def _members():
    """(oracle params, bits, frames per batch, frames) of four uneven members."""
    out = []
    p = oracle_params(spatial="fresnel", z_m=0.25, T=32, stride=32, fs_hz=71400.0, band_lo_bin=1,
                      band_hi_bin=15, moments=("M0", "M1", "M2"), H=64, W=64)
    out.append((p, 16, 32, synth.random_frames(32 * 4, 64, 64, 12, seed=11)))
    p = oracle_params(spatial="asp", z_m=0.3, T=16, stride=8, fs_hz=20000.0, band_lo_bin=1,
                      band_hi_bin=8, moments=("M0", "M2N"), H=32, W=64)
    out.append((p, 16, 24, synth.random_frames(24 * 4, 32, 64, 12, seed=12)))
    p = oracle_params(spatial="asp", z_m=0.3, T=64, stride=64, H=128, W=128)
    sc = synth.build(synth.scene_tiny_asp_stft(N=128))
    out.append((p, 8, 64, synth.frames(sc, 0, 64 * 4)))
    p = oracle_params(spatial="fresnel", z_m=0.3, temporal="pca", T=32, stride=32, pca_lo=2, pca_hi=3,
                      H=64, W=64)
    out.append((p, 16, 32, synth.frames(synth.build(synth.scene_pca(N=64)), 0, 32 * 4)))
    return out


def _n_img(p):
    return len(p["moments"]) if p["temporal"] == "stft" else 1


@pytest.mark.parametrize("use_graph", [True, False])
def test_group_matches_oracle_and_per_handle_calls(use_graph):
    import torch
    members = _members()
    rs = []
    try:
        for p, bits, per_batch, fr in members:
            r = hv.Renderer(p["W"], p["H"], bits, 3 * per_batch)
            hv.hv_set_params(r.h, to_hv(p, tuned=1))
            rs.append(r)
        g = hv.hv_group_open([r.h for r in rs], use_graph=use_graph)
        try:
            dev = [to_device(fr) for _, _, _, fr in members]
            wf = [r.window_floats() for r in rs]
            outs = [torch.zeros(8 * w, dtype=torch.float32, device="cuda") for w in wf]
            got = [[] for _ in rs]
            for step in range(3):
                frames = [d[step * m[2]:(step + 1) * m[2]] for d, m in zip(dev, members)]
                nw = hv.hv_render_group(g, frames, outs)
                torch.cuda.synchronize()
                for i, k in enumerate(nw):
                    got[i].append(outs[i][: k * wf[i]].cpu().numpy().copy())
            st = hv.hv_group_get_stats(g)
            assert st["steps"] == 3
            if use_graph:
                assert st["graph_launches"] == 3
                assert st["graph_instantiations"] + st["graph_updates"] == 3
                assert st["graph_updates"] >= 1  # steps 2 and 3 have the same shape
            else:
                assert st["graph_launches"] == 0
            assert st["kernel_launches"] > 0
        finally:
            hv.hv_group_close(g)
        # the last batch through the per-handle calls: ordered after the group's work
        for i, (p, bits, per_batch, fr) in enumerate(members):
            assert rs[i].push(dev[i][3 * per_batch:]) == hv.HV_OK
            k = rs[i].render(outs[i])
            torch.cuda.synchronize()
            got[i].append(outs[i][: k * wf[i]].cpu().numpy().copy())
        for i, (p, bits, per_batch, fr) in enumerate(members):
            img = np.concatenate(got[i]).reshape(-1, _n_img(p), p["H"], p["W"])
            ref = O.render(fr, p)
            assert img.shape == ref.shape, (i, img.shape, ref.shape)
            for w in range(ref.shape[0]):
                for q in range(ref.shape[1]):
                    e = rel_l2(img[w, q], ref[w, q])
                    assert e <= IMAGE_TOL, (i, w, q, e)
    finally:
        for r in rs:
            r.close()


def test_group_rejects_before_issuing_work():
    import torch
    p = oracle_params(spatial="asp", T=16, stride=16, H=32, W=32, band_lo_bin=1, band_hi_bin=7)
    pp = oracle_params(spatial="asp", temporal="pca", T=128, stride=128, pca_lo=1, pca_hi=4, H=32, W=32)
    a = hv.Renderer(32, 32, 16, 32)
    b = hv.Renderer(32, 32, 16, 256)
    try:
        hv.hv_set_params(a.h, to_hv(p))
        hv.hv_set_params(b.h, to_hv(p))
        fr = to_device(synth.random_frames(40, 32, 32, 12, seed=3))
        out = [torch.zeros(4 * a.window_floats(), device="cuda") for _ in range(2)]
        g = hv.hv_group_open([a.h, b.h])
        try:
            with pytest.raises(hv.HvError) as ei:  # 40 frames exceed member 0's 32-frame queue
                hv.hv_render_group(g, [fr, fr[:16]], out)
            assert ei.value.status == hv.HV_ERR_QUEUE_FULL
            assert a.stats()["frames_pushed"] == 0 and b.stats()["frames_pushed"] == 0
            hv.hv_profile_enable(b.h, True)
            with pytest.raises(hv.HvError) as ei:
                hv.hv_render_group(g, [fr[:16], fr[:16]], out)
            assert ei.value.status == hv.HV_ERR_STATE
            hv.hv_profile_enable(b.h, False)
            hv.hv_set_params(b.h, to_hv(pp))
            with pytest.raises(hv.HvError) as ei:
                hv.hv_render_group(g, [fr[:16], fr[:16]], out)
            assert ei.value.status == hv.HV_ERR_UNSUPPORTED
            assert a.stats()["frames_pushed"] == 0
            assert hv.hv_group_get_stats(g)["steps"] == 0
        finally:
            hv.hv_group_close(g)
        with pytest.raises(hv.HvError):
            hv.hv_group_open([a.h, a.h])
    finally:
        a.close()
        b.close()


def test_group_at_the_batched_workload_shapes():
    """Members of the batched uneven-stream workload's sizes through the graph path
    with the autotuned kernels: 1024x1024 ASP and Fresnel members, a 256x256 member
    with T = 512, a 512x512 member with T = 128 and two 128x128 members; 12-bit
    frames, S = T, M0/M1/M2 over 1-35 kHz at 71.4 kHz. Two batches of one window per
    member (the second replays the updated graph), each against the FP64 oracle.
    (The workload's 1024x1024 ASP member has T = 128; T = 32 here keeps the FP64
    oracle's work to seconds.)"""
    import math

    import torch
    shapes = [(128, 32, "fresnel"), (128, 128, "asp"), (256, 512, "asp"), (512, 128, "asp"),
              (1024, 32, "asp"), (1024, 32, "fresnel")]
    members = []
    for i, (N, T, sp) in enumerate(shapes):
        band = (math.ceil(1000.0 * T / 71400.0 - 1e-12), math.floor(35000.0 * T / 71400.0 + 1e-12))
        p = oracle_params(spatial=sp, z_m=0.25 if sp == "fresnel" else 0.30, T=T, stride=T,
                          fs_hz=71400.0, band_lo_bin=band[0], band_hi_bin=band[1],
                          moments=("M0", "M1", "M2"), H=N, W=N)
        members.append((p, synth.random_frames(2 * T, N, N, 12, seed=1003 + i)))
    rs = []
    try:
        for p, fr in members:
            r = hv.Renderer(p["W"], p["H"], 16, 2 * p["T"])
            hv.hv_set_params(r.h, to_hv(p, tuned=1))
            rs.append(r)
        g = hv.hv_group_open([r.h for r in rs], use_graph=True)
        try:
            dev = [to_device(fr) for _, fr in members]
            outs = [torch.zeros(3 * r.window_floats(), dtype=torch.float32, device="cuda") for r in rs]
            got = [[] for _ in rs]
            for step in range(2):
                frames = [d[step * p["T"]:(step + 1) * p["T"]] for d, (p, _) in zip(dev, members)]
                nw = hv.hv_render_group(g, frames, outs)
                assert nw == [1] * len(rs), nw
                torch.cuda.synchronize()
                for i in range(len(rs)):
                    got[i].append(outs[i][: rs[i].window_floats()].cpu().numpy().copy())
            st = hv.hv_group_get_stats(g)
            assert st["graph_launches"] == 2 and st["graph_updates"] >= 1
        finally:
            hv.hv_group_close(g)
        for i, (p, fr) in enumerate(members):
            img = np.stack(got[i]).reshape(2, 3, p["H"], p["W"])
            for w in range(2):
                ref = O.render(fr[w * p["T"]:(w + 1) * p["T"]], p)[0]
                for q in range(3):
                    e = rel_l2(img[w, q], ref[q])
                    assert e <= IMAGE_TOL, (shapes[i], w, q, e)
    finally:
        for r in rs:
            r.close()
