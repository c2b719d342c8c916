"""GPU parity of the PCA temporal analysis (covariance, FP64 Jacobi, projection
energy) against the FP64 oracle.

Bars: the energy image E within relative L2 1e-4; eigenvalues within 1e-6 of
the largest eigenvalue (absolute; the covariance is accumulated from float32
fields, whose own error is ~3e-7 relative).
"""
import numpy as np
import pytest

from oracle import hv_oracle as O
from paper_2508_03911_gb300 import hv, synth
from tests._util import oracle_params, rel_l2, to_device, to_hv

pytestmark = pytest.mark.gpu

IMAGE_TOL = 1e-4
LAM_TOL = 1e-6


def gpu_pca(frames, p):
    import torch
    n, H, W = frames.shape
    bits = 8 if frames.dtype == np.uint8 else 16
    r = hv.Renderer(W, H, bits, n)
    try:
        hv.hv_set_params(r.h, to_hv(p))
        wf = r.window_floats()
        assert wf == H * W
        out = torch.zeros(n * wf, dtype=torch.float32, device="cuda")
        assert r.push(to_device(frames)) == hv.HV_OK
        nw = r.render(out)
        torch.cuda.synchronize()
        lam = hv.hv_pca_eigenvalues(r.h, p["T"])
        return out.cpu().numpy()[: nw * wf].reshape(nw, H, W), lam
    finally:
        r.close()


def oracle_windows(frames, p):
    starts = O.window_starts(frames.shape[0], p["T"], p["stride"])
    res = []
    for s in starts:
        U = np.stack([O.spatial(O.convert(f), p) for f in frames[s:s + p["T"]]])
        res.append(O.pca(U, p["pca_lo"], p["pca_hi"]))
    return res


@pytest.mark.parametrize("H,W,T,S,lohi,spatial", [
    (64, 64, 32, 32, (2, 8), "fresnel"),      # the paper's PCA 32/32 shape, small frame
    (32, 64, 64, 16, (1, 5), "asp"),          # overlapping windows
    (64, 32, 32, 48, (3, 32), "none"),        # stride beyond the window, band to the end
    (128, 128, 256, 256, (2, 64), "asp"),     # the PCA workload's window shape, smaller frame
])
def test_pca_parity(H, W, T, S, lohi, spatial):
    n = T + S + 7
    fr = synth.random_frames(n, H, W, 12, seed=H + T + S)
    p = oracle_params(spatial=spatial, z_m=0.4, temporal="pca", T=T, stride=S, pca_lo=lohi[0],
                      pca_hi=lohi[1], H=H, W=W)
    img, lam = gpu_pca(fr, p)
    ref = oracle_windows(fr, p)
    assert img.shape[0] == len(ref)
    for w, rw in enumerate(ref):
        e = rel_l2(img[w], rw["E"])
        assert e <= IMAGE_TOL, (w, e)
    lam_ref = ref[-1]["lam"]
    assert np.max(np.abs(lam - lam_ref)) <= LAM_TOL * lam_ref[0]
    assert np.all(np.diff(lam) <= 0)


def test_pca_scene_window_full_size():
    """One window of the PCA workload: 512x512 12-bit frames, ASP z = 0.40 m,
    T = 256, energy over eigenvectors 2..64 (every pixel)."""
    sc = synth.build(synth.scene_pca())
    fr = synth.frames(sc, 0, 256)
    p = oracle_params(spatial="asp", z_m=0.40, temporal="pca", T=256, stride=256, pca_lo=2,
                      pca_hi=64, H=512, W=512)
    img, lam = gpu_pca(fr, p)
    ref = oracle_windows(fr, p)[0]
    e = rel_l2(img[0], ref["E"])
    print("E rel L2", e, "lam max abs / lam1", np.max(np.abs(lam - ref["lam"])) / ref["lam"][0])
    assert e <= IMAGE_TOL
    assert np.max(np.abs(lam - ref["lam"])) <= LAM_TOL * ref["lam"][0]


def test_pca_rejects_unbuilt_precisions_and_bad_basis():
    r = hv.Renderer(64, 64, 16, 8)
    try:
        for kw in (dict(pca_lo=0), dict(pca_hi=33), dict(pca_lo=5, pca_hi=4), dict(T=16)):
            p = oracle_params(temporal="pca", T=32, stride=32, pca_lo=2, pca_hi=8, H=64, W=64)
            p.update(kw)
            with pytest.raises(hv.HvError):
                hv.hv_set_params(r.h, to_hv(p))
    finally:
        r.close()
