"""GPU parity of the autofocus path: the plain z-sweep (ASP of the mean-removed
hologram, Tamura coefficient per distance) and the network input (binned
log-magnitude spectrum), against the FP64 oracle."""
import numpy as np
import pytest

from oracle import af_oracle as A
from paper_2508_03911_gb300 import hv, synth
from tests._util import oracle_params, to_device, to_hv

pytestmark = pytest.mark.gpu

# Tamura from float32 fields (relative L2 error ~1e-6): the coefficient to 1e-4.
TAMURA_TOL = 1e-4
STEP = (A.Z1 - A.Z0) / (A.NZ - 1)


def _renderer(W, H, bits, n):
    r = hv.Renderer(W, H, bits, max(n, 1))
    p = oracle_params(spatial="asp", z_m=0.3, T=16, stride=16, H=H, W=W, band_lo_bin=1, band_hi_bin=7)
    hv.hv_set_params(r.h, to_hv(p))
    return r


def gpu_sweep(frames, zs):
    import torch
    n, H, W = frames.shape
    r = _renderer(W, H, 8 if frames.dtype == np.uint8 else 16, n)
    try:
        out = torch.zeros((n, len(zs)), dtype=torch.float32, device="cuda")
        hv.hv_focus_sweep(r.h, to_device(frames), zs, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        r.close()


def test_sweep_matches_oracle_and_finds_the_focus():
    fr, zt = synth.autofocus_set(4, N=256, seed=1005)
    zs = A.z_grid()
    got = gpu_sweep(fr, zs)
    for i in range(len(fr)):
        ref = A.focus_sweep(fr[i], 852e-9, 20e-6, 20e-6)
        err = np.max(np.abs(got[i] - ref) / ref)
        assert err <= TAMURA_TOL, (i, err)
        top2 = np.sort(ref)[-2:]
        if (top2[1] - top2[0]) / top2[1] > 10 * TAMURA_TOL:
            assert int(np.argmax(got[i])) == int(np.argmax(ref))
        assert abs(zs[int(np.argmax(got[i]))] - zt[i]) <= STEP, (i, zt[i])


@pytest.mark.parametrize("H,W,bits", [(128, 128, 16), (64, 128, 8), (128, 64, 16)])
def test_sweep_other_sizes(H, W, bits):
    fr = synth.random_frames(3, H, W, bits if bits == 8 else 12, seed=H + W)
    zs = [0.1, 0.23, 0.4, 0.6]
    got = gpu_sweep(fr, zs)
    for i in range(len(fr)):
        ref = A.focus_sweep(fr[i], 852e-9, 20e-6, 20e-6, zs)
        assert np.max(np.abs(got[i] - ref) / ref) <= TAMURA_TOL


def gpu_features(frames):
    import torch
    n, H, W = frames.shape
    r = _renderer(W, H, 8 if frames.dtype == np.uint8 else 16, n)
    try:
        out = torch.zeros((n, H // 2, W // 2), dtype=torch.bfloat16, device="cuda")
        hv.hv_af_features(r.h, to_device(frames), out)
        torch.cuda.synchronize()
        return out.float().cpu().numpy()
    finally:
        r.close()


@pytest.mark.parametrize("H,W,bits", [(256, 256, 16), (64, 128, 8), (128, 64, 16), (64, 512, 8)])
def test_features_match_oracle(H, W, bits):
    """Widths up to 256 form the binned cells in the row pass's epilogue (lanes
    pair bins and rows); 512 stores the spectra and bins them in a second kernel."""
    if H == 256:
        fr, _ = synth.autofocus_set(5, N=256, seed=1007)
    else:
        fr = synth.random_frames(5, H, W, 8, seed=9)
    got = gpu_features(fr)
    for i in range(len(fr)):
        ref = A.features(fr[i])
        # bfloat16 keeps 8 significant bits: one unit in the last place is |x| 2^-7
        # at most; the float32 spectrum adds ~1e-6
        np.testing.assert_array_less(np.abs(got[i] - ref), np.abs(ref) * 2.0 ** -7 + 1e-4)
