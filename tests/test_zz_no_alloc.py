"""hv_spatial_static: the spatial transform with no allocation at all.

Callers that may not allocate device memory where they run (allocator
callbacks, plugins in a framework that owns all memory, allocator-free
real-time loops) get this entry point; its scratch is a fixed file-scope
device array. Here it must give the same complex fields as the handle path
(HV_TEMPORAL_NONE rendering), within the field tolerance of the parity tests,
on consecutive calls that reuse the shared scratch, and refuse sizes beyond
its stated maximum. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2508_03911_gb300 import hv, synth
from tests._util import oracle_params, rel_l2, to_device, to_hv

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
MAX_PIXELS = 786432


def _entry():
    f = hv.lib().hv_spatial_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                  ctypes.POINTER(hv.hv_params), ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _handle_fields(frames, p):
    """Complex fields from the existing entry points (hv_render, TEMPORAL_NONE)."""
    import torch
    n, H, W = frames.shape
    bits = 8 if frames.dtype == np.uint8 else 16
    r = hv.Renderer(W, H, bits, n)
    try:
        hv.hv_set_params(r.h, to_hv(p))
        out = torch.zeros(n * H * W * 2, dtype=torch.float32, device="cuda")
        assert r.push(to_device(frames)) == hv.HV_OK
        assert r.render(out) == n
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        r.close()


def _static_fields(frames, p, stream=None):
    import torch
    n, H, W = frames.shape
    bits = 8 if frames.dtype == np.uint8 else 16
    dev = to_device(frames)
    out = torch.full((n * H * W * 2,), float("nan"), dtype=torch.float32, device="cuda")
    prm = to_hv(p)
    st = _entry()(dev.data_ptr(), bits, n, ctypes.byref(prm), out.data_ptr(), stream)
    assert st == hv.HV_OK, st
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _cplx(v, n, H, W):
    v = v.reshape(n, H, W, 2)
    return v[..., 0] + 1j * v[..., 1]


CASES = [
    # (frames, H, W, bits, spatial, z, extra settings)
    (4, 256, 256, 16, "asp", 0.30, {}),
    (3, 512, 512, 16, "fresnel", 0.25, {}),   # exactly the maximum pixel count
    (5, 64, 128, 8, "fresnel", -0.2, {}),
    (2, 128, 64, 8, "asp", 0.45, {}),
    (3, 128, 128, 16, "fresnel", 0.25, {"fftshift": 0}),
    (2, 64, 64, 16, "asp", 0.30, {"highpass": 0.05}),
]


def test_static_matches_handle_path_on_consecutive_calls():
    import torch
    torch.cuda.synchronize()
    for i, (n, H, W, bits, spatial, z, extra) in enumerate(CASES):
        fr = synth.random_frames(n, H, W, 12 if bits == 16 else 8, seed=900 + i)
        if bits == 16:
            fr = fr.astype(np.uint16)
        p = oracle_params(spatial=spatial, z_m=z, temporal="none", T=1, stride=1, H=H, W=W,
                          pitch_y_m=17e-6, **extra)
        ref = _cplx(_handle_fields(fr, p), n, H, W)
        for call in range(2):  # two calls in a row share (and reuse) the scratch
            got = _cplx(_static_fields(fr, p), n, H, W)
            assert np.all(np.isfinite(got))
            for f in range(n):
                e = rel_l2(got[f], ref[f])
                assert e <= FIELD_TOL, (i, call, f, e)


def test_static_on_a_torch_stream_and_limits():
    import torch
    n, H, W = 2, 64, 64
    fr = synth.random_frames(n, H, W, 12, seed=5).astype(np.uint16)
    p = oracle_params(spatial="asp", z_m=0.3, temporal="none", T=1, stride=1, H=H, W=W)
    ref = _cplx(_handle_fields(fr, p), n, H, W)
    s = torch.cuda.Stream()
    got = _cplx(_static_fields(fr, p, stream=s.cuda_stream), n, H, W)
    assert rel_l2(got, ref) <= FIELD_TOL
    f = _entry()
    dev = to_device(fr)
    out = torch.zeros(16, device="cuda")
    prm = to_hv(p)
    # beyond the stated maximum: 13 frames of 256 x 256, and 1024-wide frames
    big = to_hv(oracle_params(spatial="asp", temporal="none", T=1, stride=1, H=256, W=256))
    assert f(dev.data_ptr(), 16, MAX_PIXELS // (256 * 256) + 1, ctypes.byref(big), out.data_ptr(),
             None) == hv.HV_ERR_ARG
    wide = to_hv(oracle_params(spatial="asp", temporal="none", T=1, stride=1, H=16, W=1024))
    assert f(dev.data_ptr(), 16, 1, ctypes.byref(wide), out.data_ptr(), None) == hv.HV_ERR_ARG
    assert f(None, 16, 1, ctypes.byref(prm), out.data_ptr(), None) == hv.HV_ERR_ARG
    assert f(dev.data_ptr(), 12, 1, ctypes.byref(prm), out.data_ptr(), None) == hv.HV_ERR_ARG
    assert f(dev.data_ptr(), 16, 0, ctypes.byref(prm), out.data_ptr(), None) == hv.HV_ERR_ARG


def test_static_against_the_oracle_and_the_identity():
    """Against the FP64 oracle directly (not only the handle path), and the
    transform 'none', whose output is the converted frame exactly."""
    from oracle import hv_oracle as O
    n, H, W = 2, 128, 128
    fr = synth.random_frames(n, H, W, 12, seed=77).astype(np.uint16)
    for spatial, extra in (("asp", {}), ("fresnel", {"fftshift": 0}), ("asp", {"highpass": 0.04})):
        p = oracle_params(spatial=spatial, z_m=0.27, temporal="none", T=1, stride=1, H=H, W=W, **extra)
        for call in range(2):
            got = _cplx(_static_fields(fr, p), n, H, W)
            for f in range(n):
                ref = O.spatial(O.convert(fr[f]), p)
                assert rel_l2(got[f], ref) <= FIELD_TOL, (spatial, extra, call, f)
    p = oracle_params(spatial="none", temporal="none", T=1, stride=1, H=H, W=W)
    for call in range(2):
        got = _cplx(_static_fields(fr, p), n, H, W)
        assert np.array_equal(got.real, fr.astype(np.float64))
        assert np.all(got.imag == 0)


def test_static_refuses_misaligned_pointers_and_highpass_without_asp():
    import torch
    f = _entry()
    fr = synth.random_frames(1, 64, 64, 12, seed=3).astype(np.uint16)
    dev = to_device(fr)
    out = torch.zeros(64 * 64 * 2 + 4, dtype=torch.float32, device="cuda")
    p = to_hv(oracle_params(spatial="asp", temporal="none", T=1, stride=1, H=64, W=64))
    # out 4 bytes past an 8-byte boundary; 16-bit frames at an odd address
    assert f(dev.data_ptr(), 16, 1, ctypes.byref(p), out.data_ptr() + 4, None) == hv.HV_ERR_ARG
    raw = torch.zeros(64 * 64 * 2 + 2, dtype=torch.uint8, device="cuda")
    assert f(raw.data_ptr() + 1, 16, 1, ctypes.byref(p), out.data_ptr(), None) == hv.HV_ERR_ARG
    fres = to_hv(oracle_params(spatial="fresnel", temporal="none", T=1, stride=1, H=64, W=64,
                               highpass=0.05))
    assert f(dev.data_ptr(), 16, 1, ctypes.byref(fres), out.data_ptr(), None) == hv.HV_ERR_ARG
    # a refused call leaves no CUDA error behind, and a valid call still works
    torch.cuda.synchronize()
    assert f(dev.data_ptr(), 16, 1, ctypes.byref(p), out.data_ptr(), None) == hv.HV_OK
    torch.cuda.synchronize()
    assert torch.isfinite(out[: 64 * 64 * 2]).all()
