"""Helpers shared by the tests: oracle-parameter translation and error metrics."""
import numpy as np

from paper_2508_03911_gb300 import hv


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=np.complex128 if np.iscomplexobj(b) else np.float64)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def oracle_params(**kw) -> dict:
    p = dict(spatial="asp", z_m=0.3, lambda_m=852e-9, pitch_x_m=20e-6, pitch_y_m=20e-6,
             fftshift=1, temporal="stft", T=64, stride=64, fs_hz=20000.0, band_lo_bin=4,
             band_hi_bin=28, moments=("M0",), pca_lo=2, pca_hi=64)
    p.update(kw)
    return p


def to_hv(p: dict, **extra) -> "hv.hv_params":
    """The C-ABI settings block equivalent to an oracle parameter dict."""
    H, W = p["H"], p["W"]
    return hv.make_params(W, H, spatial=p["spatial"], z=p["z_m"], lam=p["lambda_m"],
                          pitch=p["pitch_x_m"], pitch_y=p["pitch_y_m"], fftshift=p["fftshift"],
                          temporal=p["temporal"], T=p["T"], stride=p["stride"], fs=p["fs_hz"],
                          band=(p["band_lo_bin"], p["band_hi_bin"]), moments=p["moments"],
                          pca=(p["pca_lo"], p["pca_hi"]), highpass=p.get("highpass", 0.0),
                          **extra)


def images_from(out: np.ndarray, n_win: int, p: dict) -> np.ndarray:
    """Reshape a rendered buffer into (n_win, n_img, H, W) (complex for TEMPORAL_NONE)."""
    H, W = p["H"], p["W"]
    if p["temporal"] == "none":
        v = out[: n_win * H * W * 2].reshape(n_win, H, W, 2)
        return (v[..., 0] + 1j * v[..., 1])[:, None]
    n_img = len(p["moments"]) if p["temporal"] == "stft" else 1
    return out[: n_win * n_img * H * W].reshape(n_win, n_img, H, W)


# Device copies handed to the library: its copies run on the handle's own stream,
# so each tensor must be complete before they run and must outlive them. Kept
# until the end of the test (conftest releases them after a device synchronise).
_KEEP = []


def to_device(frames: np.ndarray):
    """Raw frames as a CUDA tensor with the same bytes (uint16 travels as int16),
    complete on the device when this returns and kept alive for the test."""
    import torch
    a = frames.view(np.int16) if frames.dtype == np.uint16 else frames
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    _KEEP.append(t)
    return t


def release_device_buffers():
    import sys
    if _KEEP and "torch" in sys.modules:
        sys.modules["torch"].cuda.synchronize()
    _KEEP.clear()
