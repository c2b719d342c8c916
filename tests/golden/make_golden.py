"""Writes tests/golden/oracle_small.json: sampled oracle outputs on small seeded
cases, used as a regression fixture for the oracle itself.

Calls only oracle/ (and the seeded input generator).  Run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hv_oracle as O  # noqa: E402
from paper_2508_03911_gb300 import synth  # noqa: E402

CASES = {
    # ASP + sliding STFT on uint16 frames, all five moment outputs
    "asp_stft_u16_32x32_T16_S4": dict(
        frames=dict(n=40, H=32, W=32, bits=12, seed=7),
        params=dict(spatial="asp", z_m=0.2, lambda_m=852e-9, pitch_x_m=20e-6, pitch_y_m=20e-6,
                    temporal="stft", T=16, stride=4, fs_hz=20000.0, band_lo_bin=2,
                    band_hi_bin=6, moments=("M0", "M1", "M2", "M1N", "M2N"))),
    # Fresnel (fftshift) + STFT on uint8 frames
    "fresnel_stft_u8_16x32_T8_S8": dict(
        frames=dict(n=16, H=16, W=32, bits=8, seed=8),
        params=dict(spatial="fresnel", z_m=0.25, lambda_m=852e-9, pitch_x_m=20e-6,
                    pitch_y_m=20e-6, fftshift=1, temporal="stft", T=8, stride=8,
                    fs_hz=71400.0, band_lo_bin=1, band_hi_bin=3, moments=("M0", "M2"))),
    # ASP + PCA energy over eigenvectors 2..6
    "asp_pca_u16_16x16_T12": dict(
        frames=dict(n=12, H=16, W=16, bits=12, seed=9),
        params=dict(spatial="asp", z_m=0.4, lambda_m=852e-9, pitch_x_m=20e-6, pitch_y_m=20e-6,
                    temporal="pca", T=12, stride=12, pca_lo=2, pca_hi=6)),
}


def sample(img):
    flat = img.ravel()
    idx = np.linspace(0, flat.size - 1, 16).astype(int)
    return {"shape": list(img.shape), "sum": float(flat.sum()),
            "idx": idx.tolist(), "val": [float(v) for v in flat[idx]]}


def main():
    out = {"_note": "oracle regression fixture; values written by make_golden.py from oracle/ only"}
    for name, c in CASES.items():
        f = c["frames"]
        fr = synth.random_frames(f["n"], f["H"], f["W"], f["bits"], f["seed"])
        img = O.render(fr, c["params"])
        out[name] = dict(c, result=sample(img))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print("wrote", path)


if __name__ == "__main__":
    main()
