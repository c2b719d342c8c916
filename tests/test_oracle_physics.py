"""End-to-end sanity of the oracle on the seeded synthetic scene.

The scene's Doppler disk (3 kHz, inside the 4..28 bin band at fs = 20 kHz,
T = 64) must render bright in M0 exactly where off-axis geometry puts it: the
+1 order is displaced by z * lam / (4 dx) (carrier at 1/(4 dx)), wrapping
modulo the frame, and it is in focus only at the object distance.
"""
import numpy as np
import pytest

from oracle import hv_oracle as O
from paper_2508_03911_gb300 import synth

N = 256


@pytest.fixture(scope="module")
def tiny_frames():
    sc = synth.build(synth.scene_tiny_asp_stft())
    return sc, synth.frames(sc, 0, 64)


def _params(z):
    return dict(spatial="asp", z_m=z, lambda_m=852e-9, pitch_x_m=20e-6, pitch_y_m=20e-6,
                temporal="stft", T=64, stride=64, fs_hz=20000.0, band_lo_bin=4,
                band_hi_bin=28, moments=("M0",))


def _disk_contrast(M0, sc, z):
    shift_px = z * sc.lam / (4 * sc.pitch) / sc.pitch
    c = (N / 2 + sc.doppler_center_px()[0] - shift_px) % N
    yy, xx = np.mgrid[0:N, 0:N]
    dy = np.minimum(np.abs(yy - c), N - np.abs(yy - c))
    dx = np.minimum(np.abs(xx - c), N - np.abs(xx - c))
    inside = dy ** 2 + dx ** 2 <= (N / 16) ** 2
    return M0[inside].mean() / np.median(M0[~inside])


def test_doppler_disk_renders_at_predicted_location(tiny_frames):
    sc, fr = tiny_frames
    assert fr.dtype == np.uint8 and fr.shape == (64, N, N)
    M0 = O.render(fr, _params(0.30))[0, 0]
    assert _disk_contrast(M0, sc, 0.30) >= 10.0


def test_focus_is_sharpest_at_object_distance(tiny_frames):
    sc, fr = tiny_frames
    c_focus = _disk_contrast(O.render(fr, _params(0.30))[0, 0], sc, 0.30)
    for z in (0.15, 0.45):
        assert _disk_contrast(O.render(fr, _params(z))[0, 0], sc, z) < 0.5 * c_focus


def test_generator_is_chunk_reproducible():
    sc = synth.build(synth.scene_tiny_asp_stft(N=32, n_static=16, n_doppler=4))
    a = synth.frames(sc, 0, 6)
    b = np.concatenate([synth.frames(sc, 0, 2), synth.frames(sc, 2, 4)])
    assert np.array_equal(a, b)
    assert abs(a.mean() / 255.0 - 0.30) < 0.05
