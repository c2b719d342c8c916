"""Independent pins of the oracle's whole-path assembly, render().

render() builds window w from frames w S .. w S + T - 1 of the stream (windows of
T frames repeated every S frames, Table IV "time stride"), transforms each frame
spatially once, and stacks the selected moments of every complete window,
window-major, in the order M0, M1, M2, M1N, M2N (Sec. III-B.1). Neither test
below reuses that indexing:

* piecewise tones: the stream is built segment by segment (segments of S frames,
  each with its own integer amplitudes of a DC term, a T/4 tone and a Nyquist
  tone, different for every pixel), so a window with S < T straddles several
  segments. Each window's spectrum is then a sum of finite geometric series,
  one per (segment part, tone), written in closed form; the moments follow. A
  wrong window start, a reused or skipped frame, a moment stacked out of order
  or a transposed pixel changes at least one image.
* commutation: the spatial transform and the temporal DFT are both linear and act
  on different axes, so the temporal DFT of a window's raw frames, propagated
  bin by bin, gives the same spectrum as render()'s spatial-then-temporal
  order. This route takes the window's frames from a slice of the stream.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import hv_oracle as O


def geometric(q: complex, n0: int, n: int) -> complex:
    """sum_{t = n0}^{n0 + n - 1} q^t in closed form."""
    if abs(q - 1.0) < 1e-15:
        return complex(n)
    return q ** n0 * (1.0 - q ** n) / (1.0 - q)


def piecewise_stream(T, S, n_seg, H, W, seed):
    """Integer frames built segment by segment: in segment j (frames j S .. j S +
    S - 1), pixel p carries a_j(p) + b_j(p) cos(2 pi (T/4) t / T) + c_j(p) (-1)^t,
    which is an integer for every t (cos(pi t / 2) is 1, 0, -1, 0). Returns the
    frames and the amplitudes."""
    rng = np.random.default_rng(seed)
    a = rng.integers(40, 90, (n_seg, H, W))
    b = rng.integers(-20, 21, (n_seg, H, W))
    c = rng.integers(-15, 16, (n_seg, H, W))
    t = np.arange(n_seg * S)
    cos4 = np.rint(np.cos(np.pi * t / 2)).astype(np.int64)
    nyq = np.where(t % 2 == 0, 1, -1)
    seg = t // S
    frames = a[seg] + b[seg] * cos4[:, None, None] + c[seg] * nyq[:, None, None]
    assert frames.min() >= 0 and frames.max() <= 255
    return frames.astype(np.uint8), a, b, c


def closed_form_window(w, T, S, a, b, c, k):
    """S_k of window w (starting at frame w S), per pixel, from the segment
    amplitudes: the window's local time tau = t - w S; a tone exp(2 pi i m t / T)
    equals exp(2 pi i m w S / T) exp(2 pi i m tau / T) there."""
    H, W = a.shape[1:]
    out = np.zeros((H, W), dtype=np.complex128)
    t0 = w * S
    # split the window into its parts of constant segment
    tau = 0
    while tau < T:
        j = (t0 + tau) // S
        n = min(T - tau, (j + 1) * S - (t0 + tau))
        for amp, m in ((a[j], 0), (b[j] * 0.5, T // 4), (b[j] * 0.5, -(T // 4)), (c[j], T // 2)):
            # sum_tau exp(2 pi i m (t0 + tau) / T) exp(-2 pi i k tau / T)
            phase = cmath.exp(2j * math.pi * m * t0 / T)
            q = cmath.exp(2j * math.pi * (m - k) / T)
            out += amp * phase * geometric(q, tau, n)
        tau += n
    return out


def closed_form_moments(w, T, S, fs, klo, khi, a, b, c):
    P = {k: np.abs(closed_form_window(w, T, S, a, b, c, k)) ** 2 for k in range(klo, khi + 1)}

    def f_khz(k):
        kk = k if k < (T + 1) // 2 else k - T
        return kk * fs / T / 1000.0

    M0 = sum(P.values())
    M1 = sum(f_khz(k) * P[k] for k in P)
    M2 = sum(f_khz(k) ** 2 * P[k] for k in P)
    M1N = np.where(M0 > 0, M1 / np.where(M0 > 0, M0, 1), 0.0)
    M2N = np.where(M0 > 0, np.sqrt(np.maximum(M2 / np.where(M0 > 0, M0, 1), 0.0)), 0.0)
    return {"M0": M0, "M1": M1, "M2": M2, "M1N": M1N, "M2N": M2N}


@pytest.mark.parametrize("T,S,n_seg,band", [
    (8, 4, 7, (0, 7)),     # half-overlapping windows, full band (every bin, negative ones too)
    (16, 4, 9, (1, 8)),    # windows straddle 4 segments; band includes the T/4 tone
    (16, 12, 6, (3, 9)),   # stride not dividing T; band excludes DC
    (8, 8, 5, (2, 6)),     # back-to-back windows
    (8, 12, 6, (1, 4)),    # gaps between windows (S > T)
])
def test_render_matches_closed_form_per_window(T, S, n_seg, band):
    H, W = 3, 5  # non-square: a transposed pixel layout fails
    fs = 20000.0
    klo, khi = band
    frames, a, b, c = piecewise_stream(T, S, n_seg, H, W, seed=T * 100 + S)
    n = frames.shape[0]
    moments = ("M0", "M1", "M2", "M1N", "M2N")
    p = dict(spatial="none", temporal="stft", T=T, stride=S, fs_hz=fs, band_lo_bin=klo,
             band_hi_bin=khi, moments=moments)
    img = O.render(frames, p)
    # the number of complete windows, counted from the segment construction
    n_win = 0
    while n_win * S + T <= n:
        n_win += 1
    assert img.shape == (n_win, 5, H, W)
    for w in range(n_win):
        ref = closed_form_moments(w, T, S, fs, klo, khi, a, b, c)
        for q, name in enumerate(moments):
            scale = max(1.0, float(np.max(np.abs(ref[name]))))
            assert np.max(np.abs(img[w, q] - ref[name])) <= 1e-9 * scale, (w, name)
    # a subset of the moments keeps their relative order
    p2 = dict(p, moments=("M2N", "M0"))
    img2 = O.render(frames, p2)
    assert img2.shape == (n_win, 2, H, W)
    assert np.array_equal(img2[:, 0], img[:, 0]) and np.array_equal(img2[:, 1], img[:, 4])


def test_render_tail_and_short_streams():
    """Frames after the last complete window are not rendered; fewer than T frames
    render nothing."""
    T, S = 8, 4
    frames, a, b, c = piecewise_stream(T, S, 5, 2, 2, seed=7)
    p = dict(spatial="none", temporal="stft", T=T, stride=S, fs_hz=1000.0, band_lo_bin=0,
             band_hi_bin=7, moments=("M0",))
    full = O.render(frames, p)
    # 20 frames: windows at 0, 4, 8, 12 (the one at 16 would need frames 16..23)
    assert full.shape[0] == 4
    ragged = O.render(frames[:19], p)  # 19 frames: windows at 0, 4 and 8 only
    assert ragged.shape[0] == 3
    assert np.array_equal(ragged, full[:3])
    assert O.render(frames[:7], p).shape[0] == 0


@pytest.mark.parametrize("spatial,T,S", [("asp", 8, 3), ("fresnel", 8, 8), ("asp", 16, 4)])
def test_render_commutes_with_the_spatial_transform(spatial, T, S):
    """Temporal DFT of the window's raw frames first, then the spatial transform of
    every bin: the spectrum equals render()'s spatial-then-temporal one."""
    rng = np.random.default_rng(len(spatial) * 31 + T + S)
    H, W = 16, 8
    n = T + 3 * S + 2
    frames = rng.integers(0, 4096, (n, H, W)).astype(np.uint16)
    klo, khi = 1, T // 2
    p = dict(spatial=spatial, z_m=0.21, lambda_m=852e-9, pitch_x_m=20e-6, pitch_y_m=23e-6,
             fftshift=1, temporal="stft", T=T, stride=S, fs_hz=7000.0, band_lo_bin=klo,
             band_hi_bin=khi, moments=("M0", "M1", "M2"))
    img = O.render(frames, p)
    w = 0
    for s0 in range(0, n - T + 1, S):
        raw = frames[s0:s0 + T].astype(np.float64)
        D = np.fft.fft(raw, axis=0)                       # temporal DFT of the raw window
        Sk = np.stack([O.spatial(D[k], p) for k in range(T)])  # then the spatial transform
        P = np.abs(Sk[klo:khi + 1]) ** 2
        f = O.bin_frequency_khz(np.arange(klo, khi + 1), T, p["fs_hz"])
        ref = [P.sum(0), np.tensordot(f, P, 1), np.tensordot(f * f, P, 1)]
        for q in range(3):
            assert np.allclose(img[w, q], ref[q], rtol=1e-9, atol=1e-9 * np.abs(ref[q]).max()), (w, q)
        w += 1
    assert w == img.shape[0]
