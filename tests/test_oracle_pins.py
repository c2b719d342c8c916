"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes one part of the oracle to brute force on tiny inputs, a closed
form, an invariant, or a special case whose answer is known from the
mathematics -- chosen so that a dropped term, a wrong sign, a wrong axis or a
transposed operand in the oracle fails at least one of them.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import hv_oracle as O

RNG = np.random.default_rng(12345)


def crandn(*shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


# --------------------------------------------------------------- conversion

def test_convert_exhaustive_u8_u16():
    v8 = np.arange(256, dtype=np.uint8).reshape(1, 16, 16)
    c = O.convert(v8)
    assert np.array_equal(c.real, np.arange(256).reshape(1, 16, 16))
    assert np.all(c.imag == 0)
    v16 = np.arange(65536, dtype=np.uint16).reshape(1, 256, 256)
    c = O.convert(v16)
    assert np.array_equal(c.real, np.arange(65536).reshape(1, 256, 256))
    assert np.all(c.imag == 0)


# ------------------------------------------------------------------- 2-D DFT

@pytest.mark.parametrize("H,W", [(8, 8), (4, 8)])
def test_fft2_matches_brute_force_dft(H, W):
    u = crandn(H, W)
    F = O.fft2(u)
    for m in range(H):
        for n in range(W):
            acc = 0j
            for y in range(H):
                for x in range(W):
                    acc += u[y, x] * cmath.exp(-2j * math.pi * (m * y / H + n * x / W))
            assert abs(F[m, n] - acc) <= 1e-12 * max(1.0, abs(acc))
    assert np.allclose(O.ifft2(F), u, atol=1e-13)


def test_fft2_parseval():
    u = crandn(3, 16, 32)
    F = O.fft2(u)
    assert np.isclose((np.abs(F) ** 2).sum(), 16 * 32 * (np.abs(u) ** 2).sum(), rtol=1e-12)


# ----------------------------------------------------------------------- ASP

LAM, DX, DY = 852e-9, 20e-6, 17e-6


def test_asp_z0_is_identity():
    u = crandn(16, 32)
    assert np.allclose(O.asp(u, LAM, DX, DY, 0.0), u, atol=1e-12)


def test_asp_round_trip():
    u = crandn(32, 16)
    v = O.asp(O.asp(u, LAM, DX, DY, 0.3), LAM, DX, DY, -0.3)
    assert np.max(np.abs(v - u)) <= 1e-10 * np.max(np.abs(u))


@pytest.mark.parametrize("m0,n0", [(-5, 3), (7, -2), (0, 0)])
def test_asp_plane_wave_closed_form(m0, n0):
    """A grid plane wave exp(i (kx0 x + ky0 y)) propagates to itself times
    exp(i z sqrt(k^2 - kx0^2 - ky0^2)); x = j dx, y = l dy."""
    H, W, z = 16, 32, 0.3
    j = np.arange(W)[None, :]
    l = np.arange(H)[:, None]
    kx0 = 2 * math.pi * m0 / (W * DX)
    ky0 = 2 * math.pi * n0 / (H * DY)
    u = np.exp(1j * (kx0 * j * DX + ky0 * l * DY))
    k = 2 * math.pi / LAM
    expect = u * cmath.exp(1j * z * math.sqrt(k * k - kx0 * kx0 - ky0 * ky0))
    got = O.asp(u, LAM, DX, DY, z)
    assert np.max(np.abs(got - expect)) <= 1e-9


def test_asp_evanescent_components_vanish():
    # lambda = 60 um on a 20 um grid: frequencies above k are evanescent.
    lam, d, H, W = 60e-6, 20e-6, 8, 16
    k = 2 * math.pi / lam
    m0 = 7  # kx = 2 pi 7 / (16 * 20um) > k
    assert 2 * math.pi * m0 / (W * d) > k
    j = np.arange(W)[None, :] * np.ones((H, 1))
    u = np.exp(2j * math.pi * m0 * j / W)
    assert np.max(np.abs(O.asp(u, lam, d, d, 0.1))) <= 1e-12
    m1 = 1  # propagating
    u1 = np.exp(2j * math.pi * m1 * j / W)
    assert np.max(np.abs(O.asp(u1, lam, d, d, 0.1))) == pytest.approx(1.0)


# ------------------------------------------------------------------- Fresnel

@pytest.mark.parametrize("shift", [False, True])
@pytest.mark.parametrize("m0,n0", [(3, -2), (0, 0), (-4, 5)])
def test_fresnel_collapses_paraxial_point_wave(shift, m0, n0):
    """The paraxial wave exp(-i pi ((x-a)^2 + (y-b)^2) / (lam z)) of a point at
    (a, b) = (m0 lam z / (W dx), n0 lam z / (H dy)) becomes a single DFT bin
    (m0, n0) of height H W exp(-i pi (a^2 + b^2)/(lam z)) exp(-i pi (m0 + n0)),
    with centred coordinates x = (j - W/2) dx, y = (l - H/2) dy."""
    H, W, z = 16, 32, 0.25
    a = m0 * LAM * z / (W * DX)
    b = n0 * LAM * z / (H * DY)
    x = (np.arange(W) - W / 2) * DX
    y = (np.arange(H) - H / 2) * DY
    u = np.exp(-1j * math.pi * ((x[None, :] - a) ** 2 + (y[:, None] - b) ** 2) / (LAM * z))
    F = O.fresnel(u, LAM, DX, DY, z, fftshift=shift)
    amp = H * W * cmath.exp(-1j * math.pi * (a * a + b * b) / (LAM * z)) * cmath.exp(-1j * math.pi * (m0 + n0))
    row = (n0 + (H // 2 if shift else 0)) % H
    col = (m0 + (W // 2 if shift else 0)) % W
    expect = np.zeros((H, W), complex)
    expect[row, col] = amp
    assert np.max(np.abs(F - expect)) <= 1e-8 * H * W


def test_fresnel_linearity():
    u, v = crandn(8, 16), crandn(8, 16)
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    lhs = O.fresnel(a * u + b * v, LAM, DX, DY, 0.2)
    rhs = a * O.fresnel(u, LAM, DX, DY, 0.2) + b * O.fresnel(v, LAM, DX, DY, 0.2)
    assert np.allclose(lhs, rhs, atol=1e-10)


# ---------------------------------------------------------------- windows

def test_window_starts():
    assert O.window_starts(10, 4, 3) == [0, 3, 6]
    assert O.window_starts(3, 4, 1) == []
    assert O.window_starts(8, 4, 4) == [0, 4]
    assert O.window_starts(100_000, 512, 64)[-1] == 64 * ((100_000 - 512) // 64)


def test_band_from_hz_paper_scale_stream():
    # 1..35 kHz at fs = 71.4 kHz, T = 512: bin width 139.45 Hz.
    assert O.band_bins_from_hz(1000.0, 35000.0, 71400.0, 512) == (8, 250)
    # edges that fall exactly on a bin are kept
    assert O.band_bins_from_hz(1000.0, 2000.0, 64000.0, 64) == (1, 2)


# ------------------------------------------------------------------- STFT

def _tone(T, k0, amp):
    t = np.arange(T)[:, None, None]
    return amp[None] * np.exp(2j * math.pi * k0 * t / T)


@pytest.mark.parametrize("k0,inband", [(6, True), (3, False), (29, False), (28, True)])
def test_stft_pure_tone_lands_in_its_bin(k0, inband):
    T, fs = 64, 20000.0
    amp = crandn(4, 8)
    U = _tone(T, k0, amp)
    m = O.stft_moments(U, fs, 4, 28)
    A2 = np.abs(amp) ** 2
    f = k0 * fs / T / 1000.0          # kHz
    if inband:
        assert np.allclose(m["M0"], A2 * T * T, rtol=1e-12)
        assert np.allclose(m["M1"], f * A2 * T * T, rtol=1e-12)
        assert np.allclose(m["M2"], f * f * A2 * T * T, rtol=1e-12)
        assert np.allclose(m["M1N"], f, rtol=1e-12)
        assert np.allclose(m["M2N"], abs(f), rtol=1e-12)
    else:
        assert np.max(m["M0"]) <= 1e-18 * T * T * A2.max()


def test_stft_negative_frequency_bin():
    T, fs = 32, 1000.0
    U = _tone(T, T - 3, np.ones((2, 2)))     # exp(2 pi i (T-3) t / T) = exp(-2 pi i 3 t / T)
    m = O.stft_moments(U, fs, T - 3, T - 3)
    assert np.allclose(m["M1N"], -3 * fs / T / 1000.0, rtol=1e-12)


def test_stft_two_tones_closed_form():
    T, fs, k1, k2 = 128, 50000.0, 10, 21
    amp = np.ones((3, 5))
    U = _tone(T, k1, amp) + 2.0 * _tone(T, k2, amp)
    m = O.stft_moments(U, fs, 8, 40)
    f1, f2 = k1 * fs / T / 1e3, k2 * fs / T / 1e3
    assert np.allclose(m["M0"], 5 * T * T, rtol=1e-12)
    assert np.allclose(m["M1N"], (f1 + 4 * f2) / 5, rtol=1e-12)
    assert np.allclose(m["M2N"], math.sqrt((f1 * f1 + 4 * f2 * f2) / 5), rtol=1e-12)


def test_stft_full_band_parseval_and_constant_signal():
    T = 64
    U = crandn(T, 4, 4)
    m = O.stft_moments(U, 20000.0, 0, T - 1)
    assert np.allclose(m["M0"], T * (np.abs(U) ** 2).sum(axis=0), rtol=1e-12)
    C = np.ones((T, 4, 4)) * (3 - 2j)
    m = O.stft_moments(C, 20000.0, 4, 28)
    assert np.max(m["M0"]) <= 1e-20 * (T * 13) ** 2
    assert np.all(m["M1N"][m["M0"] == 0] == 0)


# -------------------------------------------------------------------- PCA

def _unitary(n, m):
    q, _ = np.linalg.qr(crandn(n, m))
    return q


def test_pca_known_spectrum():
    """X = Q diag(s) W^H with orthonormal Q (P x T) and unitary W: the
    eigenvalues of X^H X are s^2, and the energy of the projection on the
    eigenvectors ranked j_lo..j_hi (descending) is sum_j s_j^2 |Q[p, j]|^2."""
    T, H, Wd = 12, 6, 5
    P = H * Wd
    Q = _unitary(P, T)
    Wm = _unitary(T, T)
    s = RNG.permutation(np.linspace(1.0, 12.0, T))       # distinct, shuffled
    X = Q @ np.diag(s) @ Wm.conj().T
    U = X.T.reshape(T, H, Wd)
    r = O.pca(U, 2, 5)
    order = np.argsort(s)[::-1]
    assert np.allclose(r["lam"], s[order] ** 2, rtol=1e-10)
    sel = order[1:5]
    expect = (np.abs(Q[:, sel]) ** 2 * (s[sel] ** 2)[None]).sum(axis=1).reshape(H, Wd)
    assert np.allclose(r["E"], expect, rtol=1e-9, atol=1e-12)


def test_pca_rank_one_and_trace():
    T, H, Wd = 16, 4, 8
    u = crandn(H * Wd)
    v = crandn(T)
    X = np.outer(u, v.conj())
    r = O.pca(X.T.reshape(T, H, Wd), 2, T)
    nu, nv = np.linalg.norm(u) ** 2, np.linalg.norm(v) ** 2
    assert r["lam"][0] == pytest.approx(nu * nv, rel=1e-10)
    assert np.max(np.abs(r["lam"][1:])) <= 1e-9 * nu * nv
    assert np.max(r["E"]) <= 1e-9 * nu * nv
    r1 = O.pca(X.T.reshape(T, H, Wd), 1, 1)
    assert np.allclose(r1["E"].ravel(), np.abs(u) ** 2 * nv, rtol=1e-9)
    # trace and eigen-residual on a general window
    Ug = crandn(T, H, Wd)
    r = O.pca(Ug, 1, T)
    assert r["lam"].sum() == pytest.approx((np.abs(Ug) ** 2).sum(), rel=1e-10)
    C, V, lam = r["C"], r["V"], r["lam"]
    assert np.linalg.norm(C @ V - V * lam[None]) <= 1e-10 * np.linalg.norm(C)
    assert np.allclose(V.conj().T @ V, np.eye(T), atol=1e-12)
    assert np.all(np.diff(lam) <= 0)


# ------------------------------------------------------------------ Tamura

def test_tamura_constant_and_two_level():
    assert O.tamura(np.full((8, 8), 5.0)) == 0.0
    assert O.tamura(np.zeros((4, 4))) == 0.0
    img = np.zeros((8, 8))
    img[:4] = 1.0
    img[4:] = 3.0
    assert O.tamura(img) == pytest.approx(math.sqrt(1.0 / 2.0), rel=1e-12)


# ---------------------------------------------------------------- high-pass

def test_highpass_plane_waves_below_and_above_cutoff():
    """A grid plane wave of radius r cycles/pixel survives the filter iff r >= cutoff."""
    H, W = 16, 32
    j = np.arange(W)[None, :]
    l = np.arange(H)[:, None]
    for m0, n0 in [(1, 0), (3, -2), (-6, 4), (0, 0)]:
        u = np.exp(2j * math.pi * (m0 * j / W + n0 * l / H))
        r = math.hypot(m0 / W, n0 / H)
        for cut in (0.05, 0.15, 0.3):
            got = O.highpass(u, cut)
            expect = u if r >= cut else np.zeros_like(u)
            assert np.max(np.abs(got - expect)) <= 1e-12
    assert np.allclose(O.highpass(u, 0.0), u)
