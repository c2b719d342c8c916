"""FP64 CPU oracle of the hologram-rendering hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check and
the benchmark's CPU-baseline / reference arm may import this module.  The
product path never calls it and has no CPU fallback.

It is a plain, slow, obviously-correct restatement of what the rendering path
computes, in float64 / complex128, written from the method description:

* Sec. III-B.1 (space and time transformations): each raw frame is converted to
  complex, transformed spatially (angular-spectrum propagation or Fresnel
  transform), pushed into a time-transformation queue, and a short-time
  temporal transform (FFT, or PCA via covariance / eigendecomposition /
  projection onto a sub-basis) is applied to windows of consecutive
  propagated frames; a statistical moment is then taken per pixel over a range
  of temporal indices.
* Sec. VI-B (Table IV): windows of T frames repeated every S frames ("time
  stride").

The paper prints no formulas.  The formulas used here are the textbook forms
of the named operations; every point where the paper is silent is resolved by
a stated reading (see the docstrings, each marked READING).

Library primitives used as single steps: numpy.fft (forward transform is
unnormalised, inverse carries 1/n) and numpy.linalg.eigh.  There is no tiling,
fusion or reordering beyond the definitions.

Pinned by tests/test_oracle_pins.py (brute-force DFT, Parseval, closed-form
plane-wave propagation, Fresnel chirp collapse, pure temporal tones, PCA
trace / rank-one / known-spectrum cases, exhaustive conversion).
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------- conversion


def convert(frames: np.ndarray) -> np.ndarray:
    """Integer frames -> complex field, re = pixel value, im = 0 (Sec. III-B.1).

    READING: values are not rescaled (12-bit samples stay in 0..4095).
    """
    if frames.dtype not in (np.uint8, np.uint16):
        raise TypeError("frames must be uint8 or uint16")
    return frames.astype(np.float64).astype(np.complex128)


# ------------------------------------------------------------ 2-D transforms


def fft2(u: np.ndarray) -> np.ndarray:
    """Unnormalised forward 2-D DFT over the last two axes.

    F[m, n] = sum_{y, x} u[y, x] exp(-2 pi i (m y / H + n x / W)).
    READING (paper silent on conventions): forward unnormalised, inverse 1/(HW).
    """
    return np.fft.fft2(u, axes=(-2, -1))


def ifft2(U: np.ndarray) -> np.ndarray:
    """Inverse 2-D DFT with the 1/(HW) factor."""
    return np.fft.ifft2(U, axes=(-2, -1))


def spatial_frequencies(n: int, d: float) -> np.ndarray:
    """Angular spatial frequency of DFT bin m in FFT order: 2 pi m' / (n d),
    with m' = m for m < n/2 and m' = m - n otherwise."""
    m = np.arange(n)
    m = np.where(m < n // 2, m, m - n)
    return 2.0 * np.pi * m / (n * d)


def asp_transfer(H: int, W: int, lam: float, dx: float, dy: float, z: float) -> np.ndarray:
    """Angular-spectrum transfer function H(kx, ky) = exp(i z sqrt(k^2 - kx^2 - ky^2)).

    Angular-spectrum propagation is named in Sec. III-B.1 and Sec. VI-B.1.
    READINGS: evanescent components (kx^2 + ky^2 > k^2) are set to 0; the global
    phase exp(i k z) is kept; the phase is evaluated in float64 directly.
    """
    k = 2.0 * np.pi / lam
    kx = spatial_frequencies(W, dx)[None, :]
    ky = spatial_frequencies(H, dy)[:, None]
    kz2 = k * k - kx * kx - ky * ky
    out = np.zeros((H, W), dtype=np.complex128)
    prop = kz2 >= 0
    out[prop] = np.exp(1j * z * np.sqrt(kz2[prop]))
    return out


def asp(u: np.ndarray, lam: float, dx: float, dy: float, z: float) -> np.ndarray:
    """Angular-spectrum propagation by z: IFFT2( FFT2(u) * H ) (Sec. III-B.1).

    READING: the reconstruction applies H(+z) with the user's z, no fftshift.
    """
    H, W = u.shape[-2:]
    return ifft2(fft2(u) * asp_transfer(H, W, lam, dx, dy, z))


def fresnel_chirp(H: int, W: int, lam: float, dx: float, dy: float, z: float) -> np.ndarray:
    """Input chirp exp(i pi (x^2 + y^2) / (lam z)), x = (j - W/2) dx, y = (l - H/2) dy."""
    x = (np.arange(W) - W / 2) * dx
    y = (np.arange(H) - H / 2) * dy
    return np.exp(1j * np.pi * (x[None, :] ** 2 + y[:, None] ** 2) / (lam * z))


def fresnel(u: np.ndarray, lam: float, dx: float, dy: float, z: float,
            fftshift: bool = True) -> np.ndarray:
    """Single-FFT Fresnel transform: FFT2(u * chirp), optionally fftshifted.

    The Fresnel transform is named in Sec. III-B.1 and Sec. VI-B.2.
    READINGS: the output prefactor exp(ikz)/(i lam z) and the output chirp are
    dropped (constant in time per pixel, so moments and PCA energies ignore
    them); fftshift (when on) moves the zero frequency to the frame centre.
    """
    H, W = u.shape[-2:]
    out = fft2(u * fresnel_chirp(H, W, lam, dx, dy, z))
    if fftshift:
        out = np.fft.fftshift(out, axes=(-2, -1))
    return out


def highpass(u: np.ndarray, cutoff: float) -> np.ndarray:
    """Ideal radial high-pass spatial filter (Sec. VI-B.1 applies one after the
    angular-spectrum propagation; shape and cutoff are unspecified).

    READING: zero every DFT bin whose radius sqrt((m'/W)^2 + (n'/H)^2) in cycles
    per pixel (signed FFT-order indices) is below `cutoff`.
    """
    H, W = u.shape[-2:]
    m = np.arange(W)
    m = np.where(m < W // 2, m, m - W) / W
    n = np.arange(H)
    n = np.where(n < H // 2, n, n - H) / H
    keep = (m[None, :] * m[None, :] + n[:, None] * n[:, None]) >= cutoff * cutoff
    return ifft2(fft2(u) * keep)


def spatial(frames_c: np.ndarray, p: dict) -> np.ndarray:
    """Apply the configured spatial transform to complex frames [..., H, W]."""
    kind = p["spatial"]
    if kind == "none":
        return frames_c.copy()
    if kind == "asp":
        out = asp(frames_c, p["lambda_m"], p["pitch_x_m"], p["pitch_y_m"], p["z_m"])
        if p.get("highpass", 0.0) > 0.0:
            out = highpass(out, p["highpass"])
        return out
    if kind == "fresnel":
        return fresnel(frames_c, p["lambda_m"], p["pitch_x_m"], p["pitch_y_m"], p["z_m"],
                       bool(p.get("fftshift", 1)))
    raise ValueError(kind)


# ------------------------------------------------------------------ windows


def window_starts(n_frames: int, T: int, S: int) -> list[int]:
    """Starts of the complete windows over a stream of n_frames frames.

    Window w covers frames w*S .. w*S+T-1 (T = window, S = time stride,
    Table IV); only complete windows are rendered.
    """
    if n_frames < T:
        return []
    return list(range(0, n_frames - T + 1, S))


def band_bins_from_hz(f_lo: float, f_hi: float, fs: float, T: int) -> tuple[int, int]:
    """Inclusive positive-frequency bin range [ceil(f_lo T/fs), floor(f_hi T/fs)].

    READING: a band given in Hz keeps the bins whose centre frequency k fs / T
    lies inside [f_lo, f_hi].
    """
    return int(math.ceil(f_lo * T / fs - 1e-12)), int(math.floor(f_hi * T / fs + 1e-12))


# ---------------------------------------------------------------- STFT path


def bin_frequency_khz(k: np.ndarray, T: int, fs: float) -> np.ndarray:
    """Frequency of temporal bin k in kHz; bins k >= T/2 map to (k - T) fs / T."""
    k = np.asarray(k)
    kk = np.where(k < (T + 1) // 2, k, k - T)
    return kk * fs / T / 1000.0


def stft_moments(U: np.ndarray, fs: float, k_lo: int, k_hi: int) -> dict:
    """Short-time FFT over one window and its band moments (Sec. III-B.1).

    U: propagated frames of one window, shape (T, H, W) complex.
    S_k(p) = sum_t U_t(p) exp(-2 pi i k t / T)  (forward, unnormalised);
    P_k = |S_k|^2;  M0 = sum_band P_k;  M1 = sum_band f_k P_k;
    M2 = sum_band f_k^2 P_k, with f_k in kHz; band = k_lo..k_hi inclusive.
    Normalised outputs M1/M0 and sqrt(M2/M0) are 0 where M0 == 0.
    READINGS: rectangular window; no temporal mean subtraction; positive
    (non-mirrored) band; M1/M2 in kHz units.
    """
    T = U.shape[0]
    S = np.fft.fft(U, axis=0)
    P = S.real ** 2 + S.imag ** 2
    ks = np.arange(k_lo, k_hi + 1)
    f = bin_frequency_khz(ks, T, fs)
    Pb = P[k_lo:k_hi + 1]
    M0 = Pb.sum(axis=0)
    M1 = np.tensordot(f, Pb, axes=(0, 0))
    M2 = np.tensordot(f * f, Pb, axes=(0, 0))
    with np.errstate(divide="ignore", invalid="ignore"):
        M1N = np.where(M0 > 0, M1 / M0, 0.0)
        M2N = np.where(M0 > 0, np.sqrt(np.maximum(M2 / M0, 0.0)), 0.0)
    return {"M0": M0, "M1": M1, "M2": M2, "M1N": M1N, "M2N": M2N}


MOMENT_ORDER = ("M0", "M1", "M2", "M1N", "M2N")


# ----------------------------------------------------------------- PCA path


def pca(U: np.ndarray, j_lo: int, j_hi: int) -> dict:
    """PCA of one window and the energy of its projection on a sub-basis.

    Sec. III-B.1: a covariance matrix of the window, its eigendecomposition and
    a projection onto a sub-basis.  With X the P x T matrix whose column t is
    frame t flattened (P = H W):
      C = X^H X  (T x T Hermitian),  C = V diag(lam) V^H,  lam descending;
      Y = X V[:, j_lo-1 : j_hi]  (eigenvectors j_lo..j_hi, 1-based, inclusive);
      E(p) = sum_j |Y[p, j]|^2.
    READINGS: no mean subtraction and no 1/P scaling (neither changes the
    eigenvectors or E up to the stated scale); eigenvector phases are arbitrary
    so only lam and E are outputs.
    """
    T, H, W = U.shape
    X = U.reshape(T, H * W).T
    C = X.conj().T @ X
    lam, V = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    V = V[:, order]
    Y = X @ V[:, j_lo - 1:j_hi]
    E = (Y.real ** 2 + Y.imag ** 2).sum(axis=1).reshape(H, W)
    return {"C": C, "lam": lam, "V": V, "E": E}


# -------------------------------------------------------------- whole path


def render(frames: np.ndarray, p: dict) -> np.ndarray:
    """Render every complete window of a raw stream (Sec. III-B, Fig. 1).

    Returns images window-major: STFT -> (n_win, n_sel_moments, H, W) in the
    order M0, M1, M2, M1N, M2N restricted to p["moments"]; PCA -> (n_win, 1, H, W).
    """
    T, S = p["T"], p["stride"]
    starts = window_starts(frames.shape[0], T, S)
    H, W = frames.shape[1:]
    outs = []
    # Spatial transform of each frame once (the time-transformation queue).
    needed = sorted({s + t for s in starts for t in range(T)})
    prop = {}
    for f in needed:
        prop[f] = spatial(convert(frames[f]), p)
    for s in starts:
        Uw = np.stack([prop[s + t] for t in range(T)])
        if p["temporal"] == "stft":
            m = stft_moments(Uw, p["fs_hz"], p["band_lo_bin"], p["band_hi_bin"])
            outs.append(np.stack([m[name] for name in MOMENT_ORDER if name in p["moments"]]))
        elif p["temporal"] == "pca":
            outs.append(pca(Uw, p["pca_lo"], p["pca_hi"])["E"][None])
        else:
            raise ValueError(p["temporal"])
    if not outs:
        return np.zeros((0, 0, H, W))
    return np.stack(outs)


# ----------------------------------------------------------- focus metrics


def tamura(img: np.ndarray) -> float:
    """Tamura coefficient sqrt(sigma / mu) of an amplitude image.

    READING: population standard deviation; 0 when the mean is 0.
    """
    a = np.asarray(img, dtype=np.float64)
    mu = a.mean()
    if mu == 0:
        return 0.0
    return math.sqrt(a.std() / mu)

# ----------------------------------------------------------- post-processing


def gaussian_kernel(size: int, sigma: float) -> np.ndarray:
    """size x size kernel exp(-(dx^2 + dy^2) / (2 sigma^2)), dx, dy in -(size//2)..size//2,
    normalised to sum 1."""
    r = np.arange(size) - size // 2
    g = np.exp(-(r[None, :] ** 2 + r[:, None] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def convolve_periodic(img: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """out[y, x] = sum_{a, b} kern[a, b] img[(y + a - K//2) mod H, (x + b - K//2) mod W].

    READING: the paper convolves rendered images with a given kernel (Sec. III-B,
    post-processing) without naming the boundary; the image is taken as periodic,
    as a Fourier-domain convolution of the same size computes it. The kernel is
    applied as a correlation (not flipped), so a user kernel acts as written.
    """
    K = kern.shape[0]
    out = np.zeros(img.shape, dtype=np.float64)
    for a in range(K):
        for b in range(K):
            out += kern[a, b] * np.roll(img, shift=(K // 2 - a, K // 2 - b), axis=(0, 1))
    return out


def postprocess(images: np.ndarray, kern=None, renormalize=False, accumulate=1) -> np.ndarray:
    """Post-processing of one stream of rendered images (Sec. III-B): convolution,
    then re-normalisation, then the moving average of the accumulation buffer.

    images: (n, H, W), in rendering order. READINGS: re-normalisation divides an
    image by its spatial mean (0 where the mean is 0); the accumulation buffer of
    size A outputs, for image t, the mean of images max(0, t - A + 1) .. t after
    the steps above.
    """
    out = []
    for img in np.asarray(images, dtype=np.float64):
        v = convolve_periodic(img, np.asarray(kern, dtype=np.float64)) if kern is not None else img.copy()
        if renormalize:
            m = v.mean()
            v = v / m if m != 0 else np.zeros_like(v)
        out.append(v)
    out = np.stack(out) if out else np.zeros((0,) + tuple(np.shape(images)[1:]))
    acc = np.empty_like(out)
    for t in range(out.shape[0]):
        lo = max(0, t - accumulate + 1)
        acc[t] = out[lo:t + 1].mean(axis=0)
    return acc

