"""Seeded synthetic interferogram streams.

This module produces test and benchmark INPUT only.  It holds none of the
rendering method's arithmetic (no Fourier transform, no propagation kernel, no
temporal analysis): the object waves are written down analytically as sums of
spherical waves from point scatterers, interfered with a tilted plane reference
and passed through Poisson shot noise.  Both the CUDA path and the CPU oracle
consume the arrays it returns; neither is imported here.

Physics of the scene (off-axis Doppler holography, Sec. I and Sec. VI of the
paper describe the application; the scene itself is ours):

* a "static" speckle object: ``n_static`` point scatterers with random
  amplitude and uniform random phase, spread over a disk of radius N/4 pixels
  in a plane at distance ``z_obj`` from the sensor;
* a "Doppler" disk: ``n_doppler`` scatterers in a disk of radius N/16 pixels,
  offset from the centre, whose phase turns at a Doppler frequency (one
  frequency for the whole disk, or one per scatterer group);
* the sensor field of a scatterer at (xm, ym, z) is the converging spherical
  wave ``exp(-i k r) / r`` so that propagating the recorded field by +z
  refocuses the object (the reconstruction convention of the rendering path);
* a plane reference ``a * exp(2 pi i (x + y) / (4 dx))`` (carrier at bin N/4)
  with ``|R|^2 / <|O|^2> = ref_ratio``;
* intensity ``|R + O_t|^2`` scaled so that its mean is ``mean_fraction`` of
  full scale, then Poisson noise and clipping to the pixel depth.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    """Seeded description of one synthetic recording."""

    N: int = 256                 # frame is N x N pixels
    bits: int = 8                # 8 -> uint8 frames, 12 or 16 -> uint16 frames
    lam: float = 852e-9          # wavelength [m]
    pitch: float = 20e-6         # sensor pixel pitch [m]
    z_obj: float = 0.30          # object distance [m]
    fs: float = 20_000.0         # camera frame rate [Hz]
    doppler_hz: tuple = (3000.0,)  # one entry per Doppler scatterer group
    n_static: int = 384
    n_doppler: int = 64
    ref_ratio: float = 10.0
    mean_fraction: float = 0.30
    seed: int = 1000
    noise: bool = True
    # filled by build()
    _static: np.ndarray | None = field(default=None, repr=False)
    _groups: list = field(default_factory=list, repr=False)
    _ref: np.ndarray | None = field(default=None, repr=False)
    _gain: float = 0.0

    @property
    def full_scale(self) -> int:
        return (1 << self.bits) - 1 if self.bits <= 16 else 65535

    @property
    def dtype(self):
        return np.uint8 if self.bits <= 8 else np.uint16

    def doppler_center_px(self) -> tuple[float, float]:
        """Object-plane centre of the Doppler disk, in pixels from frame centre."""
        return (self.N / 8.0, self.N / 8.0)


def _spherical_sum(N, pitch, lam, z, xs, ys, amps):
    """Sum of converging spherical waves a_m exp(-i k r_m) / r_m on the sensor grid."""
    k = 2.0 * np.pi / lam
    coords = (np.arange(N) - N / 2) * pitch
    X = coords[None, :]
    Y = coords[:, None]
    out = np.zeros((N, N), dtype=np.complex128)
    for xm, ym, am in zip(xs, ys, amps):
        r = np.sqrt((X - xm) ** 2 + (Y - ym) ** 2 + z * z)
        out += am * np.exp(-1j * k * r) * (z / r)
    return out


def build(scene: Scene) -> Scene:
    """Draw the scatterers and precompute the static and Doppler sensor fields."""
    rng = np.random.Generator(np.random.PCG64(scene.seed))
    N, p = scene.N, scene.pitch

    def disk(n, radius_px, cx_px, cy_px):
        rad = radius_px * np.sqrt(rng.random(n))
        ang = 2.0 * np.pi * rng.random(n)
        return (cx_px + rad * np.cos(ang)) * p, (cy_px + rad * np.sin(ang)) * p

    xs, ys = disk(scene.n_static, N / 4.0, 0.0, 0.0)
    amp = (0.25 + 0.75 * (rng.random(scene.n_static) < 0.3)) * np.exp(
        2j * np.pi * rng.random(scene.n_static))
    static = _spherical_sum(N, p, scene.lam, scene.z_obj, xs, ys, amp)

    cx, cy = scene.doppler_center_px()
    xd, yd = disk(scene.n_doppler, N / 16.0, cx, cy)
    ampd = np.exp(2j * np.pi * rng.random(scene.n_doppler))
    G = len(scene.doppler_hz)
    groups = []
    for g in range(G):
        sel = slice(g, None, G)
        groups.append((float(scene.doppler_hz[g]),
                       _spherical_sum(N, p, scene.lam, scene.z_obj, xd[sel], yd[sel], ampd[sel])))

    # Normalise <|O|^2> = 1 over static + Doppler parts.
    power = np.mean(np.abs(static) ** 2) + sum(np.mean(np.abs(f) ** 2) for _, f in groups)
    s = 1.0 / np.sqrt(power)
    static *= s
    groups = [(f, fld * s) for f, fld in groups]

    coords = np.arange(N)
    phase = 2.0 * np.pi * (coords[None, :] + coords[:, None]) / 4.0
    ref = np.sqrt(scene.ref_ratio) * np.exp(1j * phase)

    i0 = np.abs(ref + static + sum(f for _, f in groups)) ** 2
    scene._gain = scene.mean_fraction * scene.full_scale / float(np.mean(i0))
    scene._static, scene._groups, scene._ref = static, groups, ref
    scene._noise_seed = int(rng.integers(0, 2**63 - 1))
    return scene


def frames(scene: Scene, t0: int, n: int) -> np.ndarray:
    """Frames t0 .. t0+n-1 of the recording, shape (n, N, N), uint8/uint16.

    Frame t depends only on (seed, t): chunked generation is reproducible.
    """
    if scene._static is None:
        build(scene)
    N = scene.N
    out = np.empty((n, N, N), dtype=scene.dtype)
    base = scene._ref + scene._static
    for i in range(n):
        t = t0 + i
        u = base.copy()
        for f, fld in scene._groups:
            u += np.exp(2j * np.pi * f * t / scene.fs) * fld
        inten = scene._gain * (u.real ** 2 + u.imag ** 2)
        if scene.noise:
            rng = np.random.Generator(np.random.PCG64([scene._noise_seed, t]))
            inten = rng.poisson(inten).astype(np.float64)
        else:
            inten = np.rint(inten)
        np.clip(inten, 0, scene.full_scale, out=inten)
        out[i] = inten.astype(scene.dtype)
    return out


# Scenes of the five workloads (seeded 1000 + i).
def scene_tiny_asp_stft(**kw) -> Scene:
    """64 frames of 256x256 uint8, object at 0.30 m, 3 kHz Doppler disk at fs=20 kHz."""
    d = dict(N=256, bits=8, z_obj=0.30, fs=20_000.0, doppler_hz=(3000.0,), seed=1000)
    d.update(kw)
    return Scene(**d)


def scene_stream_fresnel(**kw) -> Scene:
    """256x256 12-bit frames at 71.4 kHz, Doppler groups spread over 2..20 kHz."""
    d = dict(N=256, bits=12, z_obj=0.25, fs=71_400.0,
             doppler_hz=tuple(np.linspace(2000.0, 20000.0, 8)), seed=1001)
    d.update(kw)
    return Scene(**d)


def scene_pca(**kw) -> Scene:
    """512x512 12-bit frames, object at 0.40 m."""
    d = dict(N=512, bits=12, z_obj=0.40, fs=20_000.0,
             doppler_hz=(1500.0, 3000.0, 4500.0, 6000.0), seed=1002)
    d.update(kw)
    return Scene(**d)


def random_complex(shape, seed) -> np.ndarray:
    """Seeded complex normal array (complex128), for kernel-level parity cases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_frames(n, H, W, bits, seed) -> np.ndarray:
    """Seeded uniform integer frames (full range of the pixel depth)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hi = (1 << bits)
    dt = np.uint8 if bits <= 8 else np.uint16
    return rng.integers(0, hi, size=(n, H, W), dtype=np.int64).astype(dt)


# ------------------------------------------------ autofocus holograms

AF_Z_RANGE = (0.10, 0.60)


def _pixel_point_field(N, pitch, lam, z, ipx, ipy, amps):
    """Sum of converging spherical waves a_m exp(-i k r_m) z / r_m from scatterers at
    pixel centres (column ipx, row ipy of the sensor grid). Every scatterer's wave
    is a shifted copy of one point-spread function, tabulated once on the 2N x 2N
    grid of pixel offsets (phase k (r - z) in float64 from rho^2 / (r + z), the
    exponential in complex64; the common factor exp(-i k z) is dropped)."""
    k = 2.0 * np.pi / lam
    d = (np.arange(2 * N) - N) * pitch
    rho2 = d[None, :] ** 2 + d[:, None] ** 2
    r = np.sqrt(rho2 + z * z)
    ph = np.mod(k * rho2 / (r + z), 2.0 * np.pi).astype(np.float32)
    psf = np.empty(ph.shape, dtype=np.complex64)
    psf.real = np.cos(ph)
    psf.imag = -np.sin(ph)
    psf *= (z / r).astype(np.float32)
    out = np.zeros((N, N), dtype=np.complex64)
    for px, py, am in zip(ipx, ipy, amps):
        out += np.complex64(am) * psf[N - py:2 * N - py, N - px:2 * N - px]
    return out.astype(np.complex128)


def autofocus_hologram(N, seed, index, z=None, n_pts=24, radius_px=32.0, pitch=20e-6, lam=852e-9,
                       bits=12, ref_ratio=10.0, mean_fraction=0.30):
    """One off-axis hologram of a sparse point-scatterer object for the autofocus
    workload, and the object distance z it was recorded at.

    The object: n_pts scatterers at pixel centres in a disk of radius radius_px
    pixels (a fixed physical size, whatever N), amplitudes 0.25 or 1 (30 % bright: amplitude
    structure, so that the in-focus image has contrast) with uniform random
    phases, at z ~ U[0.10, 0.60] m unless z is given. Sensor field, reference,
    scaling and Poisson noise follow the stream scenes of this module. Hologram
    `index` of set `seed` depends only on (seed, index).
    """
    rng = np.random.Generator(np.random.PCG64([seed, index]))
    if z is None:
        z = AF_Z_RANGE[0] + (AF_Z_RANGE[1] - AF_Z_RANGE[0]) * rng.random()
    rad = radius_px * np.sqrt(rng.random(n_pts))
    ang = 2.0 * np.pi * rng.random(n_pts)
    ipx = np.rint(N / 2 + rad * np.cos(ang)).astype(np.int64)
    ipy = np.rint(N / 2 + rad * np.sin(ang)).astype(np.int64)
    amp = (0.25 + 0.75 * (rng.random(n_pts) < 0.3)) * np.exp(2j * np.pi * rng.random(n_pts))
    f = _pixel_point_field(N, pitch, lam, z, ipx, ipy, amp)
    f /= np.sqrt(np.mean(np.abs(f) ** 2))
    c = np.arange(N)
    ref = np.sqrt(ref_ratio) * np.exp(1j * 2.0 * np.pi * (c[None, :] + c[:, None]) / 4.0)
    inten = np.abs(ref + f) ** 2
    full = (1 << bits) - 1
    inten *= mean_fraction * full / inten.mean()
    inten = rng.poisson(inten).astype(np.float64)
    np.clip(inten, 0, full, out=inten)
    return inten.astype(np.uint16 if bits > 8 else np.uint8), float(z)


def _af_chunk(args):
    N, seed, lo, hi = args
    fr = np.empty((hi - lo, N, N), dtype=np.uint16)
    zs = np.empty(hi - lo)
    for i in range(lo, hi):
        fr[i - lo], zs[i - lo] = autofocus_hologram(N, seed, i)
    return lo, fr, zs


def autofocus_set(n, N=256, seed=1004, workers=1):
    """Holograms 0..n-1 of set `seed` (uint16, (n, N, N)) and their distances z.
    workers > 1 spreads the work over a spawn-started process pool (start it
    before any CUDA call: a forked child of a CUDA process can hang)."""
    frames = np.empty((n, N, N), dtype=np.uint16)
    zs = np.empty(n)
    step = max(1, min(256, -(-n // max(1, workers * 4))))
    jobs = [(N, seed, lo, min(n, lo + step)) for lo in range(0, n, step)]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            for lo, fr, z in pool.imap_unordered(_af_chunk, jobs):
                frames[lo:lo + len(z)] = fr
                zs[lo:lo + len(z)] = z
    else:
        for job in jobs:
            lo, fr, z = _af_chunk(job)
            frames[lo:lo + len(z)] = fr
            zs[lo:lo + len(z)] = z
    return frames, zs

