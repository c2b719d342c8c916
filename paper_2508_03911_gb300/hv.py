"""Python binding of the C ABI in include/hv.h (ctypes; argument marshalling only).

Every step of the rendering path runs in the CUDA kernels of libhv.so. There is
no Python or CPU fallback: importing this module on a machine without the built
library raises, and so does opening a handle without a CUDA device.

The functions carry the C names (hv_open, hv_set_params, hv_push_frames,
hv_render, hv_close, ...). `Renderer` is a small convenience wrapper.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhv.so")

HV_OK, HV_ERR_ARG, HV_ERR_STATE, HV_ERR_QUEUE_FULL = 0, -1, -2, -3
HV_ERR_NOMEM, HV_ERR_CUDA, HV_ERR_TIMEOUT, HV_ERR_UNSUPPORTED = -4, -5, -6, -7
HV_MEM_HOST, HV_MEM_DEVICE, HV_MEM_HOST_ASYNC, HV_MEM_DEVICE_ASYNC = 0, 1, 2, 3
HV_SPATIAL_NONE, HV_SPATIAL_ASP, HV_SPATIAL_FRESNEL = 0, 1, 2
HV_TEMPORAL_STFT, HV_TEMPORAL_PCA, HV_TEMPORAL_NONE = 0, 1, 2
HV_MOM_M0, HV_MOM_M1, HV_MOM_M2, HV_MOM_M1N, HV_MOM_M2N = 1, 2, 4, 8, 16
HV_PREC_FP32, HV_PREC_BF16, HV_PREC_SPLIT_BF16 = 0, 1, 2
HV_INJECT_NONE, HV_INJECT_FUSED_STALL = 0, 1

STATUS_NAMES = {0: "HV_OK", -1: "HV_ERR_ARG", -2: "HV_ERR_STATE", -3: "HV_ERR_QUEUE_FULL",
                -4: "HV_ERR_NOMEM", -5: "HV_ERR_CUDA", -6: "HV_ERR_TIMEOUT",
                -7: "HV_ERR_UNSUPPORTED"}
MOMENT_BITS = {"M0": HV_MOM_M0, "M1": HV_MOM_M1, "M2": HV_MOM_M2, "M1N": HV_MOM_M1N,
               "M2N": HV_MOM_M2N}
SPATIAL = {"none": HV_SPATIAL_NONE, "asp": HV_SPATIAL_ASP, "fresnel": HV_SPATIAL_FRESNEL}
TEMPORAL = {"stft": HV_TEMPORAL_STFT, "pca": HV_TEMPORAL_PCA, "none": HV_TEMPORAL_NONE}
PRECISION = {"fp32": HV_PREC_FP32, "bf16": HV_PREC_BF16, "split_bf16": HV_PREC_SPLIT_BF16}


class hv_open_desc(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("device", C.c_int32), ("max_width", C.c_uint32),
                ("max_height", C.c_uint32), ("pixel_bits", C.c_uint32),
                ("queue_capacity_frames", C.c_uint32), ("time_queue_frames", C.c_uint32),
                ("reserved", C.c_uint32), ("stream", C.c_void_p)]


class hv_params(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("width", C.c_uint32), ("height", C.c_uint32),
                ("spatial", C.c_int32), ("fftshift", C.c_int32), ("z_m", C.c_double),
                ("lambda_m", C.c_double), ("pitch_x_m", C.c_double), ("pitch_y_m", C.c_double),
                ("temporal", C.c_int32), ("T", C.c_uint32), ("stride", C.c_uint32),
                ("moments_mask", C.c_uint32), ("fs_hz", C.c_double),
                ("band_lo_bin", C.c_uint32), ("band_hi_bin", C.c_uint32),
                ("band_lo_hz", C.c_double), ("band_hi_hz", C.c_double),
                ("pca_lo", C.c_uint32), ("pca_hi", C.c_uint32), ("precision", C.c_int32),
                ("tuned", C.c_int32), ("spatial_chunk", C.c_uint32), ("spatial_kernel", C.c_uint32),
                ("highpass_cpp", C.c_double), ("stft_kernel", C.c_int32), ("reserved", C.c_uint32)]


class hv_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("frames_pushed", "frames_rejected", "frames_dropped",
                                          "frames_propagated", "windows_rendered",
                                          "kernel_launches")]


class hv_profile(C.Structure):
    _fields_ = [("spatial_ms", C.c_double), ("temporal_ms", C.c_double), ("renders", C.c_uint64),
                ("frames", C.c_uint64), ("windows", C.c_uint64), ("pca_cov_ms", C.c_double),
                ("pca_eig_ms", C.c_double), ("pca_proj_ms", C.c_double),
                ("pca_sweeps", C.c_uint64), ("pca_sweeps_f32", C.c_uint64)]


class hv_peaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("fp64_tflops", C.c_double), ("sm_count", C.c_int),
                ("sm_clock_khz", C.c_int)]


class hv_tuning(C.Structure):
    _fields_ = [("tuned", C.c_int32), ("spatial_kernel", C.c_int32), ("spatial_chunk", C.c_uint32),
                ("stft_kernel", C.c_int32), ("candidate_us_per_frame", C.c_float * 12),
                ("stft_us_per_window", C.c_float * 6)]


class hv_post(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("kernel_size", C.c_uint32), ("kernel", C.c_void_p),
                ("gauss_sigma", C.c_float), ("renormalize", C.c_int32), ("accumulate", C.c_uint32),
                ("reserved", C.c_uint32)]


class hv_holo_header(C.Structure):
    _fields_ = [("version", C.c_uint16), ("bits_per_pixel", C.c_uint16), ("width", C.c_uint32),
                ("height", C.c_uint32), ("n_images", C.c_uint32), ("data_bytes", C.c_uint64),
                ("endianness", C.c_uint8), ("data_type", C.c_uint8), ("reserved", C.c_uint8 * 6)]


class hv_group_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("steps", "graph_launches", "graph_instantiations",
                                          "graph_updates", "kernel_launches")] + \
               [("capture_us_last", C.c_double)]


class HvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load libhv.so (built by paper_2508_03911_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2508_03911_gb300.build` "
                          "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    sig = {
        "hv_open": ([P(hv_open_desc), P(C.c_void_p)], C.c_int),
        "hv_set_params": ([C.c_void_p, P(hv_params)], C.c_int),
        "hv_get_params": ([C.c_void_p, P(hv_params)], C.c_int),
        "hv_push_frames": ([C.c_void_p, C.c_void_p, C.c_uint32, C.c_int], C.c_int),
        "hv_render": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, P(C.c_uint32)], C.c_int),
        "hv_window_floats": ([C.c_void_p, P(C.c_size_t)], C.c_int),
        "hv_pca_eigenvalues": ([C.c_void_p, P(C.c_double), C.c_uint32], C.c_int),
        "hv_get_stats": ([C.c_void_p, P(hv_stats)], C.c_int),
        "hv_get_tuning": ([C.c_void_p, P(hv_tuning)], C.c_int),
        "hv_synchronize": ([C.c_void_p], C.c_int),
        "hv_debug_inject": ([C.c_void_p, C.c_int], C.c_int),
        "hv_profile_enable": ([C.c_void_p, C.c_int], C.c_int),
        "hv_profile_read": ([C.c_void_p, P(hv_profile)], C.c_int),
        "hv_close": ([C.c_void_p], C.c_int),
        "hv_last_error": ([C.c_void_p], C.c_char_p),
        "hv_group_open": ([P(C.c_void_p), C.c_uint32, C.c_void_p, C.c_int, P(C.c_void_p)], C.c_int),
        "hv_render_group": ([C.c_void_p, P(C.c_void_p), P(C.c_uint32), P(C.c_void_p), P(C.c_size_t),
                             P(C.c_uint32)], C.c_int),
        "hv_group_get_stats": ([C.c_void_p, P(hv_group_stats)], C.c_int),
        "hv_group_last_error": ([C.c_void_p], C.c_char_p),
        "hv_group_close": ([C.c_void_p], C.c_int),
        "hv_set_postprocess": ([C.c_void_p, P(hv_post)], C.c_int),
        "hv_holo_read_header": ([C.c_char_p, P(hv_holo_header)], C.c_int),
        "hv_holo_read_frames": ([C.c_char_p, C.c_uint64, C.c_uint32, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
        "hv_holo_read_footer": ([C.c_char_p, C.c_char_p, C.c_size_t, P(C.c_size_t)], C.c_int),
        "hv_holo_write": ([C.c_char_p, P(hv_holo_header), C.c_void_p, C.c_char_p], C.c_int),
        "hv_focus_sweep": ([C.c_void_p, C.c_void_p, C.c_uint32, P(C.c_double), C.c_uint32, C.c_void_p],
                           C.c_int),
        "hv_af_features": ([C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p], C.c_int),
        "hv_version": ([], C.c_char_p),
        "hv_probe_peaks": ([C.c_int, C.c_void_p, P(hv_peaks)], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def exported_symbols() -> list[str]:
    return [n for n in dir(lib()) if n.startswith("hv_")]


def _check(h, status):
    if status != HV_OK:
        msg = lib().hv_last_error(h).decode(errors="replace")
        raise HvError(status, msg)
    return status


# ------------------------------------------------------------ C-named calls

def hv_open(max_width, max_height, pixel_bits, queue_capacity_frames, device=0,
            time_queue_frames=0, stream=None) -> C.c_void_p:
    d = hv_open_desc(C.sizeof(hv_open_desc), device, max_width, max_height, pixel_bits,
                     queue_capacity_frames, time_queue_frames, 0, stream)
    h = C.c_void_p()
    _check(None, lib().hv_open(C.byref(d), C.byref(h)))
    return h


def make_params(width, height, spatial="asp", z=0.3, lam=852e-9, pitch=20e-6, pitch_y=None,
                fftshift=1, temporal="stft", T=64, stride=None, fs=20000.0, band=(4, 28),
                band_hz=None, moments=("M0",), pca=(2, 64), precision="fp32", tuned=0,
                spatial_chunk=0, spatial_kernel="auto", highpass=0.0, stft_kernel="auto") -> hv_params:
    p = hv_params()
    p.struct_size = C.sizeof(hv_params)
    p.width, p.height = width, height
    p.spatial = SPATIAL[spatial]
    p.fftshift = int(fftshift)
    p.z_m, p.lambda_m = z, lam
    p.pitch_x_m = pitch
    p.pitch_y_m = pitch if pitch_y is None else pitch_y
    p.temporal = TEMPORAL[temporal]
    p.T = T
    p.stride = T if stride is None else stride
    p.moments_mask = sum(MOMENT_BITS[m] for m in moments)
    p.fs_hz = fs
    p.band_lo_bin, p.band_hi_bin = band
    if band_hz is not None:
        p.band_lo_hz, p.band_hi_hz = band_hz
    p.pca_lo, p.pca_hi = pca
    p.precision = PRECISION[precision]
    p.tuned = int(tuned)
    p.spatial_chunk = spatial_chunk
    p.spatial_kernel = {"auto": 0, "multipass": 1, "cluster": 2, "persistent": 3, "fused": 4}[spatial_kernel]
    p.highpass_cpp = highpass
    p.stft_kernel = {"auto": 0, "walk": 1, "window": 2, "window_wide": 3, "window_pipelined": 4,
                     "window_tma": 5, "window_tma_pipelined": 6}[stft_kernel]
    return p


def hv_set_params(h, p: hv_params):
    _check(h, lib().hv_set_params(h, C.byref(p)))


def hv_get_params(h) -> hv_params:
    p = hv_params()
    _check(h, lib().hv_get_params(h, C.byref(p)))
    return p


def _ptr_kind(x):
    """(pointer, mem_kind, nbytes) of a torch tensor (cpu or cuda) or numpy array."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, HV_MEM_HOST, x.nbytes
    # torch tensor (imported lazily: torch is plumbing only)
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    kind = HV_MEM_DEVICE if x.is_cuda else HV_MEM_HOST
    return x.data_ptr(), kind, x.numel() * x.element_size()


def hv_push_frames(h, frames, n=None, async_=False) -> int:
    """Push frames (numpy / torch, shape (n, H, W), uint8 or uint16). async_: a host
    source's copy is only queued on the copy stream (HV_MEM_HOST_ASYNC); a device
    source, whose frames must be complete already, is read in place by the spatial
    stage (HV_MEM_DEVICE_ASYNC); keep it unchanged until its windows are rendered
    and hv_synchronize has returned.
    Returns the status (HV_OK or HV_ERR_QUEUE_FULL); other errors raise."""
    ptr, kind, _ = _ptr_kind(frames)
    if async_:
        kind = HV_MEM_HOST_ASYNC if kind == HV_MEM_HOST else HV_MEM_DEVICE_ASYNC
    n = frames.shape[0] if n is None else n
    s = lib().hv_push_frames(h, C.c_void_p(ptr), n, kind)
    if s not in (HV_OK, HV_ERR_QUEUE_FULL):
        _check(h, s)
    return s


def hv_render(h, out, async_=False) -> int:
    """Render into `out` (float32 numpy / torch, host or device). async_: a host
    output is only queued (valid after hv_synchronize). Returns windows."""
    ptr, kind, nbytes = _ptr_kind(out)
    if async_ and kind == HV_MEM_HOST:
        kind = HV_MEM_HOST_ASYNC
    n = C.c_uint32(0)
    _check(h, lib().hv_render(h, C.c_void_p(ptr), nbytes // 4, kind, C.byref(n)))
    return n.value


def hv_window_floats(h) -> int:
    f = C.c_size_t(0)
    _check(h, lib().hv_window_floats(h, C.byref(f)))
    return f.value


def hv_pca_eigenvalues(h, n) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _check(h, lib().hv_pca_eigenvalues(h, out.ctypes.data_as(C.POINTER(C.c_double)), n))
    return out


def hv_get_stats(h) -> dict:
    s = hv_stats()
    _check(h, lib().hv_get_stats(h, C.byref(s)))
    return {n: getattr(s, n) for n, _ in hv_stats._fields_}


def hv_profile_enable(h, on=True):
    _check(h, lib().hv_profile_enable(h, int(on)))


def hv_profile_read(h) -> dict:
    p = hv_profile()
    _check(h, lib().hv_profile_read(h, C.byref(p)))
    return {n: getattr(p, n) for n, _ in hv_profile._fields_}


def hv_get_tuning(h) -> dict:
    t = hv_tuning()
    _check(h, lib().hv_get_tuning(h, C.byref(t)))
    return {"tuned": t.tuned, "spatial_kernel": t.spatial_kernel, "spatial_chunk": t.spatial_chunk,
            "candidate_us_per_frame": list(t.candidate_us_per_frame), "stft_kernel": t.stft_kernel,
            "stft_us_per_window": list(t.stft_us_per_window)}


def hv_synchronize(h):
    _check(h, lib().hv_synchronize(h))


def hv_debug_inject(h, what: int):
    _check(h, lib().hv_debug_inject(h, what))


def hv_close(h):
    lib().hv_close(h)


def hv_last_error(h=None) -> str:
    return lib().hv_last_error(h).decode(errors="replace")


def hv_version() -> str:
    return lib().hv_version().decode()


def hv_probe_peaks(device=0, stream=None) -> dict:
    """Measured FP32 / FP64 FMA throughput of the device (TFLOP/s)."""
    p = hv_peaks()
    s = lib().hv_probe_peaks(device, C.c_void_p(stream or 0), C.byref(p))
    if s != HV_OK:
        raise HvError(s, "hv_probe_peaks failed")
    return {n: getattr(p, n) for n, _ in hv_peaks._fields_}


def hv_set_postprocess(h, kernel=None, kernel_size=None, sigma=0.0, renormalize=False, accumulate=1):
    """Post-processing of rendered images: a K x K kernel (array) or a Gaussian of
    `sigma` with `kernel_size`, re-normalisation, moving average over `accumulate`."""
    k = None
    if kernel is not None:
        k = np.ascontiguousarray(kernel, dtype=np.float32)
        kernel_size = k.shape[0]
    p = hv_post(C.sizeof(hv_post), int(kernel_size or 0), C.c_void_p(k.ctypes.data if k is not None else 0),
                float(sigma), int(bool(renormalize)), int(accumulate), 0)
    _check(h, lib().hv_set_postprocess(h, C.byref(p)))


# -------------------------------------------------------------- .holo files

def _holo_check(s, what):
    if s != HV_OK:
        raise HvError(s, what)


def holo_read_header(path) -> dict:
    h = hv_holo_header()
    _holo_check(lib().hv_holo_read_header(os.fsencode(path), C.byref(h)), f"cannot read the header of {path}")
    return {n: getattr(h, n) for n, _ in hv_holo_header._fields_ if n != "reserved"}


def holo_read_frames(path, first, out, stream=None):
    """Frames first .. first + len(out) - 1 into `out` (numpy array or torch tensor,
    host or device, shape (n, H, W) of the file's pixel type)."""
    ptr, kind, _ = _ptr_kind(out)
    _holo_check(lib().hv_holo_read_frames(os.fsencode(path), first, out.shape[0], C.c_void_p(ptr), kind,
                                          C.c_void_p(stream or 0)), f"cannot read frames of {path}")


def holo_read_footer(path) -> str:
    n = C.c_size_t(0)
    _holo_check(lib().hv_holo_read_footer(os.fsencode(path), None, 0, C.byref(n)), f"cannot read {path}")
    buf = C.create_string_buffer(n.value + 1)
    _holo_check(lib().hv_holo_read_footer(os.fsencode(path), buf, n.value + 1, C.byref(n)), f"cannot read {path}")
    return buf.value.decode()


def holo_write(path, frames: np.ndarray, footer=None, data_type=0):
    """Write frames (n, H, W) uint8/uint16/float32 host array and an optional JSON footer."""
    a = np.ascontiguousarray(frames)
    h = hv_holo_header(7, a.dtype.itemsize * 8, a.shape[2], a.shape[1], a.shape[0], a.nbytes, 0, data_type)
    _holo_check(lib().hv_holo_write(os.fsencode(path), C.byref(h), C.c_void_p(a.ctypes.data),
                                    footer.encode() if footer is not None else None), f"cannot write {path}")


# --------------------------------------------------------------- autofocus

def hv_focus_sweep(h, frames, z, metric):
    """Tamura coefficient of every (frame, distance): frames a device tensor
    (n, H, W), z a sequence of distances, metric a float32 device tensor (n, nz)."""
    ptr, kind, _ = _ptr_kind(frames)
    mptr, mkind, mbytes = _ptr_kind(metric)
    if kind != HV_MEM_DEVICE or mkind != HV_MEM_DEVICE:
        raise ValueError("frames and metric must be device memory")
    zz = np.ascontiguousarray(z, dtype=np.float64)
    n = frames.shape[0]
    if mbytes < n * zz.size * 4:
        raise ValueError("metric too small")
    _check(h, lib().hv_focus_sweep(h, C.c_void_p(ptr), n, zz.ctypes.data_as(C.POINTER(C.c_double)),
                                   zz.size, C.c_void_p(mptr)))


def hv_af_features(h, frames, out):
    """Network inputs (n, H/2, W/2) as bfloat16 bit patterns into the device tensor out
    (torch.int16 or torch.bfloat16, n * H/2 * W/2 elements)."""
    ptr, kind, _ = _ptr_kind(frames)
    optr, okind, obytes = _ptr_kind(out)
    if kind != HV_MEM_DEVICE or okind != HV_MEM_DEVICE:
        raise ValueError("frames and out must be device memory")
    n, H, W = frames.shape
    if obytes < n * (H // 2) * (W // 2) * 2:
        raise ValueError("out too small")
    _check(h, lib().hv_af_features(h, C.c_void_p(ptr), n, C.c_void_p(optr)))


# ------------------------------------------------------------------ groups

def _gcheck(g, status):
    if status != HV_OK:
        raise HvError(status, lib().hv_group_last_error(g).decode(errors="replace"))
    return status


def hv_group_open(handles, stream=None, use_graph=True) -> C.c_void_p:
    """Group over open handles; `stream` is a cudaStream_t handle (int) or None."""
    arr = (C.c_void_p * len(handles))(*[C.c_void_p(h.value if isinstance(h, C.c_void_p) else h)
                                        for h in handles])
    g = C.c_void_p()
    s = lib().hv_group_open(arr, len(handles), C.c_void_p(stream or 0), int(use_graph), C.byref(g))
    if s != HV_OK:
        raise HvError(s, "hv_group_open failed")
    return g


def hv_render_group(g, frames, outs) -> list[int]:
    """One batch: frames[i] (device tensor (n, H, W) or None) pushed to member i,
    then its complete windows rendered into the device tensor outs[i]. Returns
    the windows rendered per member."""
    n = len(outs)
    fp = (C.c_void_p * n)()
    nf = (C.c_uint32 * n)()
    op = (C.c_void_p * n)()
    cap = (C.c_size_t * n)()
    for i in range(n):
        if frames is not None and frames[i] is not None:
            ptr, kind, _ = _ptr_kind(frames[i])
            if kind != HV_MEM_DEVICE:
                raise ValueError("group frames must be device memory")
            fp[i] = ptr
            nf[i] = frames[i].shape[0]
        ptr, kind, nbytes = _ptr_kind(outs[i])
        if kind != HV_MEM_DEVICE:
            raise ValueError("group outputs must be device memory")
        op[i] = ptr
        cap[i] = nbytes // 4
    nw = (C.c_uint32 * n)()
    _gcheck(g, lib().hv_render_group(g, fp, nf, op, cap, nw))
    return list(nw)


def hv_group_get_stats(g) -> dict:
    st = hv_group_stats()
    _gcheck(g, lib().hv_group_get_stats(g, C.byref(st)))
    return {n: getattr(st, n) for n, _ in hv_group_stats._fields_}


def hv_group_close(g):
    lib().hv_group_close(g)


class Renderer:
    """Owns one handle. `params` keywords are those of make_params."""

    def __init__(self, max_width, max_height, pixel_bits, queue_capacity_frames, device=0,
                 time_queue_frames=0, stream=None):
        self.h = hv_open(max_width, max_height, pixel_bits, queue_capacity_frames, device,
                         time_queue_frames, stream)

    def set_params(self, width, height, **kw):
        hv_set_params(self.h, make_params(width, height, **kw))

    def push(self, frames, async_=False):
        return hv_push_frames(self.h, frames, async_=async_)

    def render(self, out, async_=False):
        return hv_render(self.h, out, async_=async_)

    def window_floats(self):
        return hv_window_floats(self.h)

    def stats(self):
        return hv_get_stats(self.h)

    def synchronize(self):
        hv_synchronize(self.h)

    def close(self):
        if self.h is not None:
            hv_close(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
