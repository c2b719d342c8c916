""".holo files: the reader and writer against a header packed by hand from the
field list of the paper's "Holofile system" section (magic, version 7, bits per
pixel, width, height, images, data size, endianness, data type, padding to 64
bytes), byte-exact frames and footer, big-endian data, and malformed files."""
import struct

import numpy as np
import pytest

from paper_2508_03911_gb300 import hv


def packed(frames: np.ndarray, footer: bytes = b"", version=7, endian=0, dtype_flag=0, bits=None,
           data_bytes=None, magic=b"HOLO") -> bytes:
    n, H, W = frames.shape
    bits = frames.dtype.itemsize * 8 if bits is None else bits
    nbytes = frames.nbytes if data_bytes is None else data_bytes
    hdr = struct.pack("<4sHHIIIQBB", magic, version, bits, W, H, n, nbytes, endian, dtype_flag)
    hdr += b"\0" * (64 - len(hdr))
    assert len(hdr) == 64
    data = frames.astype(frames.dtype.newbyteorder(">")).tobytes() if endian else frames.tobytes()
    return hdr + data + footer


def test_reader_parses_a_hand_packed_file(tmp_path):
    fr = np.random.default_rng(0).integers(0, 4096, (5, 12, 20)).astype(np.uint16)
    p = tmp_path / "a.holo"
    p.write_bytes(packed(fr, b'{"z": 0.3}'))
    h = hv.holo_read_header(p)
    assert (h["version"], h["bits_per_pixel"], h["width"], h["height"], h["n_images"]) == (7, 16, 20, 12, 5)
    assert h["data_bytes"] == fr.nbytes and h["endianness"] == 0 and h["data_type"] == 0
    out = np.zeros((3, 12, 20), dtype=np.uint16)
    hv.holo_read_frames(p, 1, out)
    assert np.array_equal(out, fr[1:4])
    assert hv.holo_read_footer(p) == '{"z": 0.3}'


def test_writer_matches_the_documented_layout(tmp_path):
    fr = np.random.default_rng(1).integers(0, 256, (4, 8, 16)).astype(np.uint8)
    p = tmp_path / "w.holo"
    hv.holo_write(p, fr, footer='{"a": 1}')
    assert p.read_bytes() == packed(fr, b'{"a": 1}')
    hv.holo_write(p, fr)
    assert p.read_bytes() == packed(fr)
    assert hv.holo_read_footer(p) == ""


def test_big_endian_pixels_are_swapped(tmp_path):
    fr = np.array([[[0x0102, 0xA0B0], [0x0FFF, 7]]], dtype=np.uint16)
    p = tmp_path / "b.holo"
    p.write_bytes(packed(fr, endian=1))
    out = np.zeros_like(fr)
    hv.holo_read_frames(p, 0, out)
    assert np.array_equal(out, fr)


@pytest.mark.parametrize("kw,status", [
    (dict(magic=b"HOLA"), hv.HV_ERR_ARG),
    (dict(version=6), hv.HV_ERR_UNSUPPORTED),
    (dict(bits=12), hv.HV_ERR_ARG),
    (dict(data_bytes=10), hv.HV_ERR_ARG),
    (dict(endian=2), hv.HV_ERR_ARG),
])
def test_malformed_headers_are_rejected(tmp_path, kw, status):
    fr = np.zeros((2, 4, 4), dtype=np.uint16)
    p = tmp_path / "m.holo"
    p.write_bytes(packed(fr, **kw))
    with pytest.raises(hv.HvError) as ei:
        hv.holo_read_header(p)
    assert ei.value.status == status


def test_truncated_file_and_range_errors(tmp_path):
    fr = np.zeros((3, 4, 4), dtype=np.uint16)
    p = tmp_path / "t.holo"
    p.write_bytes(packed(fr)[:-5])
    with pytest.raises(hv.HvError):
        hv.holo_read_header(p)
    p.write_bytes(packed(fr))
    with pytest.raises(hv.HvError):
        hv.holo_read_frames(p, 2, np.zeros((2, 4, 4), dtype=np.uint16))
    with pytest.raises(hv.HvError):
        hv.holo_read_header(tmp_path / "missing.holo")
