"""File-mode input: a .holo recording read straight into device memory (pinned
bounce buffer) and rendered, against the oracle on the same frames."""
import numpy as np
import pytest

from oracle import hv_oracle as O
from paper_2508_03911_gb300 import hv, synth
from tests._util import oracle_params, rel_l2, to_hv

pytestmark = pytest.mark.gpu


def test_holo_file_replay(tmp_path):
    import torch
    sc = synth.build(synth.scene_tiny_asp_stft(N=64))
    fr = synth.frames(sc, 0, 128)
    path = tmp_path / "rec.holo"
    hv.holo_write(path, fr, footer='{"spatial": "asp", "z_m": 0.3}')
    h = hv.holo_read_header(path)
    dev = torch.empty((h["n_images"], h["height"], h["width"]), dtype=torch.uint8, device="cuda")
    hv.holo_read_frames(path, 0, dev)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), fr)
    p = oracle_params(H=64, W=64)
    r = hv.Renderer(64, 64, 8, 128)
    try:
        hv.hv_set_params(r.h, to_hv(p))
        assert r.push(dev) == hv.HV_OK
        out = torch.zeros(4 * r.window_floats(), device="cuda")
        n = r.render(out)
        torch.cuda.synchronize()
    finally:
        r.close()
    img = out.cpu().numpy()[: n * 64 * 64].reshape(n, 1, 64, 64)
    ref = O.render(fr, p)
    assert img.shape == ref.shape
    for w in range(n):
        assert rel_l2(img[w, 0], ref[w, 0]) <= 1e-4
