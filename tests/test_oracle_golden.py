"""The oracle still reproduces its committed regression fixture."""
import json
import os

import numpy as np
import pytest

from oracle import hv_oracle as O
from paper_2508_03911_gb300 import synth

PATH = os.path.join(os.path.dirname(__file__), "golden", "oracle_small.json")
GOLD = json.load(open(PATH))
NAMES = [k for k in GOLD if not k.startswith("_")]


@pytest.mark.parametrize("name", NAMES)
def test_oracle_matches_golden(name):
    c = GOLD[name]
    f = c["frames"]
    fr = synth.random_frames(f["n"], f["H"], f["W"], f["bits"], f["seed"])
    img = O.render(fr, c["params"])
    r = c["result"]
    assert list(img.shape) == r["shape"]
    assert img.sum() == pytest.approx(r["sum"], rel=1e-12)
    np.testing.assert_allclose(img.ravel()[r["idx"]], r["val"], rtol=1e-11)
