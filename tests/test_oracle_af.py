"""Pins of the autofocus oracle: convolution against its brute-force definition,
back-propagation against central finite differences, Adam against its closed
first step, bf16 rounding on exact ties, the feature against a fringe whose
spectrum is known, the network head against a closed form, and the sweep
against the distance the generator recorded the hologram at (spherical waves,
not the ASP the sweep uses)."""
import math

import numpy as np
import pytest

from oracle import af_oracle as A
from oracle import hv_oracle as O
from paper_2508_03911_gb300 import synth


def brute_conv(x, w, b):
    n, c, H, W = x.shape
    o = w.shape[0]
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    y = np.zeros((n, o, Ho, Wo))
    for a in range(n):
        for q in range(o):
            for i in range(Ho):
                for j in range(Wo):
                    s = b[q]
                    for ch in range(c):
                        for di in range(3):
                            for dj in range(3):
                                yy, xx = 2 * i + di - 1, 2 * j + dj - 1
                                if 0 <= yy < H and 0 <= xx < W:
                                    s += w[q, ch, di, dj] * x[a, ch, yy, xx]
                    y[a, q, i, j] = s
    return y


@pytest.mark.parametrize("shape", [(2, 3, 6, 6), (1, 2, 5, 7), (1, 1, 8, 4)])
def test_conv_matches_brute_force(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape)
    w = rng.standard_normal((4, shape[1], 3, 3))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(A.conv_s2(x, w, b), brute_conv(x, w, b), rtol=1e-12, atol=1e-12)


def _tiny_problem(seed=3, n=3, side=16):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 1, side, side))
    z = rng.uniform(0.1, 0.6, n)
    flat = A.init_params(seed)
    flat += 0.05 * rng.standard_normal(flat.shape)  # non-zero biases too
    return flat, x, z


def test_gradients_match_finite_differences_directional():
    flat, x, z = _tiny_problem()
    L, g = A.gradients(flat, x, z)
    assert abs(L - A.loss(flat, x, z)) < 1e-14
    rng = np.random.default_rng(11)
    for _ in range(6):
        d = rng.standard_normal(flat.shape)
        eps = 1e-6
        fd = (A.loss(flat + eps * d, x, z) - A.loss(flat - eps * d, x, z)) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd)), (fd, g @ d)


def test_gradients_match_finite_differences_per_tensor():
    flat, x, z = _tiny_problem(seed=5)
    _, g = A.gradients(flat, x, z)
    rng = np.random.default_rng(2)
    o = 0
    for name, s in A.param_shapes():
        n = int(np.prod(s))
        for k in rng.choice(n, size=min(n, 4), replace=False):
            e = np.zeros_like(flat)
            e[o + k] = 1e-6
            fd = (A.loss(flat + e, x, z) - A.loss(flat - e, x, z)) / 2e-6
            assert abs(fd - g[o + k]) <= 1e-6 + 1e-5 * abs(fd), (name, k, fd, g[o + k])
        o += n
    assert o == A.n_params() == flat.size


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(0)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p1, m, v = A.adam_step(p0, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    np.testing.assert_allclose(p1, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_rounding_ties_to_even():
    one = 1.0
    cases = {one: one, one + 2.0 ** -8: one, one + 3 * 2.0 ** -8: one + 2.0 ** -6,
             one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7, -2.5: -2.5, 0.0: 0.0}
    for v, want in cases.items():
        assert A.bf16(np.array([v]))[0] == want, (v, A.bf16(np.array([v]))[0], want)


def test_features_of_a_fringe():
    N, kx = 64, 10
    x = np.arange(N)
    fr = (1000 + 500 * np.cos(2 * np.pi * kx * x / N))[None, :].repeat(N, 0).astype(np.uint16)
    f = A.features(fr)
    assert f.shape == (N // 2, N // 2)
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1) < 1e-12
    # the fringe's two bins (row N/2, columns N/2 +- kx) fall in binned cells
    # (N/4, (N/2 +- kx) / 2); the DC bin is zero after the mean is removed
    top = sorted(np.argsort(f.ravel())[-2:])
    want = sorted([(N // 4) * (N // 2) + (N // 2 - kx) // 2, (N // 4) * (N // 2) + (N // 2 + kx) // 2])
    assert top == want


def test_head_closed_form():
    flat = np.zeros(A.n_params())
    p = A.unflatten(flat)
    p["b4"][:] = np.linspace(-1, 1, 64)          # a4 = relu(b4) everywhere
    p["f1w"][:] = 0.01
    p["f1b"][:] = -0.05
    p["f2w"][:] = 0.5
    p["f2b"][:] = 0.2
    flat = A.flatten(p)
    x = np.random.default_rng(0).standard_normal((2, 1, 16, 16))
    y, acts = A.forward(flat, x)
    g = np.maximum(np.linspace(-1, 1, 64), 0)
    h = np.maximum(0.01 * g.sum() - 0.05, 0)
    np.testing.assert_allclose(y, 0.5 * 32 * h + 0.2, rtol=1e-12)


def test_tamura_of_a_spike():
    img = np.zeros((8, 8))
    img[3, 4] = 7.0
    assert abs(O.tamura(img) - math.sqrt(math.sqrt(63))) < 1e-12


@pytest.mark.slow
def test_sweep_finds_the_recorded_distance():
    """The sweep's maximum lies within one step of the distance the generator used."""
    fr, z = synth.autofocus_hologram(256, 1006, 0, z=0.27)
    j, zj = A.focus_label(fr, 852e-9, 20e-6, 20e-6)
    assert abs(zj - z) <= (A.Z1 - A.Z0) / (A.NZ - 1), (zj, z)
