"""Pins of the oracle's post-processing (convolution, re-normalisation, moving
average): identities, the wrapped and rotated copy a point image produces,
brute-force modular sums, and closed forms of the moving average."""
import numpy as np
import pytest

from oracle import hv_oracle as O


def test_delta_kernel_is_identity():
    img = np.random.default_rng(0).standard_normal((8, 12))
    k = np.zeros((3, 3))
    k[1, 1] = 1.0
    np.testing.assert_allclose(O.convolve_periodic(img, k), img, rtol=0, atol=1e-15)


@pytest.mark.parametrize("K,y0,x0", [(3, 0, 5), (5, 6, 0), (5, 1, 9)])
def test_point_image_gives_rotated_wrapped_kernel(K, y0, x0):
    H, W = 7, 10
    img = np.zeros((H, W))
    img[y0, x0] = 1.0
    k = np.arange(K * K, dtype=np.float64).reshape(K, K) + 1.0  # no symmetry
    out = O.convolve_periodic(img, k)
    c = K // 2
    want = np.zeros((H, W))
    for d in range(-c, c + 1):
        for e in range(-c, c + 1):
            want[(y0 + d) % H, (x0 + e) % W] += k[c - d, c - e]
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)


def test_matches_modular_double_loop():
    rng = np.random.default_rng(3)
    img = rng.standard_normal((5, 6))
    k = rng.standard_normal((3, 3))
    out = O.convolve_periodic(img, k)
    for y in range(5):
        for x in range(6):
            s = sum(k[a, b] * img[(y + a - 1) % 5, (x + b - 1) % 6] for a in range(3) for b in range(3))
            assert abs(out[y, x] - s) < 1e-12


def test_gaussian_kernel_and_sum_preservation():
    g = O.gaussian_kernel(7, 1.3)
    assert abs(g.sum() - 1) < 1e-15 and np.allclose(g, g.T) and np.allclose(g, g[::-1, ::-1])
    assert g[3, 3] == g.max()
    np.testing.assert_allclose(g[3, 4] / g[3, 3], np.exp(-1 / (2 * 1.3 ** 2)), rtol=1e-14)
    img = np.random.default_rng(1).random((16, 16))
    assert abs(O.convolve_periodic(img, g).sum() - img.sum()) < 1e-10


def test_renormalisation():
    img = np.random.default_rng(2).random((3, 6, 6)) + 0.5
    out = O.postprocess(img, renormalize=True)
    np.testing.assert_allclose(out.mean(axis=(1, 2)), 1.0, rtol=1e-14)
    np.testing.assert_allclose(out[1] * img[1].mean(), img[1], rtol=1e-14)
    assert np.all(O.postprocess(np.zeros((1, 4, 4)), renormalize=True) == 0)


@pytest.mark.parametrize("A", [1, 3, 5])
def test_moving_average_closed_form(A):
    n = 9
    imgs = np.arange(n, dtype=np.float64)[:, None, None] * np.ones((n, 2, 3))
    out = O.postprocess(imgs, accumulate=A)
    for t in range(n):
        lo = max(0, t - A + 1)
        assert np.allclose(out[t], (lo + t) / 2.0)
