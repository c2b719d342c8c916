"""FP64 oracle of the learned autofocus: the plain z-sweep with the Tamura focus
metric, the log-spectrum feature, and the small CNN (forward, loss, backward,
Adam). Test infrastructure only: the tests, the smoke check and the bench's CPU
baseline use it; the product path never does.

The paper has no autofocus: its pipeline propagates to a distance the user sets
(Sec. III-B.1). This module states the method the CNN is trained to replace, in
plain definitions:

* Sweep: z_j = 0.10 + j * 0.50 / 63 m, j = 0..63. For each z_j, the hologram
  with its mean removed is propagated by angular spectrum (the same ASP as
  hv_oracle.asp) and the Tamura coefficient sqrt(sigma / mu) of the amplitude
  |U| is taken over the whole image. The focus label is the z_j of the largest
  coefficient. READING: the mean is removed first (the DC term |R|^2 of an
  off-axis hologram otherwise dominates |U| and the metric loses its peak).
* Feature: the magnitude of the centred 2-D spectrum of the mean-removed
  hologram, averaged over 2 x 2 bins (N x N -> N/2 x N/2), log(1 + .),
  standardised to zero mean and unit (population) deviation per image.
* CNN: four 3 x 3 convolutions with stride 2 and zero padding 1 (channels
  1 -> 16 -> 32 -> 64 -> 64), each followed by ReLU; a global average pool; a
  dense layer 64 -> 32 with ReLU; a dense layer 32 -> 1. The output y predicts
  the normalised distance t = (z - 0.35) / 0.25; the loss is mean((y - t)^2)
  over the batch.
* Adam with bias correction (beta1 0.9, beta2 0.999, eps 1e-8 by default).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import hv_oracle as O

Z0, Z1, NZ = 0.10, 0.60, 64
Z_MID, Z_HALF = 0.35, 0.25
CHANNELS = (1, 16, 32, 64, 64)
HIDDEN = 32

# ------------------------------------------------------------------ sweep


def z_grid() -> np.ndarray:
    """The 64 distances of the plain sweep."""
    return Z0 + np.arange(NZ) * ((Z1 - Z0) / (NZ - 1))


def focus_sweep(frame: np.ndarray, lam: float, dx: float, dy: float, zs=None) -> np.ndarray:
    """Tamura coefficient of |ASP(h - mean h, z)| for every z of the sweep."""
    zs = z_grid() if zs is None else np.asarray(zs, dtype=np.float64)
    u0 = O.convert(frame)
    u0 = u0 - u0.mean()
    return np.array([O.tamura(np.abs(O.asp(u0, lam, dx, dy, float(z)))) for z in zs])


def focus_label(frame, lam, dx, dy) -> tuple[int, float]:
    """Index and distance of the sweep's maximum."""
    t = focus_sweep(frame, lam, dx, dy)
    j = int(np.argmax(t))
    return j, float(z_grid()[j])


# ---------------------------------------------------------------- feature


def features(frame: np.ndarray) -> np.ndarray:
    """Standardised log-magnitude spectrum, 2 x 2 binned: (N, N) -> (N/2, N/2)."""
    u = O.convert(frame)
    u = u - u.mean()
    F = O.fft2(u)
    M = np.abs(np.fft.fftshift(F))
    H, W = M.shape
    B = M.reshape(H // 2, 2, W // 2, 2).mean(axis=(1, 3))
    x = np.log1p(B)
    return (x - x.mean()) / x.std()


# -------------------------------------------------------------------- CNN


def param_shapes() -> list[tuple[str, tuple]]:
    """Parameter tensors in their flat order (the C ABI's order too)."""
    shapes = []
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        shapes.append((f"w{l + 1}", (co, ci, 3, 3)))
        shapes.append((f"b{l + 1}", (co,)))
    shapes += [("f1w", (HIDDEN, CHANNELS[4])), ("f1b", (HIDDEN,)), ("f2w", (1, HIDDEN)), ("f2b", (1,))]
    return shapes


def n_params() -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unflatten(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, s in param_shapes():
        n = int(np.prod(s))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, s in param_shapes():
        if name.startswith("w") or name.endswith("w"):
            fan_in = int(np.prod(s[1:]))
            b = math.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-b, b, size=s).ravel())
        else:
            parts.append(np.zeros(int(np.prod(s))))
    return np.concatenate(parts)


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_s2(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n, o, i, j] = b[o] + sum_{c, di, dj} w[o, c, di, dj] x[n, c, 2i + di - 1, 2j + dj - 1],
    zero outside the input (stride 2, padding 1)."""
    n, c, H, W = x.shape
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    xp = np.zeros((n, c, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = np.broadcast_to(b[None, :, None, None], (n, w.shape[0], Ho, Wo)).copy()
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + 2 * Ho:2, dj:dj + 2 * Wo:2]  # x[2i + di - 1, 2j + dj - 1]
            y += np.einsum("ncij,oc->noij", patch, w[:, :, di, dj])
    return y


def conv_s2_backward(x, w, dy):
    """Gradients of conv_s2 with respect to x, w and b for the upstream dy."""
    n, c, H, W = x.shape
    Ho, Wo = dy.shape[2], dy.shape[3]
    xp = np.zeros((n, c, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + 2 * Ho:2, dj:dj + 2 * Wo:2]
            dw[:, :, di, dj] = np.einsum("noij,ncij->oc", dy, patch)
            dxp[:, :, di:di + 2 * Ho:2, dj:dj + 2 * Wo:2] += np.einsum("noij,oc->ncij", dy, w[:, :, di, dj])
    return dxp[:, :, 1:H + 1, 1:W + 1], dw, dy.sum(axis=(0, 2, 3))


def forward(flat: np.ndarray, x: np.ndarray, bf16_acts: bool = False) -> tuple[np.ndarray, dict]:
    """Network output y (normalised distance) for inputs x (n, 1, h, w), and the
    saved activations. bf16_acts rounds the input and every stored activation to
    bfloat16, as the GPU kernels store them."""
    p = unflatten(flat)
    a = bf16(x) if bf16_acts else np.asarray(x, dtype=np.float64)
    acts = {"a0": a}
    for l in range(4):
        z = conv_s2(a, p[f"w{l + 1}"], p[f"b{l + 1}"])
        a = np.maximum(z, 0.0)
        if bf16_acts:
            a = bf16(a)
        acts[f"a{l + 1}"] = a
    g = a.mean(axis=(2, 3))
    h = np.maximum(g @ p["f1w"].T + p["f1b"], 0.0)
    y = (h @ p["f2w"].T + p["f2b"])[:, 0]
    acts.update(g=g, h=h)
    return y, acts


def target(z: np.ndarray) -> np.ndarray:
    return (np.asarray(z, dtype=np.float64) - Z_MID) / Z_HALF


def predict_z(flat, x, bf16_acts=False) -> np.ndarray:
    return Z_MID + Z_HALF * forward(flat, x, bf16_acts)[0]


def loss(flat, x, z, bf16_acts=False) -> float:
    y, _ = forward(flat, x, bf16_acts)
    return float(np.mean((y - target(z)) ** 2))


def gradients(flat, x, z, bf16_acts=False) -> tuple[float, np.ndarray]:
    """Loss and its gradient with respect to the flat parameters (back-propagation)."""
    p = unflatten(flat)
    y, acts = forward(flat, x, bf16_acts)
    n = y.shape[0]
    t = target(z)
    L = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / n                      # dL/dy
    grads = {}
    h, g = acts["h"], acts["g"]
    grads["f2w"] = dy[None, :] @ h              # (1, 32)
    grads["f2b"] = np.array([dy.sum()])
    dh = dy[:, None] * p["f2w"]                 # (n, 32)
    dh = dh * (h > 0)
    grads["f1w"] = dh.T @ g
    grads["f1b"] = dh.sum(axis=0)
    dg = dh @ p["f1w"]                          # (n, 64)
    a4 = acts["a4"]
    da = np.broadcast_to(dg[:, :, None, None] / (a4.shape[2] * a4.shape[3]), a4.shape).copy()
    for l in range(4, 0, -1):
        dz = da * (acts[f"a{l}"] > 0)
        dx, dw, db = conv_s2_backward(acts[f"a{l - 1}"], p[f"w{l}"], dz)
        grads[f"w{l}"], grads[f"b{l}"] = dw, db
        da = dx
    return L, flatten(grads)


def adam_step(flat, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
