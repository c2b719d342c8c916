"""GPU parity of the autofocus network's kernels (include/hv_af.h) against the
FP64 oracle: forward output, gradient of every parameter tensor, the Adam
update, and a short training run that must fit a small set.

The oracle runs with the GPU's storage precision: inputs, convolution weights
and stored activations rounded to bfloat16 (the rounding being part of the
method as built); every sum is float64 there and float32 on the GPU. The two
differ by float32 accumulation error (~1e-6 relative) and by the rare
activation whose float32 and float64 values round to neighbouring bfloat16
numbers (2^-8 relative, a few per batch), hence the bars below."""
import numpy as np
import pytest

from oracle import af_oracle as A

pytestmark = pytest.mark.gpu


def _setup(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    flat = A.init_params(seed)
    flat = flat + 0.02 * rng.standard_normal(flat.size)
    p = A.unflatten(flat)
    for l in range(1, 5):
        p[f"w{l}"] = A.bf16(p[f"w{l}"])      # the GPU's convolution weights are bfloat16
    flat = A.flatten(p).astype(np.float32).astype(np.float64)
    x = A.bf16(rng.standard_normal((n, 1, 128, 128)))
    z = rng.uniform(0.1, 0.6, n)
    xd = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda()
    zd = torch.from_numpy(z.astype(np.float32)).cuda()
    return flat, x, z, xd, zd


def _net(n):
    from paper_2508_03911_gb300 import af
    return af.Autofocus(n)


@pytest.mark.parametrize("n", [6, 3])
def test_forward_matches_oracle(n):
    """Layers 2-4 run as tensor-core implicit GEMMs over tiles of 128 output
    pixels: n = 3 leaves the last-layer tile half full (192 pixels)."""
    import torch
    flat, x, z, xd, zd = _setup(n, 1)
    with _net(8) as net:
        net.set_params(flat)
        out = torch.zeros(n, device="cuda")
        net.forward(xd, out)
        net.synchronize()
        got = out.cpu().numpy()
    ref = A.predict_z(flat, x, bf16_acts=True)
    err = np.max(np.abs(got - ref))
    print(f"forward max |dz| {err:.3e} m")
    assert err <= 1e-3, (got, ref)


def test_gradients_match_oracle():
    import torch
    flat, x, z, xd, zd = _setup(6, 2)
    with _net(8) as net:
        net.set_params(flat)
        loss = torch.zeros(1, device="cuda")
        grad = torch.zeros(A.n_params(), device="cuda")
        net.loss_grad(xd, zd, loss, grad)
        torch.cuda.synchronize()
        g = grad.cpu().numpy().astype(np.float64)
        L = float(loss.item())
    Lr, gr = A.gradients(flat, x, z.astype(np.float32).astype(np.float64), bf16_acts=True)
    assert abs(L - Lr) <= 1e-3 * Lr, (L, Lr)
    o = 0
    for name, s in A.param_shapes():
        k = int(np.prod(s))
        e = np.linalg.norm(g[o:o + k] - gr[o:o + k]) / max(np.linalg.norm(gr[o:o + k]), 1e-30)
        print(f"{name}: rel L2 {e:.2e}")
        assert e <= 1e-2, (name, e)
        o += k


def test_adam_update_matches_oracle():
    import torch
    flat, x, z, xd, zd = _setup(4, 3)
    with _net(4) as net:
        net.set_params(flat)
        grad = torch.zeros(A.n_params(), device="cuda")
        loss = torch.zeros(1, device="cuda")
        net.loss_grad(xd, zd, loss, grad)
        net.train_step(xd, zd, lr=1e-3)
        torch.cuda.synchronize()
        g = grad.cpu().numpy().astype(np.float64)
        p1 = net.get_params().astype(np.float64)
    want, _, _ = A.adam_step(flat, g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3)
    assert np.max(np.abs(p1 - want)) <= 1e-3 * 1e-3 + 1e-6 * np.max(np.abs(flat))


def test_short_training_fits_a_small_set():
    import torch
    flat, x, z, xd, zd = _setup(32, 4)
    with _net(32) as net:
        net.set_params(flat)
        loss = torch.zeros(1, device="cuda")
        net.loss_grad(xd, zd, loss)
        torch.cuda.synchronize()  # the network runs on a stream of its own
        l0 = float(loss.item())
        for _ in range(300):
            net.train_step(xd, zd, loss, lr=2e-3)
        torch.cuda.synchronize()
        l1 = float(loss.item())
    print(f"loss {l0:.4f} -> {l1:.4f}")
    assert l1 < 0.2 * l0


def test_bf16_network_error_against_the_unrounded_fp64_oracle():
    """The error of the BF16 network itself: the GPU (bf16 input, bf16 convolution
    weights, bf16 stored activations, float32 sums) against the FP64 oracle with no
    rounding at all (float64 input, weights and activations). Stated per output:
    forward error in metres, and the relative L2 error of every parameter
    tensor's gradient."""
    import torch
    n = 8
    rng = np.random.default_rng(11)
    flat = A.init_params(11) + 0.02 * rng.standard_normal(A.n_params())
    flat = flat.astype(np.float32).astype(np.float64)  # the GPU's float32 master copy
    x = rng.standard_normal((n, 1, 128, 128))
    z = rng.uniform(0.1, 0.6, n).astype(np.float32).astype(np.float64)
    xd = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda()
    zd = torch.from_numpy(z.astype(np.float32)).cuda()
    with _net(n) as net:
        net.set_params(flat)
        out = torch.zeros(n, device="cuda")
        net.forward(xd, out)
        loss = torch.zeros(1, device="cuda")
        grad = torch.zeros(A.n_params(), device="cuda")
        net.loss_grad(xd, zd, loss, grad)
        net.synchronize()
        zp = out.cpu().numpy().astype(np.float64)
        g = grad.cpu().numpy().astype(np.float64)
        L = float(loss.item())
    z_ref = A.predict_z(flat, x, bf16_acts=False)
    L_ref, g_ref = A.gradients(flat, x, z, bf16_acts=False)
    dz = np.max(np.abs(zp - z_ref))
    print(f"BF16 network vs FP64: forward max |dz| {dz * 1e3:.3f} mm "
          f"(sweep step {0.5 / 63 * 1e3:.2f} mm), loss {L:.5f} vs {L_ref:.5f}")
    assert dz <= 0.5 / 63 / 4  # well inside a quarter of a sweep step
    assert abs(L - L_ref) <= 2e-2 * L_ref
    o = 0
    errs = {}
    for name, s in A.param_shapes():
        k = int(np.prod(s))
        errs[name] = np.linalg.norm(g[o:o + k] - g_ref[o:o + k]) / max(np.linalg.norm(g_ref[o:o + k]), 1e-30)
        print(f"  gradient {name}: rel L2 {errs[name]:.2e}")
        o += k
    # bar: the input and every stored activation carry bf16 rounding (unit roundoff
    # u = 2^-9); the first layer's weight gradient pairs the rounded input with an
    # error signal back-propagated through three bf16-stored layers and their ReLU
    # masks, so its error reaches tens of u; 0.1 (about 50 u) bounds every tensor
    for name, e in errs.items():
        assert e <= 0.1, (name, e)
