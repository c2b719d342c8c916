"""Learned autofocus: build a labelled set with the plain sweep, train the network
on the GPU, and measure it against the sweep.

    python -m paper_2508_03911_gb300.autofocus [--n-train 50000] [--n-test 1000]
        [--epochs 30] [--batch 256] [--lr 2e-3] [--workers 16] [--report PATH]
        [--weights PATH]

Holograms: 256 x 256 uint16 (12-bit) off-axis holograms of sparse point-
scatterer objects at z ~ U[0.10, 0.60] m (synth.autofocus_hologram), training
set seed 1004, test set seed 1005. Labels: the plain sweep (hv_focus_sweep, 64
distances 0.10 .. 0.60 m, Tamura coefficient of the propagated amplitude), its
best distance. Network input: hv_af_features (128 x 128 binned log-spectrum).
Every GPU step runs in libhv.so; this module only orders the calls.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

Z0, Z1, NZ = 0.10, 0.60, 64
STEP = (Z1 - Z0) / (NZ - 1)
PITCH, LAM = 20e-6, 852e-9


def z_grid() -> np.ndarray:
    return Z0 + np.arange(NZ) * STEP


def he_uniform(seed: int) -> np.ndarray:
    """Initial parameters in the flat order of hv_af.h: weights U(-b, b) with
    b = sqrt(6 / fan_in), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shapes = [((16, 1, 3, 3), True), ((16,), False), ((32, 16, 3, 3), True), ((32,), False),
              ((64, 32, 3, 3), True), ((64,), False), ((64, 64, 3, 3), True), ((64,), False),
              ((32, 64), True), ((32,), False), ((1, 32), True), ((1,), False)]
    out = []
    for s, is_w in shapes:
        n = int(np.prod(s))
        if is_w:
            b = math.sqrt(6.0 / int(np.prod(s[1:])))
            out.append(rng.uniform(-b, b, n))
        else:
            out.append(np.zeros(n))
    return np.concatenate(out).astype(np.float32)


class Pipeline:
    """The GPU side: one handle for the sweep and the features, one network."""

    def __init__(self, max_batch=256, chunk=512, device=0):
        import torch

        from . import af, hv
        self.torch, self.hv = torch, hv
        self.dev = torch.device("cuda", device)
        self.chunk = chunk
        self.r = hv.Renderer(256, 256, 16, chunk, device=device)
        self.r.set_params(256, 256, spatial="asp", z=0.3, T=16, stride=16, band=(1, 7))
        self.net = af.Autofocus(max_batch, device=device)
        self.zs = z_grid()

    def label_and_features(self, frames: np.ndarray):
        """Sweep labels (index, distance), the full sweep, and network inputs of
        uint16 holograms, chunk by chunk."""
        torch, hv = self.torch, self.hv
        n = frames.shape[0]
        feats = torch.empty((n, 1, 128, 128), dtype=torch.bfloat16, device=self.dev)
        metric = torch.empty((n, NZ), dtype=torch.float32, device=self.dev)
        for a in range(0, n, self.chunk):
            b = min(n, a + self.chunk)
            fr = torch.from_numpy(frames[a:b].view(np.int16)).to(self.dev)
            hv.hv_focus_sweep(self.r.h, fr, self.zs, metric[a:b])
            hv.hv_af_features(self.r.h, fr, feats[a:b])
        self.r.synchronize()
        m = metric.cpu().numpy()
        j = np.argmax(m, axis=1)
        return j, self.zs[j], m, feats

    def predict(self, feats):
        torch = self.torch
        n, batch = feats.shape[0], self.net.max_batch
        out = torch.empty(n, dtype=torch.float32, device=self.dev)
        for a in range(0, n, batch):
            b = min(n, a + batch)
            self.net.forward(feats[a:b], out[a:b])
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def close(self):
        self.net.close()
        self.r.close()


def train(p: Pipeline, feats, z_label, epochs, batch, lr, seed=7, log=None):
    """Adam with a cosine step size from lr to lr/100; batches are contiguous slices
    of the (already shuffled) set, visited in a fresh random order every epoch."""
    torch = p.torch
    n = feats.shape[0]
    zt = torch.from_numpy(z_label.astype(np.float32)).to(p.dev)
    nb = n // batch
    total = epochs * nb
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, device=p.dev)
    hist = []
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        acc = 0.0
        for bi in rng.permutation(nb):
            s = slice(bi * batch, (bi + 1) * batch)
            eta = lr * (0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * step / total)))
            p.net.train_step(feats[s], zt[s], loss, lr=eta)
            step += 1
            if bi == nb - 1 or step % 50 == 0:
                torch.cuda.synchronize()
                acc = float(loss.item())
        hist.append(acc)
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {acc:.5f} ({time.perf_counter() - t0:.1f} s)")
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def time_sweep_and_net(p: Pipeline, frames: np.ndarray, reps=3):
    """Time per hologram (host clock around synchronised batches of up to `chunk`
    holograms) of the plain sweep and of features + network."""
    torch, hv = p.torch, p.hv
    n = min(frames.shape[0], p.chunk)
    fr = torch.from_numpy(frames[:n].view(np.int16)).to(p.dev)
    metric = torch.empty((n, NZ), dtype=torch.float32, device=p.dev)
    feats = torch.empty((n, 1, 128, 128), dtype=torch.bfloat16, device=p.dev)
    z = torch.empty(n, dtype=torch.float32, device=p.dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps / n

    def sweep():
        hv.hv_focus_sweep(p.r.h, fr, p.zs, metric)
        p.r.synchronize()

    def net():
        hv.hv_af_features(p.r.h, fr, feats)
        p.r.synchronize()
        for a in range(0, n, p.net.max_batch):
            b = min(n, a + p.net.max_batch)
            p.net.forward(feats[a:b], z[a:b])
        torch.cuda.synchronize()

    return timed(sweep), timed(net)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=50000)
    ap.add_argument("--n-test", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--report", default=None)
    ap.add_argument("--weights", default=None)
    args = ap.parse_args(argv)

    from . import synth
    t0 = time.perf_counter()
    # holograms on the host first: the process pool starts before any CUDA call
    tr_frames, tr_z = synth.autofocus_set(args.n_train, N=256, seed=1004, workers=args.workers)
    te_frames, te_z = synth.autofocus_set(args.n_test, N=256, seed=1005, workers=args.workers)
    t_gen = time.perf_counter() - t0
    print(f"generated {args.n_train} + {args.n_test} holograms in {t_gen:.1f} s", flush=True)

    p = Pipeline(max_batch=args.batch)
    try:
        t1 = time.perf_counter()
        tr_j, tr_lab, _, tr_x = p.label_and_features(tr_frames)
        te_j, te_lab, _, te_x = p.label_and_features(te_frames)
        t_lab = time.perf_counter() - t1
        del tr_frames
        sweep_vs_true = np.abs(te_lab - te_z) / STEP
        print(f"labelled in {t_lab:.1f} s; sweep vs recorded z on the test set: "
              f"{np.mean(sweep_vs_true <= 1):.3f} within 1 step", flush=True)
        p.net.set_params(he_uniform(1))
        hist, t_train = train(p, tr_x, tr_lab, args.epochs, args.batch, args.lr, log=print)
        pred = p.predict(te_x)
        err_steps = np.abs(pred - te_lab) / STEP
        base = np.abs(np.mean(tr_lab) - te_lab) / STEP  # a constant guess, the training mean
        t_sweep, t_net = time_sweep_and_net(p, te_frames)
        rep = {
            "n_train": args.n_train, "n_test": args.n_test, "epochs": args.epochs, "batch": args.batch,
            "lr": args.lr, "train_seconds": round(t_train, 2), "label_seconds": round(t_lab, 2),
            "generate_seconds": round(t_gen, 1),
            "final_train_loss": hist[-1] if hist else None,
            "test_within_1_step_of_sweep": float(np.mean(err_steps <= 1.0)),
            "test_mae_steps_vs_sweep": float(np.mean(err_steps)),
            "test_median_steps_vs_sweep": float(np.median(err_steps)),
            "test_p90_steps_vs_sweep": float(np.percentile(err_steps, 90)),
            "test_mae_steps_vs_recorded_z": float(np.mean(np.abs(pred - te_z) / STEP)),
            "sweep_within_1_step_of_recorded_z": float(np.mean(sweep_vs_true <= 1.0)),
            "constant_guess_mae_steps": float(np.mean(base)),
            "sweep_us_per_hologram": round(t_sweep * 1e6, 2),
            "net_us_per_hologram": round(t_net * 1e6, 2),
            "speedup": round(t_sweep / t_net, 1),
        }
        print(json.dumps(rep), flush=True)
        if args.report:
            with open(args.report, "w") as f:
                json.dump(rep, f, indent=1)
        if args.weights:
            p.net.get_params().tofile(args.weights)
    finally:
        p.close()


if __name__ == "__main__":
    main()
