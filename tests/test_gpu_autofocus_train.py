"""What the trained network gains over the method without it: trained on the
GPU (8,192 holograms labelled by the plain sweep, 20 epochs), it estimates the
focus distance of unseen holograms close to the sweep's answer at a fraction of
the sweep's cost, while a constant guess misses by ~16 sweep steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trained_network_against_the_sweep():
    import torch

    from paper_2508_03911_gb300 import autofocus as AF
    from paper_2508_03911_gb300 import synth
    tr, _ = synth.autofocus_set(8192, N=256, seed=1004, workers=16)
    te, te_z = synth.autofocus_set(256, N=256, seed=1005, workers=16)
    p = AF.Pipeline(max_batch=256)
    try:
        _, tr_lab, _, tr_x = p.label_and_features(tr)
        _, te_lab, _, te_x = p.label_and_features(te)
        # the sweep itself finds the recorded distance
        assert np.mean(np.abs(te_lab - te_z) <= AF.STEP) >= 0.97
        p.net.set_params(AF.he_uniform(1))
        hist, _ = AF.train(p, tr_x, tr_lab, epochs=20, batch=256, lr=2e-3)
        pred = p.predict(te_x)
        err = np.abs(pred - te_lab) / AF.STEP
        const = np.abs(np.mean(tr_lab) - te_lab) / AF.STEP
        t_sweep, t_net = AF.time_sweep_and_net(p, te)
        print(f"within 1 step {np.mean(err <= 1):.3f}, MAE {err.mean():.2f} steps "
              f"(constant guess {const.mean():.1f}); sweep {t_sweep * 1e6:.1f} us, network "
              f"{t_net * 1e6:.1f} us per hologram")
        assert hist[-1] < 0.01
        assert err.mean() <= 2.0 and np.median(err) <= 1.5
        assert np.mean(err <= 1) >= 0.4
        assert err.mean() < 0.2 * const.mean()
        assert t_net < t_sweep / 4
    finally:
        p.close()
    torch.cuda.synchronize()
