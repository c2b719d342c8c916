"""Host logic of bench.py that needs no GPU: the sizing of the CPU-baseline
sample (a first sample of 2-3 windows, then one scaled to the time budget,
capped by the step's frames and the oracle's memory)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _fake_sampler(per_window_s):
    calls = []

    def sample(w, n):
        nwin = (n - w["T"]) // w["S"] + 1
        calls.append(n)
        dt = per_window_s * nwin
        return n / dt, nwin, dt

    return sample, calls


def test_overlapping_windows_scale_to_the_budget():
    b = _bench()
    w = dict(b.WORKLOADS["stream_fresnel_256_t512_s64"])
    b.oracle_sample, calls = _fake_sampler(1.0)
    r = b.cpu_baseline(w, budget_s=12.0)
    assert calls[0] == 512 + 2 * 64                 # 3 windows first
    assert calls[1] == 512 + 11 * 64                # then 12 windows (~12 s)
    assert r["sample"].startswith("first 1216 frames of the workload (12 windows)")
    assert r["cores"] == 1 and r["kind"] == "oracle"


def test_long_first_sample_is_kept():
    b = _bench()
    w = dict(b.WORKLOADS["pca_512_t256"])
    b.oracle_sample, calls = _fake_sampler(5.0)    # 2 windows take 10 s >= 2/3 of 12 s
    b.cpu_baseline(w, budget_s=12.0)
    assert calls == [2 * 256]


def test_sample_is_capped_by_the_step_and_memory():
    b = _bench()
    w = dict(b.WORKLOADS["pca_fresnel_256_t32"])
    b.oracle_sample, calls = _fake_sampler(1e-3)   # very fast: the budget would ask for ~24k windows
    b.cpu_baseline(w, budget_s=12.0)
    cap_mem = (4 << 30) // (w["N"] * w["N"] * 16)
    assert calls[-1] == min(w["batch"] * w["batches"], cap_mem)
