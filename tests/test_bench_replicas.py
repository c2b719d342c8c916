"""The multi-GPU path of bench.py on CPU: world-size-2 gloo process groups run the
replica timing (max over ranks, whole-job throughput) and the reference arm's
rank rule (only rank 0 works and prints)."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    elapsed = [1.5, 2.5][rank]  # rank 1 is the slow replica
    td.barrier()
    t = b.max_over_ranks(elapsed, td, "cpu")
    v = b.job_value(world, 4, 1000, t)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "v": v}, f)
    td.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["t"] == 2.5                      # every rank sees the slowest time
        assert d["v"] == pytest.approx(2 * 4 * 1000 / 2.5)


def test_no_process_group_is_identity():
    b = _bench()
    assert b.max_over_ranks(3.25, None, "cpu") == 3.25
    assert b.job_value(1, 10, 4096, 2.0) == 20480


def test_reference_arm_only_rank0_prints():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "tiny_asp_stft_256_t64", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
