"""The multi-GPU path is replicas only (queries are independent; no
collective on the data path).  bench.py aggregates whole-job throughput as
all ranks' units over the slowest rank's time: checked here with two gloo
ranks on CPU, each reporting a different time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms_local = [100.0, 250.0][rank]
        value, ms = bench.job_throughput(40, ms_local, world, device="cpu")
        q.put((rank, value, ms))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_uses_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, ms in got:
        assert ms == 250.0                       # both ranks see the slowest time
        assert value == pytest.approx(2 * 40 / 0.250)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(10, 500.0, 1) == (20.0, 500.0)


def test_serving_trace_is_poisson_with_the_stated_mix():
    """The served workload's arrivals: exponential gaps at the given rate,
    80% of requests from the UCI-shaped clients, every client id valid."""
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_2506_18150_gb300 import synthetic as syn
    arr, cl = syn.serving_trace(50.0, 20_000, 32, 8, 0.8, seed=3)
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    gaps = np.diff(arr)
    assert abs(gaps.mean() - 1 / 50.0) < 0.05 / 50.0
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05          # exponential: CV = 1
    uci = cl < 32
    assert abs(uci.mean() - 0.8) < 0.02 and cl.max() < 40 and cl.min() >= 0
    assert len(np.unique(cl[uci])) == 32 and len(np.unique(cl[~uci])) == 8
    a2, c2 = syn.serving_trace(50.0, 20_000, 32, 8, 0.8, seed=3)
    assert np.array_equal(arr, a2) and np.array_equal(cl, c2)      # seeded


def test_spawned_replicas_report_the_whole_job(tmp_path):
    """bench.py --gpus N without torchrun starts N ranks itself
    (bench.spawn_replicas); here two gloo ranks of a stub step on CPU."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    out = tmp_path / "out.txt"
    with open(out, "w") as f:
        rc = bench.spawn_replicas(2, os.path.join(ROOT, "tests", "replica_stub.py"), ["--gpus", "2"],
                                  env=dict(os.environ, OMP_NUM_THREADS="1"), stdout=f)
    assert rc == 0
    lines = [ln for ln in open(out).read().splitlines() if ln.startswith("{")]
    assert len(lines) == 1                       # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["ms"] == 250.0 and d["value"] == pytest.approx(2 * 40 / 0.250)
    assert d["argv"] == ["--gpus", "2"]


def test_bench_rejects_a_mismatched_world():
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2"], cwd=ROOT,
                       env=dict(os.environ, WORLD_SIZE="4", RANK="0", LOCAL_RANK="0"), capture_output=True,
                       text=True, timeout=120)
    assert r.returncode != 0 and "does not match WORLD_SIZE" in r.stderr
