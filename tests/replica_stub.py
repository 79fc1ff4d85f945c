"""A stand-in for bench.py's step, run by tests/test_replicas.py through
bench.spawn_replicas: each rank joins a gloo group from the torchrun
environment, reports a per-rank time, and rank 0 prints the whole-job line
that bench.py would print (replicas, max over ranks).  No GPU."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import torch.distributed as dist

    import bench
    world, rank, _ = bench.dist_env()
    dist.init_process_group("gloo")
    try:
        value, ms = bench.job_throughput(40, [100.0, 250.0, 50.0, 75.0][rank % 4], world, device="cpu")
        if rank == 0:
            print(json.dumps({"value": value, "n_gpus": world, "ms": ms, "argv": sys.argv[1:]}), flush=True)
    finally:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
