"""Worker for tests/test_replicas_gloo.py, run under torchrun with the gloo backend on CPU: each rank
reports the max-over-ranks reduction of bench.py and the seed-shifted workload it would solve."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    args = bench.parse(["--n", "24", "--gpus", str(world)])
    w, mu = bench.workload(args, rank)
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist)
    print(json.dumps({"rank": rank, "world": world, "max": ms, "void": int(w.mask.sum()), "mu": mu}), flush=True)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
