"""Worker for tests/test_replicas_gloo.py, run under torchrun with the gloo backend on CPU: each rank
writes the max-over-ranks reduction of bench.py and the seed-shifted workload it would solve to a JSON
file of its own (rank_<r>.json in the directory given as the first argument), so that the ranks'
reports cannot interleave on a shared stdout."""
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
    rec = {"rank": rank, "world": world, "max": ms, "void": int(w.mask.sum()), "mu": mu}
    with open(os.path.join(sys.argv[1], f"rank_{rank}.json"), "w") as f:
        json.dump(rec, f)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
