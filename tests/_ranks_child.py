"""One rank of a gloo process group (started by torchrun from
tests/test_bench_ranks.py): runs bench.py's multi-rank helpers and has rank 0
print what every rank saw as one JSON line."""
import json
import os
import sys

import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    step_ms = 10.0 + 5.0 * rank            # each rank's own step time
    seen = bench.max_over_ranks(step_ms, "cpu")
    mine = {"rank": rank, "max": seen, "seeds": bench.batch_seeds(rank, 4)}
    every = [None] * world
    dist.all_gather_object(every, mine)
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        print(json.dumps({"world": world, "ranks": every}), flush=True)


if __name__ == "__main__":
    main()
