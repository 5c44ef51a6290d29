"""Run under torch.distributed.run with the gloo backend (CPU): exercises the
multi-rank host logic of bench.py -- rank discovery, the barrier and the
max-over-ranks time -- and prints what rank 0 would report."""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    world, rank, local = bench.dist_env()
    dist.init_process_group("gloo")
    # rank r "takes" 10 + 5 r ms for its shard; the job takes the slowest
    dist.barrier()
    t0 = time.perf_counter()
    ms = 10.0 + 5.0 * rank
    slowest = bench.max_over_ranks(ms, world, torch.device("cpu"))
    dist.barrier()
    seen = [None] * world
    dist.all_gather_object(seen, {"rank": rank, "local": local, "slowest": slowest})
    if rank == 0:
        print(json.dumps({"world": world, "seen": seen,
                          "rate": bench.whole_job_rate(1e9, world, slowest),
                          "s": time.perf_counter() - t0}))
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
