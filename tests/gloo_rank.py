"""One rank of the CPU (gloo) check of bench.py's replica aggregation; run by
tests/test_dist_cpu.py under torch.distributed.run with two processes."""
import json
import os
import sys

import torch.distributed as dist

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def main():
    ws, rank, _ = bench.dist_env()
    dist.init_process_group("gloo")
    ms = 10.0 + 5.0 * rank  # each replica's own timed region
    t_max = bench.max_over_ranks(ms, ws, "cpu")
    value = bench.job_value(1.0e9, ws, t_max)
    dist.barrier()
    with open(os.path.join(sys.argv[1], f"rank{rank}.json"), "w") as f:  # one file per rank: no interleaving
        json.dump({"rank": rank, "ws": ws, "t_max": t_max, "value": value, "seed": bench.replica_seed(rank)}, f)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
