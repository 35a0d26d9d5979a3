"""Run under torchrun with the gloo backend: checks bench.py's replica timing
aggregation (max of the per-rank times, sum of the per-rank work)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main():
    world, rank, local = bench.dist_env()
    assert world == 2
    dist = bench.dist_init(world, "gloo")
    bench.barrier(world)
    t = 10.0 + 5.0 * rank           # rank 1 is the slower replica
    work = 1000.0 * (rank + 1)
    tmax = bench.reduce_max(t, world)
    wsum = bench.reduce_sum(work, world)
    assert tmax == 15.0, tmax
    assert wsum == 3000.0, wsum
    # the aggregate the benchmark prints: all ranks' work over the slowest rank's time
    assert abs(wsum / tmax - 200.0) < 1e-12
    bench.barrier(world)
    dist.destroy_process_group()
    print(f"rank {rank} ok")


if __name__ == "__main__":
    main()
