"""Run under torchrun with the gloo backend (two CPU ranks): the sharded weight
normalisation and systematic comb of paper_2504_18056_b300.shard against the
single-rank oracle on the same weights -- ancestors bit for bit, weights to
FP64 rounding -- for even and uneven splits and degenerate weight sets."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch.distributed as dist  # noqa: E402

import oracle  # noqa: E402
from paper_2504_18056_b300 import shard  # noqa: E402


def cases():
    rng = np.random.default_rng(31)
    P = 100_003
    yield "spread", rng.normal(0, 30, P), 0.37, 0.5
    yield "uneven split", rng.normal(0, 3, P), 0.999999, 0.2
    one = np.full(P, -1e4)
    one[P - 5] = 0.0
    yield "one survivor on the last rank", one, 0.0, 0.5
    dead0 = rng.normal(0, 1, P)
    dead0[: P // 2] = -1e6
    yield "a rank without weight", dead0, 0.61, 0.5
    yield "tiny set", rng.normal(0, 1, 3), 0.5, 0.34


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    assert world == 2
    for name, logw, u, frac in cases():
        P = logw.size
        cut = int(round(P * frac))
        lo, hi = (0, cut) if rank == 0 else (cut, P)
        w, M, S = shard.normalise(logw[lo:hi])
        teeth, anc = shard.comb(w, u, P)
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, w, teeth, anc))
        if rank == 0:
            w_all = np.concatenate([p[2] for p in parts])
            ref = oracle.lse(logw, np.zeros(P))
            np.testing.assert_allclose(w_all, ref["w"], rtol=1e-13, atol=1e-300)
            assert abs(M - ref["M"]) == 0.0, name
            got = np.full(P, -1, np.int64)
            for p in parts:
                assert np.all(got[p[3]] == -1), "a tooth owned twice"
                got[p[3]] = p[4]
            assert np.all(got >= 0), (name, "a tooth nobody owns")
            np.testing.assert_array_equal(got, oracle.resample(w_all, u), err_msg=name)
    dist.barrier()
    dist.destroy_process_group()
    print(f"rank {rank} ok")


if __name__ == "__main__":
    main()
