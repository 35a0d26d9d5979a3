"""Exchange protocol of one particle set sharded over several ranks (host side).

The benchmark runs one whole session per GPU (replicas); this module is the
protocol for the other layout, a single particle set split into contiguous
blocks, one per rank. The filter's only cross-particle steps are the weight
normalisation (Eq. 11) and the systematic resampling; everything else in a
frame is per particle. They need three collectives per frame:

  1. allreduce MAX of the ranks' largest log-weights: M;
  2. allreduce SUM of S_r = sum_i exp(logw_i - M) over each rank's block: S,
     then w_i = exp(logw_i - M - log S) on every rank (FP64);
  3. allgather of the ranks' totals of the quantised weights
     q_i = rint(w_i 2^52) (exact integers, zero below 2^-53): each rank's offset
     O_r (the totals of the ranks before it) and the grand total S_q.

Tooth m = 0..P-1 of the systematic comb sits at tau_m = ((u + m) / P) S_q
(IEEE double operations, each rounded once); its ancestor is
a_m = min{i : C_i > tau_m}, clamped to P - 1, C the inclusive prefix sum of q
over the whole set. Rank r owns the teeth with O_r <= tau_m < O_r + S_r (the
last rank also those at or past S_q) and finds their ancestors from its own
prefix sums shifted by O_r. Every sum here is an integer below 2^53, exact in a
double, so the union over the ranks is the single-rank resampling bit for bit,
whatever the split. Moving the ancestors' states to the ranks that own the
output slots is a fourth exchange (all-to-all), left to the caller.
"""
from __future__ import annotations

import numpy as np

TWO52 = float(2 ** 52)


def _dist():
    import torch.distributed as dist
    return dist


def normalise(logw, group=None):
    """Steps 1-2 on this rank's block: (w, M, S) with w the normalised weights of
    the block (FP64), M the global max log-weight and S the global sum of
    exp(logw - M)."""
    import torch
    dist = _dist()
    logw = np.asarray(logw, np.float64)
    m = torch.tensor([logw.max() if logw.size else -np.inf], dtype=torch.float64)
    dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
    M = float(m.item())
    s = torch.tensor([float(np.exp(logw - M).sum())], dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    S = float(s.item())
    return np.exp(logw - M - np.log(S)), M, S


def quantise(w):
    """q_i = rint(w_i 2^52) as exact unsigned integers (w in [0, 1])."""
    return np.rint(np.asarray(w, np.float64) * TWO52).astype(np.uint64)


def comb(w, u, P, group=None):
    """Step 3 and the comb on this rank's block of normalised weights w (the
    block's first particle has global index i0 = the sizes of the ranks before
    it): returns (teeth, ancestors), the comb positions m this rank owns and
    their global ancestor indices."""
    import torch
    dist = _dist()
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    q = quantise(w)
    csum = np.cumsum(q, dtype=np.uint64)
    total = int(csum[-1]) if csum.size else 0
    mine = torch.tensor([total, q.size], dtype=torch.int64)
    every = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(every, mine, group=group)
    totals = [int(t[0]) for t in every]
    sizes = [int(t[1]) for t in every]
    assert sum(sizes) == P, "the blocks must cover the particle set"
    O = sum(totals[:rank])
    Sq = sum(totals)
    i0 = sum(sizes[:rank])
    m = np.arange(P, dtype=np.float64)
    tau = (u + m) / P * float(Sq)            # each operation rounded once, as in the single-rank comb
    lo, hi = float(O), float(O + total)
    own = (tau >= lo) & (tau < hi)
    if rank == world - 1:
        own |= tau >= float(Sq)
    teeth = np.nonzero(own)[0]
    # a_m = min{i : O + C_i > tau_m}: C_i and O are integers below 2^53, exact in doubles
    c_global = csum.astype(np.float64) + lo
    anc = np.searchsorted(c_global, tau[teeth], side="right")
    anc = np.minimum(anc, max(q.size - 1, 0)) + i0
    return teeth.astype(np.int64), np.minimum(anc, P - 1).astype(np.int64)
