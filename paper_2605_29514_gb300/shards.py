"""Shot sharding over ranks (one process per GPU).

Shots are independent and every random number of shot s is drawn from the
Philox counter (s, event) under the run's seed, so a rank that simulates a
range of global shot indices produces exactly the records a single process
would produce for those indices.  The only exchange a sharded job needs is a
sum of per-rank tallies at the end (detection-event counts, logical flips,
log-likelihoods), done with one all-reduce."""

import numpy as np

# Global shot index of shot 0 of a rank in a weak-scaling run, in which every
# rank simulates its own batches: ranges of 10^9 shots never overlap.
RANK_STRIDE = 10 ** 9


def shard(total, world, rank):
    """(first, count) of the contiguous block of `total` shots that `rank`
    of `world` simulates in a fixed-size (strong-scaling) job."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard request")
    lo = total * rank // world
    hi = total * (rank + 1) // world
    return lo, hi - lo


def rank_base(rank):
    """First global shot index of `rank` in a weak-scaling run."""
    return rank * RANK_STRIDE


def batch_offset(rank, batch, shots_per_batch):
    """First global shot index of batch number `batch` (0, 1, ...) of `rank`
    in a weak-scaling run whose batches hold `shots_per_batch` shots: the
    batches of one rank are consecutive ranges starting at rank_base(rank),
    so ranks never share a shot as long as a rank runs fewer than
    RANK_STRIDE shots."""
    if rank < 0 or batch < 0 or shots_per_batch < 1:
        raise ValueError("bad batch request")
    if (batch + 1) * shots_per_batch > RANK_STRIDE:
        raise ValueError("a rank's shots would reach the next rank's range")
    return rank_base(rank) + batch * shots_per_batch


def allreduce_sum(arrays, dist=None, device="cpu"):
    """Element-wise sum of each numpy array over all ranks; returns the
    summed arrays.  Without an initialised process group this is the
    identity."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return [np.array(a) for a in arrays]
    import torch
    out = []
    for a in arrays:
        t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        out.append(t.cpu().numpy())
    return out
