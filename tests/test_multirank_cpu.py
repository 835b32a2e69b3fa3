"""The multi-rank path on CPU ranks (gloo, world size 2): shards partition the
shots, a shard's records are those of the same global shot indices in one
process (counter-based Philox draws), and the summed tallies of a sharded job
equal the single-process tallies."""

import os
import socket

import numpy as np
import pytest

from paper_2605_29514_gb300.shards import allreduce_sum, rank_base, shard

torch = pytest.importorskip("torch")


def test_shards_partition():
    for total in [0, 1, 7, 16384, 100001]:
        for world in [1, 2, 3, 8]:
            got = [shard(total, world, r) for r in range(world)]
            assert sum(c for _, c in got) == total
            nxt = 0
            for lo, c in got:
                assert lo == nxt and c >= 0
                nxt = lo + c
    assert rank_base(1) - rank_base(0) >= 10 ** 9
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def tallies(w, first, count):
    from oracle.circuit import detectors, logical_z
    from oracle.shot import make_program, run_shot
    from workloads import theta_table
    prog = make_program(w)
    theta = theta_table(w, len(prog.pairs))
    det_counts = None
    flips = 0
    logp = 0.0
    for s in range(first, first + count):
        res = run_shot(w, s, theta, prog)
        d = np.array(detectors(prog, res.record), dtype=np.float64)
        det_counts = d if det_counts is None else det_counts + d
        flips += logical_z(prog, res.record)
        logp += res.logp
    return det_counts, np.array([flips, logp, count], dtype=np.float64)


def _worker(rank, world, port, w, total, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = shard(total, world, rank)
    det, misc = tallies(w, first, count)
    det, misc = allreduce_sum([det, misc], dist)
    if rank == 0:
        q.put((det.tolist(), misc.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_tallies_equal_single_process():
    import multiprocessing as mp
    from workloads import D3_EXACT
    w = D3_EXACT.with_(rounds=1, p=0.05, chi_cap=8)
    total, world = 6, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, w, total, q)) for r in range(world)]
    for p in procs:
        p.start()
    det, misc = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    det1, misc1 = tallies(w, 0, total)
    assert np.array_equal(np.array(det), det1)
    assert misc[0] == misc1[0] and misc[2] == total
    assert abs(misc[1] - misc1[1]) < 1e-9 * max(1.0, abs(misc1[1]))


def test_batch_offsets_disjoint_within_and_across_ranks():
    from paper_2605_29514_gb300.shards import RANK_STRIDE, batch_offset
    B = 152
    ranges = []
    for rank in range(4):
        for b in range(30):
            lo = batch_offset(rank, b, B)
            ranges.append((lo, lo + B))
    ranges.sort()
    for (lo0, hi0), (lo1, _) in zip(ranges, ranges[1:]):
        assert hi0 <= lo1
    with pytest.raises(ValueError):
        batch_offset(0, RANK_STRIDE // B, B)


def _offset_worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2605_29514_gb300.shards import batch_offset
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # the warm-up and timed batches of bench.py on this rank: W + K/6 batches of 152
    mine = torch.tensor([batch_offset(rank, b, 152) for b in range(8)], dtype=torch.int64)
    got = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(got, mine)
    if rank == 0:
        q.put([g.tolist() for g in got])
    dist.barrier()
    dist.destroy_process_group()


def test_bench_batch_offsets_on_cpu_ranks():
    """Each rank of a two-rank gloo job computes the global shot offsets of its
    batches as bench.py does; gathered on rank 0 the shot ranges are
    pairwise disjoint."""
    import multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_offset_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    offsets = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spans = sorted((lo, lo + 152) for per_rank in offsets for lo in per_rank)
    assert len(spans) == 16
    for (lo0, hi0), (lo1, _) in zip(spans, spans[1:]):
        assert hi0 <= lo1
