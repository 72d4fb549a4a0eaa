"""The multi-GPU path of bench.py (frame-sharded replicas) on CPU: two gloo ranks.

Frames are independent, so N GPUs decode N disjoint shards and only scalars cross ranks: the
slowest rank's time (MAX) and the error counters (SUM).  Here each rank draws its shard's
channel LLRs from its own seed stream and decodes it with the FP64 oracle; the summed counters
must equal what one process gets from both shards, the seed streams must be disjoint, and the
whole-job throughput must count every rank's frames over the slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1202_1060_gb300 import inputs as I

CODE = "qc_n576_r12"
FRAMES = 12
EBN0 = 2.0


def _shard(O, c, gp, gc, rank, step=0, point=0):
    llr = O.awgn_llr(c.N, FRAMES, EBN0, I.design_rate(c), bench.channel_seed(point, step, rank))
    r = O.ndgsbp_decode(c, gp, gc, llr, 25)
    return llr, np.array([int(r.hard.any(axis=1).sum()), int(r.iters.sum()), FRAMES], dtype=np.int64)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        c = I.code_by_name(CODE)
        gp, gc = O.groups(c.M, c.M // c.Z, 0.5, 2304, unit=c.Z, cyclic=True)
        llr, counts = _shard(O, c, gp, gc, rank)
        t = torch.from_numpy(counts.copy())
        bench.sum_over_ranks(t, world)
        slowest = bench.max_over_ranks(1.0 + rank, "cpu", world)
        seeds = [None] * world
        dist.all_gather_object(seeds, [bench.channel_seed(p, s, rank) for p in range(9) for s in range(4)])
        first = [None] * world
        dist.all_gather_object(first, float(llr[0, 0]))
        if rank == 0:
            out.put(dict(counts=t.numpy().tolist(), slowest=slowest, seeds=seeds, first=first))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_sharded_decode_and_timing(oracle_mod):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # the summed counters equal one process decoding both shards
    c = I.code_by_name(CODE)
    gp, gc = oracle_mod.groups(c.M, c.M // c.Z, 0.5, 2304, unit=c.Z, cyclic=True)
    expect = sum(_shard(oracle_mod, c, gp, gc, r)[1] for r in range(world))
    assert res["counts"] == expect.tolist()
    # the slowest rank's time, and the whole-job throughput over it
    assert res["slowest"] == 2.0
    assert bench.whole_job_gbits(100, world, 1152, res["slowest"]) == pytest.approx(100 * 2 * 1152 / 2.0 / 1e9)
    # disjoint channel streams per rank (and per point and step)
    a, b = (set(s) for s in res["seeds"])
    assert len(a) == len(res["seeds"][0]) and not a & b
    assert res["first"][0] != res["first"][1]
