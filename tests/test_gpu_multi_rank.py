"""The frame-sharded replica path with the library itself (GPU): two ranks, one process each.

Frames are independent, so N GPUs decode N disjoint shards and only scalars cross ranks: the
slowest rank's time (MAX) and the error/iteration counters (SUM).  A run here gets one GPU, so
both ranks decode on it through the C ABI -- their kernels never wait on each other; the ranks
meet only in host-side gloo collectives on CPU tensors, as bench.py's reductions do.  The summed
counters, and every frame's decisions, must equal one process decoding both shards.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CODE = "qc_n2304_r12"
FRAMES = 4096
EBN0 = 1.5


def _shard(nd, torch, I, bench, code, c, groups, rank):
    """Rank `rank`'s shard: its channel LLRs (its own seed stream) decoded with the fused
    statistics; returns (counters [frames, frame errors, iterations], packed hard bits)."""
    dev = torch.device("cuda", 0)
    llr = torch.empty((FRAMES, c.N), dtype=torch.float32, device=dev)
    nd.awgn_llr(code, FRAMES, EBN0, I.design_rate(c), bench.channel_seed(4, 0, rank), llr)
    hard = torch.empty((FRAMES, (c.N + 31) // 32), dtype=torch.int32, device=dev)
    stats = torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)
    p = nd.params_default(max_iter=25)
    ws = torch.zeros(max(256, groups.workspace_size(p, FRAMES)), dtype=torch.uint8, device=dev)
    nd.decode(groups, p, llr, ws, hard, stats=stats)
    torch.cuda.synchronize()
    s = stats.cpu()
    counts = torch.tensor([int(s[nd.STAT_FRAMES]), int(s[nd.STAT_FRAME_ERRORS]), int(s[nd.STAT_ITERATIONS])],
                          dtype=torch.int64)
    return counts, hard.cpu().numpy()


def _env():
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    import bench
    from paper_1202_1060_gb300 import inputs as I
    from paper_1202_1060_gb300 import ndgsbp as nd
    c = I.code_by_name(CODE)
    code = nd.Code.from_inputs(c)
    groups = nd.Groups.build(code, c.M // c.Z, 0.5, 2304, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    return nd, torch, I, bench, code, c, groups


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nd, torch, I, bench, code, c, groups = _env()
        torch.cuda.set_device(0)
        counts, hard = _shard(nd, torch, I, bench, code, c, groups, rank)
        bench.sum_over_ranks(counts, world)
        slowest = bench.max_over_ranks(1.0 + rank, "cpu", world)
        shards = [None] * world
        dist.all_gather_object(shards, hard)
        if rank == 0:
            out.put(dict(counts=counts.tolist(), slowest=slowest, hard=shards))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_decode_their_shards_through_the_library():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    nd, torch, I, bench, code, c, groups = _env()
    alone = [_shard(nd, torch, I, bench, code, c, groups, r) for r in range(world)]
    assert res["counts"] == sum(a[0] for a in alone).tolist()
    assert res["counts"][0] == world * FRAMES
    for r in range(world):
        np.testing.assert_array_equal(res["hard"][r], alone[r][1])
    assert not np.array_equal(alone[0][1], alone[1][1])   # disjoint channel streams
    assert res["slowest"] == 2.0
