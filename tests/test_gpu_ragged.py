"""Ragged multi-code batches in one persistent launch (needs a GB300).

Four seeded QC codes (n=576 r1/2, 1152 r2/3, 2304 r3/4, 8192 r27/32), each grouped in cyclic
2-layer windows, are decoded by one launch of the tile kernel.  Every frame's result must equal
the one the tile kernel gives for that code alone (the same arithmetic, with the same lanes per
CN), the CUDA-graph replay must equal the plain launch, also after the inputs are refilled, and
sampled frames are checked against the FP64 oracle.
"""
import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I
from parity_rules import check_full

pytestmark = pytest.mark.gpu

MIX = [("qc_n576_r12", 2.5), ("qc_n1152_r23", 3.0), ("qc_n2304_r34", 3.5), ("qc_n8192_r2732", 4.0)]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp, torch


def _setup(nd, torch, frames, msg, seed=1):
    dev = torch.device("cuda")
    out = []
    for i, (name, ebn0) in enumerate(MIX):
        c = I.code_by_name(name)
        code = nd.Code.from_inputs(c)
        g = nd.Groups.build(code, c.M // c.Z, 0.5, 17 + i, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
        F = frames[i]
        llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=seed * 100 + i, dtype=np.float32)
        W = (c.N + 31) // 32
        out.append(dict(c=c, code=code, groups=g, host_llr=llr, llr=torch.from_numpy(llr).to(dev),
                        hard_bits=torch.zeros((F, W), dtype=torch.int32, device=dev),
                        iters=torch.zeros(F, dtype=torch.int32, device=dev),
                        syndrome_ok=torch.zeros(F, dtype=torch.uint8, device=dev),
                        posterior=torch.zeros((F, c.N), dtype=torch.float32, device=dev),
                        stats=torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)))
    return out


def _alone(nd, torch, b, params, lanes):
    c = b["c"]
    F = b["llr"].shape[0]
    p = nd.Params.from_buffer_copy(params)
    p.variant = nd.VARIANT_TILE
    p.lanes_per_cn = lanes
    dev = b["llr"].device
    hard = torch.zeros_like(b["hard_bits"])
    iters = torch.zeros_like(b["iters"])
    ok = torch.zeros_like(b["syndrome_ok"])
    post = torch.zeros_like(b["posterior"])
    ws = torch.zeros(b["groups"].workspace_size(p, F), dtype=torch.uint8, device=dev)
    nd.decode(b["groups"], p, b["llr"], ws, hard, iters, ok, post)
    return hard, iters, ok, post


@pytest.mark.parametrize("msg", ["f16", "f32"])
def test_ragged_equals_codes_alone(env, oracle_mod, msg):
    nd, torch = env
    params = nd.params_default(max_iter=30, msg_dtype=nd.F16 if msg == "f16" else nd.F32)
    batches = _setup(nd, torch, [400, 300, 200, 100], msg)
    rg = nd.Ragged(batches, params)
    plan, n_tiles = rg.info()
    assert plan["variant"] == nd.VARIANT_TILE and n_tiles > 0
    rg.launch()
    torch.cuda.synchronize()
    from paper_1202_1060_gb300.ndgsbp import _lib  # noqa: F401  (binding loaded)
    for b in batches:
        lanes = {8: 1, 16: 2, 32: 4}[min(x for x in (8, 16, 32) if x >= int(b["c"].row_degrees().max()))]
        hard, iters, ok, post = _alone(nd, torch, b, params, lanes)
        torch.cuda.synchronize()
        assert torch.equal(hard, b["hard_bits"]) and torch.equal(iters, b["iters"]), b["c"].name
        assert torch.equal(post, b["posterior"]) and torch.equal(ok, b["syndrome_ok"])
        st = b["stats"].cpu().numpy()
        assert st[nd.STAT_FRAMES] == b["llr"].shape[0]
        assert st[nd.STAT_ITERATIONS] == int(b["iters"].sum())
    # sampled frames against the oracle (FP32 messages only: FP16 is held to FER elsewhere)
    if msg == "f32":
        for b in batches:
            c, g = b["c"], b["groups"]
            q = g.query()
            idx = np.arange(0, b["llr"].shape[0], max(1, b["llr"].shape[0] // 12))
            ref = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], b["host_llr"][idx].astype(np.float64), 30)
            it = b["iters"].cpu().numpy()[idx]
            okf = b["syndrome_ok"].cpu().numpy()[idx]
            bits = nd.unpack_bits(b["hard_bits"][torch.from_numpy(idx).cuda()], c.N)
            check_full(f"ragged {c.name}", bits, it, okf, ref, b["host_llr"][idx].astype(np.float64),
                       lambda x: oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], x, 30))


def test_ragged_graph_replay(env):
    nd, torch = env
    params = nd.params_default(max_iter=20, msg_dtype=nd.F16)
    batches = _setup(nd, torch, [256, 192, 128, 64], "f16", seed=2)
    rg = nd.Ragged(batches, params)
    rg.launch()
    torch.cuda.synchronize()
    first = [(b["hard_bits"].clone(), b["iters"].clone(), b["posterior"].clone()) for b in batches]
    for b in batches:
        b["hard_bits"].zero_()
        b["iters"].zero_()
        b["posterior"].zero_()
    rg.graph_launch()
    rg.graph_launch()
    torch.cuda.synchronize()
    for b, (h, it, p) in zip(batches, first):
        assert torch.equal(b["hard_bits"], h) and torch.equal(b["iters"], it) and torch.equal(b["posterior"], p)
    # refill the same input buffers with new frames: the replay decodes the new contents
    for i, b in enumerate(batches):
        c = b["c"]
        new = I.channel_llr(c.N, b["llr"].shape[0], MIX[i][1], I.design_rate(c), seed=777 + i, dtype=np.float32)
        b["llr"].copy_(torch.from_numpy(new))
    rg.graph_launch()
    torch.cuda.synchronize()
    rg2 = nd.Ragged(batches, params)
    saved = [(b["hard_bits"].clone(), b["iters"].clone()) for b in batches]
    rg2.launch()
    torch.cuda.synchronize()
    for b, (h, it) in zip(batches, saved):
        assert torch.equal(b["hard_bits"], h) and torch.equal(b["iters"], it)


def test_ragged_empty_batch_and_residency_targets(env):
    """A batch with no frames in the mix, and every residency target (CTAs per SM): results are
    those of each code alone; a target under which a code's frame slot cannot fit is refused."""
    nd, torch = env
    batches = _setup(nd, torch, [60, 0, 40, 12], "f16", seed=3)
    alone = []
    for b in batches:
        if b["llr"].shape[0] == 0:
            alone.append(None)
            continue
        p = nd.params_default(max_iter=20, msg_dtype=nd.F16)
        lanes = {8: 1, 16: 2, 32: 4}[min(x for x in (8, 16, 32) if x >= int(b["c"].row_degrees().max()))]
        alone.append(_alone(nd, torch, b, p, lanes))
    torch.cuda.synchronize()
    ran = 0
    for k in (1, 2, 3, 4):
        params = nd.params_default(max_iter=20, msg_dtype=nd.F16, ctas_per_sm=k)
        try:
            rg = nd.Ragged(batches, params)
        except nd.NdgsbpError as e:
            assert e.status == nd.ERR_UNSUPPORTED and k >= 3, (k, str(e))
            continue
        plan, _ = rg.info()
        assert plan["ctas_per_sm"] <= k
        for b in batches:
            b["hard_bits"].zero_()
            b["iters"].zero_()
        rg.launch()
        torch.cuda.synchronize()
        for b, a in zip(batches, alone):
            if a is None:
                continue
            assert torch.equal(b["hard_bits"], a[0]) and torch.equal(b["iters"], a[1]), (k, b["c"].name)
        ran += 1
    assert ran >= 2


def _default_alone(nd, torch, b, params):
    """The batch decoded alone by ndgsbp_decode with the library's default plan."""
    F = b["llr"].shape[0]
    p = nd.Params.from_buffer_copy(params)
    p.variant = nd.VARIANT_AUTO
    dev = b["llr"].device
    hard = torch.zeros_like(b["hard_bits"])
    iters = torch.zeros_like(b["iters"])
    ok = torch.zeros_like(b["syndrome_ok"])
    post = torch.zeros_like(b["posterior"])
    ws = torch.zeros(max(256, b["groups"].workspace_size(p, F)), dtype=torch.uint8, device=dev)
    nd.decode(b["groups"], p, b["llr"], ws, hard, iters, ok, post)
    return hard, iters, ok, post


@pytest.mark.parametrize("msg", ["f16", "f32"])
def test_ragged_per_code_mode(env, msg):
    """Per-code mode: every code on its own default plan, forked onto concurrent streams.  Each
    batch's outputs and statistics equal those of the batch decoded alone; the graph replay
    equals the plain launch, also after the inputs are refilled; an empty batch is skipped."""
    nd, torch = env
    params = nd.params_default(max_iter=25, msg_dtype=nd.F16 if msg == "f16" else nd.F32,
                               variant=nd.VARIANT_RAGGED_PER_CODE)
    batches = _setup(nd, torch, [300, 0, 150, 80], msg, seed=4)
    rg = nd.Ragged(batches, params)
    plan, n = rg.info()
    assert plan["variant"] == nd.VARIANT_RAGGED_PER_CODE and n == len(batches)
    rg.launch()
    torch.cuda.synchronize()
    for b in batches:
        if b["llr"].shape[0] == 0:
            continue
        hard, iters, ok, post = _default_alone(nd, torch, b, params)
        torch.cuda.synchronize()
        assert torch.equal(hard, b["hard_bits"]) and torch.equal(iters, b["iters"]), b["c"].name
        assert torch.equal(post, b["posterior"]) and torch.equal(ok, b["syndrome_ok"])
        st = b["stats"].cpu().numpy()
        assert st[nd.STAT_FRAMES] == b["llr"].shape[0]
        assert st[nd.STAT_ITERATIONS] == int(b["iters"].sum())
    first = [(b["hard_bits"].clone(), b["iters"].clone()) for b in batches]
    for b in batches:
        b["hard_bits"].zero_()
        b["iters"].zero_()
    rg.graph_launch()
    rg.graph_launch()
    torch.cuda.synchronize()
    for b, (h, it) in zip(batches, first):
        assert torch.equal(b["hard_bits"], h) and torch.equal(b["iters"], it)
    for i, b in enumerate(batches):
        c, F = b["c"], b["llr"].shape[0]
        if F:
            b["llr"].copy_(torch.from_numpy(I.channel_llr(c.N, F, MIX[i][1], I.design_rate(c), seed=900 + i,
                                                          dtype=np.float32)))
    rg.graph_launch()
    torch.cuda.synchronize()
    for b in batches:
        if b["llr"].shape[0] == 0:
            continue
        hard, iters, _, _ = _default_alone(nd, torch, b, params)
        torch.cuda.synchronize()
        assert torch.equal(hard, b["hard_bits"]) and torch.equal(iters, b["iters"]), b["c"].name


def test_ragged_autotune_considers_per_code(env):
    """The ragged autotuner's winner is either a tile launch or the per-code mode, and the
    launch it describes decodes every batch as the batch decoded alone would."""
    nd, torch = env
    params = nd.params_default(max_iter=20, msg_dtype=nd.F16)
    batches = _setup(nd, torch, [400, 300, 200, 100], "f16", seed=5)
    best, ms = nd.ragged_autotune(batches, params, sample_frames=64)
    assert ms > 0 and best.variant in (nd.VARIANT_TILE, nd.VARIANT_RAGGED_PER_CODE)
    rg = nd.Ragged(batches, best)
    for b in batches:
        b["hard_bits"].zero_()
        b["iters"].zero_()
    rg.launch()
    torch.cuda.synchronize()
    for b in batches:
        if best.variant == nd.VARIANT_RAGGED_PER_CODE:
            hard, iters, _, _ = _default_alone(nd, torch, b, best)
        else:
            hard, iters, _, _ = _alone(nd, torch, b, best, b["lanes_per_cn"])
        torch.cuda.synchronize()
        assert torch.equal(hard, b["hard_bits"]) and torch.equal(iters, b["iters"]), b["c"].name
