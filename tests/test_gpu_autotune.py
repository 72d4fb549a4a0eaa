"""Autotuner (needs a GB300): the tuned launch shape is one the plan accepts, it is no slower
than the library's default on the sample it was tuned on, a second call comes from the cache
(memory and file), and decoding with the tuned shape agrees with the default shape.
"""
import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp, torch


def _decode(nd, torch, g, c, p, d_llr):
    F = d_llr.shape[0]
    dev = d_llr.device
    hard = torch.zeros((F, (c.N + 31) // 32), dtype=torch.int32, device=dev)
    iters = torch.zeros(F, dtype=torch.int32, device=dev)
    ok = torch.zeros(F, dtype=torch.uint8, device=dev)
    ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
    nd.decode(g, p, d_llr, ws, hard, iters, ok)
    torch.cuda.synchronize()
    return hard.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy()


@pytest.mark.parametrize("name,ebn0", [("qc_n2304_r12", 1.5), ("qc_n8192_r2732", 3.5)])
def test_autotune_picks_valid_fast_shape(env, tmp_path, name, ebn0):
    nd, torch = env
    c = I.code_by_name(name)
    code = nd.Code.from_inputs(c)
    g = nd.Groups.build(code, c.M // c.Z, 0.5, 2304, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    llr = I.channel_llr(c.N, 4096, ebn0, I.design_rate(c), seed=31, dtype=np.float32)
    d_llr = torch.from_numpy(llr).cuda()
    p0 = nd.params_default(max_iter=25)
    cache = str(tmp_path / "tune.txt")
    best, info = nd.autotune(g, p0, d_llr, cache_path=cache)
    print(f"\n{name}: {info['candidates']} shapes, default {info['default_ms']:.3f} ms, best "
          f"{info['best_ms']:.3f} ms (variant {best.variant}, threads {best.block_threads}, "
          f"fpc {best.frames_per_cta}, lanes {best.lanes_per_cn}, ctas/SM {best.ctas_per_sm})")
    assert info["candidates"] >= 2 and not info["from_cache"]
    assert info["best_ms"] <= info["default_ms"]
    g.plan(best, 4096)   # the plan accepts it
    # cached: in memory, and from the file in a fresh key lookup
    best2, info2 = nd.autotune(g, p0, d_llr, cache_path=cache)
    assert info2["from_cache"] and bytes(best2) == bytes(best)
    assert open(cache).read().count("\n") == 1
    # decoding with the tuned shape agrees with the default shape
    h0, i0, o0 = _decode(nd, torch, g, c, p0, d_llr)
    h1, i1, o1 = _decode(nd, torch, g, c, best, d_llr)
    both = (o0 == 1) & (o1 == 1)
    np.testing.assert_array_equal(h0[both], h1[both])
    assert abs(int(o0.sum()) - int(o1.sum())) <= max(2, len(o0) // 500)


def test_ragged_autotune(env):
    nd, torch = env
    mix = [("qc_n576_r12", 2.5, 4000), ("qc_n1152_r23", 3.0, 3000), ("qc_n2304_r34", 3.5, 2000),
           ("qc_n8192_r2732", 4.0, 1000)]
    dev = torch.device("cuda")
    batches = []
    for i, (name, eb, F) in enumerate(mix):
        c = I.code_by_name(name)
        code = nd.Code.from_inputs(c)
        g = nd.Groups.build(code, c.M // c.Z, 0.5, 17 + i, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
        llr = I.channel_llr(c.N, F, eb, I.design_rate(c), seed=900 + i, dtype=np.float32)
        W = (c.N + 31) // 32
        batches.append(dict(c=c, code=code, groups=g, llr=torch.from_numpy(llr).to(dev),
                            hard_bits=torch.zeros((F, W), dtype=torch.int32, device=dev),
                            iters=torch.zeros(F, dtype=torch.int32, device=dev),
                            syndrome_ok=torch.zeros(F, dtype=torch.uint8, device=dev)))
    p0 = nd.params_default(max_iter=25, msg_dtype=nd.F16)
    p, ms = nd.ragged_autotune(batches, p0, sample_frames=1024)
    shapes = [(b["frames_per_cta"], b["lanes_per_cn"]) for b in batches]
    print(f"\nragged tuned: threads {p.block_threads}, per-code (fpc, lanes) {shapes}, {ms:.3f} ms")
    assert ms > 0
    if p.variant == nd.VARIANT_RAGGED_PER_CODE:
        # every code on its own default plan: the batches keep the library's shape choice
        assert all(f == 0 and l == 0 for f, l in shapes)
    else:
        assert p.variant == nd.VARIANT_TILE and p.block_threads in (128, 256, 384, 512) and 1 <= p.ctas_per_sm <= 4
        assert all(1 <= f <= 16 and l in (1, 2, 4) for f, l in shapes)
    # the tuned launch decodes each code as that code alone with the same shape (per-code mode:
    # with the default plan)
    rg = nd.Ragged(batches, p)
    rg.launch()
    torch.cuda.synchronize()
    for b in batches:
        q = nd.Params.from_buffer_copy(p)
        if p.variant == nd.VARIANT_RAGGED_PER_CODE:
            q.variant = nd.VARIANT_AUTO
        else:
            q.frames_per_cta, q.lanes_per_cn = b["frames_per_cta"], b["lanes_per_cn"]
        h, i, o = _decode(nd, torch, b["groups"], b["c"], q, b["llr"])
        np.testing.assert_array_equal(b["hard_bits"].cpu().numpy(), h)
        np.testing.assert_array_equal(b["iters"].cpu().numpy(), i)
