"""Serving (continuous batching) through the C ABI server (needs a GB300).

Every frame a server decodes must come out exactly as when its batch is decoded alone by the
kernel its pool runs on: the layered QC kernel or the stream kernel for codes whose plain decode
uses it (the default), the TILE kernel for the others or when the server is created with variant
TILE.  Same
hard decisions, iteration counts and syndrome flags, bit for bit, whatever else is in flight,
however many slots the budget gives, and however the decoding is cut into epochs (its state
stays in device memory between launches).
"""
import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I
from parity_rules import check_full

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


def _grouped(nd, name):
    c = I.code_by_name(name)
    code = nd.Code.from_inputs(c)
    g = nd.Groups.build(code, c.M // c.Z, 0.5, 2304, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    return c, code, g


def _alone(nd, torch, g, c, llr, params):
    """The batch decoded alone by the kernel a server with these params uses for the code: the
    layered QC kernel or the stream kernel where the plain decode (variant AUTO) uses it, else
    the tile kernel (and the tile kernel for every code when the server is created with variant
    TILE)."""
    dev = torch.device("cuda")
    p = nd.params_default(**{f: getattr(params, f) for f, _ in params._fields_})
    p.variant = nd.VARIANT_AUTO
    listed = (nd.VARIANT_QC, nd.VARIANT_QC_GLOBAL, nd.VARIANT_STREAM_SMEM, nd.VARIANT_STREAM_GLOBAL,
              nd.VARIANT_STREAM_BULK)
    if params.variant == nd.VARIANT_TILE or g.plan(p, 1024).variant not in listed:
        p.variant = nd.VARIANT_TILE
    F = llr.shape[0]
    d_llr = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).to(dev)
    hard = torch.zeros((F, (c.N + 31) // 32), dtype=torch.int32, device=dev)
    iters = torch.zeros(F, dtype=torch.int32, device=dev)
    ok = torch.zeros(F, dtype=torch.uint8, device=dev)
    ws = torch.zeros(max(1, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
    nd.decode(g, p, d_llr, ws, hard, iters, ok)
    torch.cuda.synchronize()
    return hard.cpu().numpy().view(np.uint32), iters.cpu().numpy(), ok.cpu().numpy()


def _requests(codes, sizes, ebn0, seed):
    """Interleaved requests: (code index, LLRs) with the given frame counts."""
    out = []
    for i, F in enumerate(sizes):
        k = i % len(codes)
        c = codes[k]
        out.append((k, I.channel_llr(c.N, F, ebn0[k], I.design_rate(c), seed=seed + i, dtype=np.float32)))
    return out


@pytest.mark.parametrize("msg", ["f32", "f16"])
@pytest.mark.parametrize("epoch_iters,budget_mb", [(1, 2), (4, 8), (25, 64)])
@pytest.mark.parametrize("kernel", ["auto", "tile"])
def test_served_equals_alone(env, msg, epoch_iters, budget_mb, kernel):
    nd, torch = env
    names = ["qc_n2304_r12", "qc_n1152_r23"]
    built = [_grouped(nd, n) for n in names]
    codes = [b[0] for b in built]
    groups = [b[2] for b in built]
    params = nd.params_default(max_iter=25, msg_dtype={"f32": nd.F32, "f16": nd.F16}[msg],
                               variant=nd.VARIANT_TILE if kernel == "tile" else nd.VARIANT_AUTO)
    srv = nd.Server(groups, params, budget_mb << 20, epoch_iters=epoch_iters)
    try:
        st0 = srv.stats()
        reqs = _requests(codes, [37, 5, 200, 1, 64, 130, 3, 90], [1.25, 2.5], seed=7000)
        handles = [srv.submit(k, llr) for k, llr in reqs]
        for h in handles:
            h.wait(120000)
        st = srv.stats()
    finally:
        srv.close()
    print(f"\n{msg} epoch_iters={epoch_iters} budget {budget_mb} MiB: {st0['slots_total']} slots, "
          f"{st['epochs']} epochs")
    total = 0
    for (k, llr), h in zip(reqs, handles):
        hard, iters, ok = _alone(nd, torch, groups[k], codes[k], llr, params)
        np.testing.assert_array_equal(h.hard_words, hard)
        np.testing.assert_array_equal(h.iters, iters)
        np.testing.assert_array_equal(h.syndrome_ok, ok)
        total += llr.shape[0]
    assert st["frames_completed"] == total
    assert st["requests_completed"] == len(reqs)
    assert st["iterations"] == sum(int(h.iters.sum()) for h in handles)
    assert st["slots_in_use"] == 0


@pytest.mark.parametrize("msg", ["f32", "f16"])
@pytest.mark.parametrize("kernel", ["auto", "tile"])
def test_served_mixed_kernels(env, msg, kernel):
    """A server whose pools run on different kernels (n=576 on the QC kernel, n=8192 on the
    stream kernel -- its 2-layer window does not fit one CTA of the QC kernel -- with FP16
    messages in shared memory and FP32 messages in global memory, as the plain decode plans them;
    or both on the tile kernel), with their launches forked within each epoch: every frame equals
    its batch decoded alone."""
    nd, torch = env
    names = ["qc_n576_r12", "qc_n8192_r2732"]
    built = [_grouped(nd, n) for n in names]
    codes = [b[0] for b in built]
    groups = [b[2] for b in built]
    params = nd.params_default(max_iter=20, msg_dtype={"f32": nd.F32, "f16": nd.F16}[msg],
                               variant=nd.VARIANT_TILE if kernel == "tile" else nd.VARIANT_AUTO)
    if kernel == "auto":
        assert groups[1].plan(nd.params_default(msg_dtype=params.msg_dtype), 1024).variant in (
            nd.VARIANT_STREAM_SMEM, nd.VARIANT_STREAM_GLOBAL)
    srv = nd.Server(groups, params, 48 << 20, epoch_iters=3)
    try:
        reqs = _requests(codes, [300, 40, 7, 120, 64, 33], [2.25, 3.25], seed=7300)
        handles = [srv.submit(k, llr) for k, llr in reqs]
        for h in handles:
            h.wait(120000)
        st = srv.stats()
    finally:
        srv.close()
    for (k, llr), h in zip(reqs, handles):
        hard, iters, ok = _alone(nd, torch, groups[k], codes[k], llr, params)
        np.testing.assert_array_equal(h.hard_words, hard)
        np.testing.assert_array_equal(h.iters, iters)
        np.testing.assert_array_equal(h.syndrome_ok, ok)
    assert st["frames_completed"] == sum(llr.shape[0] for _, llr in reqs)
    assert st["slots_in_use"] == 0


@pytest.mark.parametrize("msg", ["f32", "bf16"])
def test_served_large_code_on_stream_kernel(env, msg):
    """n=16200 (the stream kernel, messages in the slots' global state) beside n=2304 (the QC
    kernel), frames parked every 2 iterations: equal to the batches decoded alone."""
    nd, torch = env
    names = ["qc_n2304_r12", "qc_n16200_r23"]
    built = [_grouped(nd, n) for n in names]
    codes = [b[0] for b in built]
    groups = [b[2] for b in built]
    params = nd.params_default(max_iter=25, msg_dtype={"f32": nd.F32, "bf16": nd.BF16}[msg])
    assert groups[1].plan(nd.params_default(msg_dtype=params.msg_dtype), 1024).variant == nd.VARIANT_STREAM_GLOBAL
    srv = nd.Server(groups, params, 64 << 20, epoch_iters=2)
    try:
        reqs = _requests(codes, [50, 9, 120, 31, 1, 40], [1.75, 1.85], seed=7600)
        handles = [srv.submit(k, llr) for k, llr in reqs]
        for h in handles:
            h.wait(120000)
        st = srv.stats()
    finally:
        srv.close()
    for (k, llr), h in zip(reqs, handles):
        hard, iters, ok = _alone(nd, torch, groups[k], codes[k], llr, params)
        np.testing.assert_array_equal(h.hard_words, hard)
        np.testing.assert_array_equal(h.iters, iters)
        np.testing.assert_array_equal(h.syndrome_ok, ok)
    assert st["frames_completed"] == sum(llr.shape[0] for _, llr in reqs)
    assert st["slots_in_use"] == 0


def test_served_against_oracle(env, oracle_mod):
    """Every served frame of a request against the FP64 oracle, under the rule of
    tests/parity_rules.py (the compared frames are chosen by the oracle alone)."""
    nd, torch = env
    c, code, g = _grouped(nd, "qc_n2304_r12")
    params = nd.params_default(max_iter=25)
    llr = I.channel_llr(c.N, 48, 1.75, I.design_rate(c), seed=7100, dtype=np.float32)
    srv = nd.Server([g], params, 4 << 20, epoch_iters=2)
    try:
        r = srv.submit(0, llr)
        r.wait(60000)
    finally:
        srv.close()
    q = g.query()
    ref = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], llr.astype(np.float64), 25)
    check_full("served n2304", r.hard_bits(), r.iters, r.syndrome_ok, ref, llr.astype(np.float64),
               lambda x: oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], x, 25))


def test_server_budget_and_errors(env):
    nd, torch = env
    c, code, g = _grouped(nd, "qc_n2304_r12")
    params = nd.params_default(max_iter=25)
    with pytest.raises(nd.NdgsbpError) as e:
        nd.Server([g], params, 1024)
    assert e.value.status == nd.ERR_BUDGET
    small = nd.Server([g], params, 1 << 20)
    big = nd.Server([g], params, 16 << 20)
    try:
        assert 0 < small.stats()["slots_total"] < big.stats()["slots_total"]
        with pytest.raises(nd.NdgsbpError) as e:
            small.submit(1, np.zeros((1, c.N), np.float32))
        assert e.value.status == nd.ERR_INVALID
    finally:
        small.close()
        big.close()
    # a Gallager code is not QC: the serving kernel does not take it
    gc = I.code_by_name("gallager36_n1008")
    gcode = nd.Code.from_inputs(gc)
    gg = nd.Groups.build(gcode, 4, 0.4, 1)
    with pytest.raises(nd.NdgsbpError) as e:
        nd.Server([gg], params, 16 << 20)
    assert e.value.status == nd.ERR_UNSUPPORTED


def test_server_wait_timeout_then_complete(env):
    """A bounded host wait that runs out returns TIMEOUT and leaves the request running."""
    nd, torch = env
    c, code, g = _grouped(nd, "qc_n2304_r12")
    params = nd.params_default(max_iter=25)
    llr = I.channel_llr(c.N, 4000, 0.5, I.design_rate(c), seed=7200, dtype=np.float32)
    srv = nd.Server([g], params, 2 << 20, epoch_iters=1)
    try:
        r = srv.submit(0, llr)
        try:
            r.wait(0)
            timed_out = False
        except nd.NdgsbpError as e:
            assert e.status == nd.ERR_TIMEOUT
            timed_out = True
        lat = r.wait(120000)
        assert lat > 0.0 and r.done()
        print(f"\nfirst wait timed out: {timed_out}; latency {lat:.1f} ms")
    finally:
        srv.close()
    hard, iters, ok = _alone(nd, torch, g, c, llr, params)
    np.testing.assert_array_equal(r.hard_words, hard)
    np.testing.assert_array_equal(r.iters, iters)
