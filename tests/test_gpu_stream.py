"""The stream kernel (decode_stream.cu) against the other kernels and the FP64 oracle (GPU).

* One lane per CN: the same arithmetic in the same order as the layered QC kernel, so every
  message storage mode (shared memory, global memory, bulk-staged layer slabs) must give the QC
  kernel's posteriors, hard decisions, iteration counts, flags and final messages bit for bit.
* Two lanes per CN: the tile kernel's lane split and pair products, so equal to the tile kernel
  at 2 lanes per CN bit for bit.
* Codes whose window needs it (n=16200, n=8192): messages after k iterations within 1e-4 of the
  oracle and full decodes under the parity rule of tests/parity_rules.py, in every mode.
"""
import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I
from parity_rules import check_full

pytestmark = pytest.mark.gpu

MSG_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp, torch


def _groups(nd, c, kind, seed=2304, n_groupings=1):
    code = nd.Code.from_inputs(c)
    nl = c.M // c.Z
    if kind == "cyclic":
        return nd.Groups.build(code, nl, 0.5, seed, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC,
                               n_groupings=n_groupings)
    if kind == "linear":
        return nd.Groups.build(code, nl - 1, 0.5, seed, unit=nd.UNIT_LAYER)
    if kind == "one_layer":
        return nd.Groups.build(code, nl, 0.0, seed, unit=nd.UNIT_LAYER)
    raise ValueError(kind)


def _run(nd, torch, g, c, llr, want_msgs=False, **kw):
    _t = torch
    dev = _t.device("cuda")
    F, W = llr.shape[0], (c.N + 31) // 32
    p = nd.params_default(**kw)
    out = dict(hard=_t.full((F, W), -1, dtype=_t.int32, device=dev),
               iters=_t.full((F,), -1, dtype=_t.int32, device=dev),
               ok=_t.full((F,), 7, dtype=_t.uint8, device=dev),
               post=_t.full((F, c.N), float("nan"), dtype=_t.float32, device=dev))
    msgs = _t.zeros((F, c.E), dtype=_t.float32, device=dev) if want_msgs else None
    ws = _t.zeros(max(256, g.workspace_size(p, F)), dtype=_t.uint8, device=dev)
    nd.decode(g, p, _t.from_numpy(llr.astype(np.float32)).to(dev), ws, out["hard"], out["iters"], out["ok"],
              out["post"], messages=msgs)
    _t.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["bits"] = nd.unpack_bits(out["hard"], c.N)
    res["plan"] = g.plan(p, F).as_dict()
    res["status"] = nd.workspace_status(ws)
    if want_msgs:
        res["msgs"] = msgs.cpu().numpy()
    return res


def _plannable(nd, g, F, **kw):
    """False when the plan refuses the parameters (e.g. FP32 messages of n=16200 do not fit in
    shared memory, so STREAM_SMEM is unsupported there)."""
    try:
        g.plan(nd.params_default(**kw), F)
        return True
    except nd.NdgsbpError as e:
        assert e.status == nd.ERR_UNSUPPORTED
        return False


def _same(a, b, label):
    for k in ("post", "iters", "ok", "hard"):
        assert np.array_equal(a[k], b[k], equal_nan=False), f"{label}: {k} differs"
    if "msgs" in a and "msgs" in b:
        assert np.array_equal(a["msgs"], b["msgs"]), f"{label}: messages differ"


MODES = ["smem", "global", "bulk"]


def _variant(nd, mode):
    return {"smem": nd.VARIANT_STREAM_SMEM, "global": nd.VARIANT_STREAM_GLOBAL,
            "bulk": nd.VARIANT_STREAM_BULK}[mode]


@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("kind", ["cyclic", "linear", "one_layer"])
def test_one_lane_equals_qc_kernel(env, kind, msg):
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    g = _groups(nd, c, kind)
    mdt = {"f32": nd.F32, "f16": nd.F16, "bf16": nd.BF16}[msg]
    for F, es in ((301, 1), (37, 0), (1, 1)):
        llr = I.channel_llr(c.N, F, 1.25, 0.5, seed=5000 + F, dtype=np.float32)
        kw = dict(max_iter=18, msg_dtype=mdt, early_stop=es)
        base = _run(nd, torch, g, c, llr, want_msgs=True, variant=nd.VARIANT_QC, **kw)
        assert base["plan"]["variant"] == nd.VARIANT_QC
        for mode in MODES:
            v = _variant(nd, mode)
            if mode == "bulk" and kind == "linear":
                # linear windows do not advance one layer per group around a ring
                with pytest.raises(nd.NdgsbpError) as e:
                    g.plan(nd.params_default(variant=v, lanes_per_cn=1, **kw), F)
                assert e.value.status == nd.ERR_UNSUPPORTED
                continue
            r = _run(nd, torch, g, c, llr, want_msgs=True, variant=v, lanes_per_cn=1, **kw)
            assert r["plan"]["variant"] == v
            assert r["status"] == 0
            _same(r, base, f"{kind}/{msg}/{mode}/F={F}/es={es}")


@pytest.mark.parametrize("mode", ["smem", "global"])
def test_cycled_groupings_equal_qc_kernel(env, mode):
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    g = _groups(nd, c, "cyclic", seed=99, n_groupings=3)
    llr = I.channel_llr(c.N, 96, 1.5, 0.5, seed=321, dtype=np.float32)
    base = _run(nd, torch, g, c, llr, want_msgs=True, max_iter=20, variant=nd.VARIANT_QC)
    r = _run(nd, torch, g, c, llr, want_msgs=True, max_iter=20, variant=_variant(nd, mode), lanes_per_cn=1)
    _same(r, base, f"cycled/{mode}")
    with pytest.raises(nd.NdgsbpError):
        g.plan(nd.params_default(variant=nd.VARIANT_STREAM_BULK), 96)


@pytest.mark.parametrize("name,ebn0", [("qc_n2304_r12", 1.25), ("qc_n2304_r34", 3.0)])
@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_two_lanes_equal_tile_kernel(env, name, ebn0, msg):
    nd, torch = env
    c = I.code_by_name(name)
    g = _groups(nd, c, "cyclic")
    F = 64 if c.N <= 2304 else 24
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=77, dtype=np.float32)
    kw = dict(max_iter=20, msg_dtype=nd.F32 if msg == "f32" else nd.F16, lanes_per_cn=2)
    base = _run(nd, torch, g, c, llr, want_msgs=True, variant=nd.VARIANT_TILE, **kw)
    for mode in MODES:
        r = _run(nd, torch, g, c, llr, want_msgs=True, variant=_variant(nd, mode), **kw)
        assert r["status"] == 0
        _same(r, base, f"{name}/{msg}/{mode}")


def _msg_err(gpu, ref):
    return float(np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), 1.0)))


@pytest.mark.parametrize("name,ebn0", [("qc_n16200_r23", 1.85), ("qc_n8192_r2732", 3.3)])
@pytest.mark.parametrize("mode", MODES)
def test_large_codes_match_oracle(env, oracle_mod, name, ebn0, mode):
    nd, torch = env
    c = I.code_by_name(name)
    g = _groups(nd, c, "cyclic")
    q = g.query()
    F = 12
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=8100, dtype=np.float32)
    l64 = llr.astype(np.float64)
    v = _variant(nd, mode)
    if not _plannable(nd, g, F, variant=v):
        assert mode == "smem" and c.N == 16200   # FP32 messages of n=16200 exceed shared memory
        return
    for k in (1, 2, 5):
        r = _run(nd, torch, g, c, llr, want_msgs=True, max_iter=k, early_stop=0, variant=v)
        assert r["plan"]["variant"] == v
        ref = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], l64, k, early_stop=False, want_c2v=True)
        err = _msg_err(r["msgs"], ref.c2v)
        assert err <= MSG_TOL, (k, err)
        assert (r["iters"] == k).all()
    full = _run(nd, torch, g, c, llr, max_iter=30, variant=v)
    ref = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], l64, 30)
    check_full(f"stream {name} {mode}", full["bits"], full["iters"], full["ok"], ref, l64,
               lambda x: oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], x, 30))
    assert full["status"] == 0


@pytest.mark.parametrize("name", ["qc_n16200_r23", "qc_n8192_r2732"])
def test_auto_plan_and_modes_agree(env, name):
    """AUTO picks the stream kernel for these codes; its three storage modes agree bit for bit
    on a batch larger than the grid (frames refilled as others stop), FP16 messages."""
    nd, torch = env
    c = I.code_by_name(name)
    g = _groups(nd, c, "cyclic")
    p = nd.params_default(max_iter=25, msg_dtype=nd.F16)
    plan = g.plan(p, 10**6)
    assert plan.variant in (nd.VARIANT_STREAM_SMEM, nd.VARIANT_STREAM_GLOBAL, nd.VARIANT_STREAM_BULK)
    F = plan.grid + 37
    ebn0 = 1.85 if c.N == 16200 else 3.3
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=4400, dtype=np.float32)
    runs = {m: _run(nd, torch, g, c, llr, max_iter=25, msg_dtype=nd.F16, variant=_variant(nd, m)) for m in MODES}
    for m in ("global", "bulk"):
        _same(runs[m], runs["smem"], f"{name}/{m}")
    assert all(r["status"] == 0 for r in runs.values())
    it = runs["bulk"]["iters"]
    assert it.min() >= 1 and it.max() <= 25


def test_bulk_wait_gives_up_and_reports(env):
    """The failure path of the bounded mbarrier waits (no GPU fault involved): with the test hook
    every CTA of a STREAM_BULK launch leaves its first bulk load unissued, so that wait can only
    give up.  The launch must end by itself, set bit 0 of the workspace status word and leave the
    outputs of the frames it could not finish unwritten; the next decode on the same context and
    workspace must clear the word and equal the shared-memory mode bit for bit."""
    nd, torch = env
    c = I.code_by_name("qc_n8192_r2732")
    g = _groups(nd, c, "cyclic")
    F = 48
    llr = I.channel_llr(c.N, F, 3.3, I.design_rate(c), seed=4711, dtype=np.float32)
    kw = dict(max_iter=20, msg_dtype=nd.F16)
    try:
        nd.test_hooks(1, 1 << 12)
        bad = _run(nd, torch, g, c, llr, variant=nd.VARIANT_STREAM_BULK, **kw)
    finally:
        nd.test_hooks(0, 0)
    assert bad["status"] & 1
    assert (bad["iters"] == -1).all()          # no frame finished: every CTA stopped on its first
    assert (bad["ok"] == 7).all()
    good = _run(nd, torch, g, c, llr, variant=nd.VARIANT_STREAM_BULK, **kw)
    ref = _run(nd, torch, g, c, llr, variant=nd.VARIANT_STREAM_SMEM, **kw)
    assert good["status"] == 0
    _same(good, ref, "bulk after a given-up wait")
    with pytest.raises(nd.NdgsbpError):
        nd.test_hooks(2, 0)
