"""Vertical (VN-group) shuffled BP on the GPU (vertical.cu) against the FP64 oracle's vertical
decoder (oracle_vertical_decode), on the same VN groups (GPU).

* messages after k = 1, 2, 5 iterations within 1e-4 (relative, floor 1) of the oracle's, for
  G = 1 (flooding), a few random groups, and G = N (one VN at a time);
* full decodes under the parity rule of tests/parity_rules.py on every frame;
* G = 1 against the oracle's textbook flooding decoder;
* messages in shared memory and in the workspace give the same results bit for bit, and any
  block size does too (same arithmetic in the same order per edge and per VN);
* 16-bit messages, the NaN/infinity rule, zero frames and the workspace checks.
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


def _run(nd, torch, vg, c, llr, want_msgs=False, llr_dtype=None, **kw):
    dev = torch.device("cuda")
    F, W = llr.shape[0], (c.N + 31) // 32
    p = nd.params_default(**kw)
    hard = torch.full((F, W), -1, dtype=torch.int32, device=dev)
    iters = torch.full((F,), -1, dtype=torch.int32, device=dev)
    ok = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    post = torch.full((F, c.N), float("nan"), dtype=torch.float32, device=dev)
    msgs = torch.zeros((F, c.E), dtype=torch.float32, device=dev) if want_msgs else None
    stats = torch.zeros(8, dtype=torch.int64, device=dev)
    ws = torch.zeros(max(256, vg.workspace_size(p, F)), dtype=torch.uint8, device=dev)
    x = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).to(dev)
    if llr_dtype is not None:
        x = x.to(llr_dtype)
    nd.decode_vertical(vg, p, x, ws, hard, iters, ok, post, stats=stats, messages=msgs)
    torch.cuda.synchronize()
    res = dict(hard=hard.cpu().numpy(), iters=iters.cpu().numpy(), ok=ok.cpu().numpy(),
               post=post.cpu().numpy(), stats=stats.cpu().numpy())
    res["bits"] = nd.unpack_bits(hard, c.N)
    if want_msgs:
        res["msgs"] = msgs.cpu().numpy()
    return res


def _msg_err(gpu, ref):
    return float(np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), 1.0)))


def _vgroups(nd, c, G, seed):
    code = nd.Code.from_inputs(c)
    vg = nd.VGroups.build(code, G, seed)
    q = vg.query()
    return vg, q["grp_ptr"], q["grp_vn"]


CASES = [("gallager36_n1008", 1, 1.75), ("gallager36_n1008", 7, 1.75), ("gallager36_n1008", 64, 1.75),
         ("qc_n2304_r12", 5, 1.5), ("qc_n576_r12", 576, 2.0), ("qc_n2304_r34", 3, 3.0)]


@pytest.mark.parametrize("name,G,ebn0", CASES)
def test_messages_match_oracle(env, oracle_mod, name, G, ebn0):
    nd, torch = env
    c = I.code_by_name(name)
    vg, gp, gv = _vgroups(nd, c, G, seed=31 + G)
    F = 24
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=700 + G, dtype=np.float32)
    l64 = llr.astype(np.float64)
    for k in (1, 2, 5):
        r = _run(nd, torch, vg, c, llr, want_msgs=True, max_iter=k, early_stop=0)
        ref = oracle_mod.vertical_decode(c, gp, gv, l64, k, early_stop=False, want_c2v=True)
        err = _msg_err(r["msgs"], ref.c2v)
        assert err <= MSG_TOL, (k, err)
        post_err = float(np.max(np.abs(r["post"] - ref.total) / np.maximum(np.abs(ref.total), 1.0)))
        assert post_err <= 4 * MSG_TOL, (k, post_err)
        assert (r["iters"] == k).all()


@pytest.mark.parametrize("name,G,ebn0", CASES)
def test_full_decode_parity(env, oracle_mod, name, G, ebn0):
    nd, torch = env
    c = I.code_by_name(name)
    vg, gp, gv = _vgroups(nd, c, G, seed=5 + G)
    F = 200 if c.N <= 1008 else 96
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=9100 + G, dtype=np.float32)
    l64 = llr.astype(np.float64)
    r = _run(nd, torch, vg, c, llr, max_iter=30)
    dec = lambda x: oracle_mod.vertical_decode(c, gp, gv, x, 30)
    ref = dec(l64)
    check_full(f"vertical {name} G={G}", r["bits"], r["iters"], r["ok"], ref, l64, dec)
    # fused statistics against the all-zero transmitted word
    assert r["stats"][0] == F
    assert r["stats"][4] == int(r["iters"].sum())


def test_one_group_is_flooding(env, oracle_mod):
    nd, torch = env
    c = I.code_by_name("gallager36_n1008")
    vg, gp, gv = _vgroups(nd, c, 1, seed=0)
    llr = I.channel_llr(c.N, 16, 1.5, 0.5, seed=44, dtype=np.float32)
    l64 = llr.astype(np.float64)
    r = _run(nd, torch, vg, c, llr, want_msgs=True, max_iter=4, early_stop=0)
    ref = oracle_mod.flood_decode(c, l64, 4, early_stop=False, want_c2v=True)
    assert _msg_err(r["msgs"], ref.c2v) <= MSG_TOL


def test_storage_and_block_sizes_agree_bitwise(env):
    """The messages in shared memory (SMEM, what AUTO picks for this code) or in the workspace
    slot (GLOBAL), and any block size, give the same bits."""
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    vg, _, _ = _vgroups(nd, c, 6, seed=3)
    llr = I.channel_llr(c.N, 150, 1.4, 0.5, seed=8, dtype=np.float32)
    base = _run(nd, torch, vg, c, llr, want_msgs=True, max_iter=25, variant=nd.VARIANT_SMEM)
    assert vg.workspace_size(nd.params_default(), 150) == 256
    assert vg.workspace_size(nd.params_default(variant=nd.VARIANT_GLOBAL), 150) > 256
    for kw in (dict(), dict(block_threads=64), dict(block_threads=512), dict(block_threads=160, ctas_per_sm=1),
               dict(variant=nd.VARIANT_GLOBAL), dict(variant=nd.VARIANT_GLOBAL, block_threads=96)):
        o = _run(nd, torch, vg, c, llr, want_msgs=True, max_iter=25, **kw)
        for k in ("post", "iters", "ok", "hard", "msgs"):
            assert np.array_equal(o[k], base[k]), (kw, k)


def test_large_code_uses_workspace_messages(env, oracle_mod):
    """n=16200: the messages (217 KB per frame in FP32, 109 KB in FP16) do not fit in shared
    memory beside the 130 KB of P and L, so they live in the workspace slot; results still match
    the oracle.  For n=2304 they stay in shared memory (no slot)."""
    nd, torch = env
    c = I.code_by_name("qc_n16200_r23")
    vg, gp, gv = _vgroups(nd, c, 9, seed=1)
    p = nd.params_default()
    slot = vg.workspace_size(p, 1) - 256
    assert slot >= 4 * c.E
    with pytest.raises(nd.NdgsbpError) as e:
        vg.workspace_size(nd.params_default(variant=nd.VARIANT_SMEM), 1)
    assert e.value.status == nd.ERR_UNSUPPORTED
    llr = I.channel_llr(c.N, 6, 1.85, I.design_rate(c), seed=61, dtype=np.float32)
    l64 = llr.astype(np.float64)
    r = _run(nd, torch, vg, c, llr, want_msgs=True, max_iter=2, early_stop=0)
    ref = oracle_mod.vertical_decode(c, gp, gv, l64, 2, early_stop=False, want_c2v=True)
    assert _msg_err(r["msgs"], ref.c2v) <= MSG_TOL
    assert vg.workspace_size(nd.params_default(msg_dtype=nd.F16), 1) - 256 >= 2 * c.E
    h = _run(nd, torch, vg, c, llr, want_msgs=True, max_iter=1, early_stop=0, msg_dtype=nd.F16)
    ref1 = oracle_mod.vertical_decode(c, gp, gv, l64, 1, early_stop=False, want_c2v=True)
    assert _msg_err(h["msgs"], ref1.c2v) <= 2e-3
    small = I.code_by_name("qc_n2304_r12")
    vs, _, _ = _vgroups(nd, small, 9, seed=1)
    assert vs.workspace_size(p, 1000) == 256


@pytest.mark.parametrize("msg", ["f16", "bf16"])
def test_16bit_messages(env, oracle_mod, msg):
    nd, torch = env
    c = I.code_by_name("gallager36_n1008")
    vg, gp, gv = _vgroups(nd, c, 7, seed=2)
    mdt = nd.F16 if msg == "f16" else nd.BF16
    llr = I.channel_llr(c.N, 300, 2.25, 0.5, seed=12, dtype=np.float32)
    l64 = llr.astype(np.float64)
    one = _run(nd, torch, vg, c, llr[:20], want_msgs=True, max_iter=1, early_stop=0, msg_dtype=mdt)
    ref1 = oracle_mod.vertical_decode(c, gp, gv, l64[:20], 1, early_stop=False, want_c2v=True)
    assert _msg_err(one["msgs"], ref1.c2v) <= (2e-3 if msg == "f16" else 1.6e-2)
    r = _run(nd, torch, vg, c, llr, max_iter=30, msg_dtype=mdt)
    ref = oracle_mod.vertical_decode(c, gp, gv, l64, 30)
    # frame error rates agree: every frame the oracle decodes to the transmitted (all-zero)
    # word is decoded to it too, but for at most 1 % of the frames
    good = (ref.synd_ok == 1) & ~ref.hard.any(axis=1)
    lost = good & r["bits"].any(axis=1)
    assert lost.sum() <= 0.01 * len(good), int(lost.sum())


def test_invalid_and_empty(env):
    nd, torch = env
    c = I.code_by_name("qc_n576_r12")
    vg, _, _ = _vgroups(nd, c, 4, seed=0)
    llr = I.channel_llr(c.N, 5, 2.5, 0.5, seed=1, dtype=np.float32)
    llr[1, 7] = np.nan
    llr[3, 0] = np.inf
    r = _run(nd, torch, vg, c, llr, max_iter=20)
    for f in (1, 3):
        assert r["iters"][f] == 0 and r["ok"][f] == 0 and not r["bits"][f].any() and (r["post"][f] == 0).all()
    assert (r["iters"][[0, 2, 4]] >= 1).all()
    assert r["stats"][nd.STAT_INVALID] == 2 and r["stats"][0] == 3
    # all-zero LLRs: the zero word satisfies every check after one iteration
    z = _run(nd, torch, vg, c, np.zeros((3, c.N), np.float32), max_iter=5)
    assert not z["bits"].any() and (z["iters"] == 1).all() and z["ok"].all()
    # zero frames: a no-op that needs no workspace
    dev = torch.device("cuda")
    p = nd.params_default()
    nd.decode_vertical(vg, p, torch.zeros((0, c.N), device=dev), torch.zeros(1, dtype=torch.uint8, device=dev),
                       torch.zeros((0, (c.N + 31) // 32), dtype=torch.int32, device=dev))
    # too small a workspace, and block_threads above the instance's bound
    need = vg.workspace_size(p, 10)
    with pytest.raises(nd.NdgsbpError) as e:
        nd.decode_vertical(vg, p, torch.zeros((10, c.N), device=dev), torch.zeros(need - 256, dtype=torch.uint8,
                           device=dev), torch.zeros((10, (c.N + 31) // 32), dtype=torch.int32, device=dev))
    assert e.value.status in (nd.ERR_WORKSPACE,)
    with pytest.raises(nd.NdgsbpError) as e:
        vg.workspace_size(nd.params_default(block_threads=1024), 10)
    assert e.value.status == nd.ERR_INVALID


def test_llr_dtypes_agree(env):
    nd, torch = env
    c = I.code_by_name("gallager36_n1008")
    vg, _, _ = _vgroups(nd, c, 7, seed=4)
    llr = I.channel_llr(c.N, 32, 1.75, 0.5, seed=5, dtype=np.float32)
    a = _run(nd, torch, vg, c, llr, max_iter=10, early_stop=0)
    b = _run(nd, torch, vg, c, llr, max_iter=10, early_stop=0, llr_dtype=torch.float64)
    assert np.array_equal(a["post"], b["post"])
