"""Groupings cycled by iteration on the GPU (needs a GB300): the QC and tile kernels against the
oracle decoding with the same groupings cycled by iteration, plans that cannot cycle refuse, and
the FER of fixed against cycled groupings on the n=2304 code."""
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


def _oracle_lists(g):
    gps, gcs, off = [], [], 0
    for gp, gc in g.groupings():
        gps.append(gp + off)
        gcs.append(gc)
        off += len(gc)
    return np.stack(gps), np.concatenate(gcs)


def _run(nd, torch, g, c, llr, want_msgs=False, **kw):
    dev = torch.device("cuda")
    F, W = llr.shape[0], (c.N + 31) // 32
    p = nd.params_default(**kw)
    out = dict(hard=torch.zeros((F, W), dtype=torch.int32, device=dev),
               iters=torch.zeros(F, dtype=torch.int32, device=dev),
               ok=torch.zeros(F, dtype=torch.uint8, device=dev),
               post=torch.zeros((F, c.N), dtype=torch.float32, device=dev))
    msgs = torch.zeros((F, c.E), dtype=torch.float32, device=dev) if want_msgs else None
    ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
    nd.decode(g, p, torch.from_numpy(llr.astype(np.float32)).to(dev), ws, out["hard"], out["iters"], out["ok"],
              out["post"], messages=msgs)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["bits"] = nd.unpack_bits(out["hard"], c.N)
    res["plan"] = g.plan(p, F).as_dict()
    if want_msgs:
        res["msgs"] = msgs.cpu().numpy()
    return res


@pytest.mark.parametrize("variant", ["qc", "tile"])
def test_cycled_groupings_match_oracle(env, oracle_mod, variant):
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    code = nd.Code.from_inputs(c)
    g = nd.Groups.build(code, 12, 0.5, 99, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC, n_groupings=3)
    gp, gc = _oracle_lists(g)
    v = nd.VARIANT_QC if variant == "qc" else nd.VARIANT_TILE
    llr = I.channel_llr(c.N, 24, 1.5, 0.5, seed=321)
    l64 = llr.astype(np.float32).astype(np.float64)
    for k in (1, 2, 5):
        r = _run(nd, torch, g, c, llr, want_msgs=True, max_iter=k, early_stop=0, variant=v)
        ref = oracle_mod.ndgsbp_decode(c, gp, gc, l64, k, early_stop=False, want_c2v=True)
        err = np.abs(r["msgs"] - ref.c2v) / np.maximum(np.abs(ref.c2v), 1.0)
        assert err.max() <= MSG_TOL, (k, err.max())
    full = _run(nd, torch, g, c, llr, max_iter=25, variant=v)
    ref = oracle_mod.ndgsbp_decode(c, gp, gc, l64, 25)
    check_full(f"cycled groupings {variant}", full["bits"], full["iters"], full["ok"], ref, l64,
               lambda x: oracle_mod.ndgsbp_decode(c, gp, gc, x, 25))


def test_cycled_qc_and_tile_agree_bitwise_and_refusals(env):
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    code = nd.Code.from_inputs(c)
    g = nd.Groups.build(code, 12, 0.5, 5, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC, n_groupings=4)
    llr = I.channel_llr(c.N, 64, 1.25, 0.5, seed=11)
    a = _run(nd, torch, g, c, llr, max_iter=20, variant=nd.VARIANT_QC)
    b = _run(nd, torch, g, c, llr, max_iter=20, variant=nd.VARIANT_TILE, lanes_per_cn=1)
    assert (a["post"] == b["post"]).all() and (a["iters"] == b["iters"]).all()
    for v in (nd.VARIANT_SMEM,):
        with pytest.raises(nd.NdgsbpError) as e:
            g.plan(nd.params_default(variant=v), 64)
        assert e.value.status == nd.ERR_UNSUPPORTED


def test_fixed_vs_cycled_groupings_fer(env):
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    code = nd.Code.from_inputs(c)
    dev = torch.device("cuda")
    F, W = 131072, (c.N + 31) // 32
    llr = torch.empty((F, c.N), dtype=torch.float32, device=dev)
    hard = torch.empty((F, W), dtype=torch.int32, device=dev)
    from scipy import stats
    print()
    for ebn0 in (1.5, 1.75):
        nd.awgn_llr(code, F, ebn0, 0.5, 5150 + int(ebn0 * 100), llr)
        for K in (1, 8):
            g = nd.Groups.build(code, 12, 0.5, 2304, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC, n_groupings=K)
            p = nd.params_default(max_iter=25)
            st = torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)
            ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
            nd.decode(g, p, llr, ws, hard, stats=st)
            s = st.cpu().numpy()
            fe, n = int(s[nd.STAT_FRAME_ERRORS]), int(s[nd.STAT_FRAMES])
            lo = 0.0 if fe == 0 else stats.beta.ppf(0.025, fe, n - fe + 1)
            hi = stats.beta.ppf(0.975, fe + 1, n - fe)
            print(f"Eb/N0 {ebn0} groupings {K}: FER {fe / n:.3e} [{lo:.3e}, {hi:.3e}], mean iterations "
                  f"{s[nd.STAT_ITERATIONS] / n:.2f}")
            assert 0 < fe / n < 0.1


@pytest.mark.parametrize("kernel", ["auto", "tile"])
def test_cycled_groupings_served_equal_alone(env, kernel):
    """Serving with groupings cycled by iteration: frames parked every 2 iterations resume with
    the grouping of their next iteration (3 groupings, so parking and the cycle fall out of
    step); every frame equals its batch decoded alone by the same kernel."""
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    code = nd.Code.from_inputs(c)
    g = nd.Groups.build(code, 12, 0.5, 7, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC, n_groupings=3)
    v = nd.VARIANT_TILE if kernel == "tile" else nd.VARIANT_AUTO
    params = nd.params_default(max_iter=20, variant=v)
    reqs = [I.channel_llr(c.N, F, 1.5, 0.5, seed=900 + i).astype(np.float32) for i, F in enumerate((50, 7, 120))]
    srv = nd.Server([g], params, 8 << 20, epoch_iters=2)
    try:
        hs = [srv.submit(0, x) for x in reqs]
        for h in hs:
            h.wait(120000)
    finally:
        srv.close()
    for x, h in zip(reqs, hs):
        r = _run(nd, torch, g, c, x, max_iter=20, variant=v)
        np.testing.assert_array_equal(h.iters, r["iters"])
        np.testing.assert_array_equal(h.hard_words, r["hard"].view(np.uint32))
        np.testing.assert_array_equal(h.syndrome_ok, r["ok"])
