"""Decoding with structure-aware groups (needs a GB300): parity with the oracle on the same
groups, and the FER of structured against random Step 1 groups on the n=1008 Gallager code
(G = 12, r = 0 and 0.4), reported with 95% Clopper-Pearson intervals."""
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


def _cp(k, n):
    from scipy import stats
    lo = 0.0 if k == 0 else stats.beta.ppf(0.025, k, n - k + 1)
    hi = 1.0 if k == n else stats.beta.ppf(0.975, k + 1, n - k)
    return lo, hi


def test_structured_groups_decode_like_oracle(env, oracle_mod):
    nd, torch = env
    c = I.code_by_name("gallager36_n1008")
    code = nd.Code.from_inputs(c)
    g = nd.Groups.build(code, 12, 0.4, 2024, flags=nd.GROUPS_STRUCTURED)
    llr = I.channel_llr(c.N, 96, 1.75, 0.5, seed=31)
    dev = torch.device("cuda")
    p = nd.params_default(max_iter=35)
    F, W = llr.shape[0], (c.N + 31) // 32
    hard = torch.zeros((F, W), dtype=torch.int32, device=dev)
    iters = torch.zeros(F, dtype=torch.int32, device=dev)
    ok = torch.zeros(F, dtype=torch.uint8, device=dev)
    ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
    nd.decode(g, p, torch.from_numpy(llr.astype(np.float32)).to(dev), ws, hard, iters, ok)
    q = g.query()
    l64 = llr.astype(np.float32).astype(np.float64)
    ref = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], l64, 35)
    check_full("structured groups", nd.unpack_bits(hard, c.N), iters.cpu().numpy(), ok.cpu().numpy(), ref, l64,
               lambda x: oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], x, 35))


def test_structured_vs_random_fer(env):
    nd, torch = env
    c = I.code_by_name("gallager36_n1008")
    code = nd.Code.from_inputs(c)
    dev = torch.device("cuda")
    F, W = 200000, (c.N + 31) // 32
    llr = torch.empty((F, c.N), dtype=torch.float32, device=dev)
    hard = torch.empty((F, W), dtype=torch.int32, device=dev)
    rows = []
    for ebn0 in (1.75, 2.0):
        nd.awgn_llr(code, F, ebn0, 0.5, 4100 + int(ebn0 * 100), llr)
        for r in (0.0, 0.4):
            for kind, flags in (("random", 0), ("structured", nd.GROUPS_STRUCTURED)):
                g = nd.Groups.build(code, 12, r, 2024, flags=flags)
                # equal CN-update budget: I = floor(50 M / U)
                imax = int(50 * c.M // g.query()["cn_updates_per_iter"])
                p = nd.params_default(max_iter=imax)
                st = torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev)
                ws = torch.zeros(max(256, g.workspace_size(p, F)), dtype=torch.uint8, device=dev)
                nd.decode(g, p, llr, ws, hard, stats=st)
                s = st.cpu().numpy()
                fe, n = int(s[nd.STAT_FRAME_ERRORS]), int(s[nd.STAT_FRAMES])
                lo, hi = _cp(fe, n)
                rows.append((ebn0, r, kind, imax, g.query()["cocsg"], fe / n, lo, hi,
                             s[nd.STAT_ITERATIONS] / n))
    print()
    for row in rows:
        print("Eb/N0 %.2f r=%.1f %-10s I_max %d  CoCSG %6.1f  FER %.3e [%.3e, %.3e]  mean it %.2f" % row)
    assert all(0.0 <= row[5] < 0.5 for row in rows)
