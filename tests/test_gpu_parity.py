"""GPU decoder vs the FP64 oracle on identical seeded inputs (needs a GB300).

Tolerances (FP32 messages):
  * CN->VN messages after k = 1, 2, 5 iterations, early stop off:
        |gpu - oracle| <= 1e-4 * max(|oracle|, 1)  on every edge;
  * full decodes, every frame (tests/parity_rules.py): iteration counts and syndrome flags equal
    on every frame whose oracle posterior has no entry below 1e-3; hard decisions equal wherever
    |oracle total LLR| >= 1e-3, except on frames that the oracle fails to decode and whose FP64
    decisions change under a relative 1e-6 perturbation of the LLRs (chosen by the oracle alone);
  * FER/BER inside the oracle's 95% Clopper-Pearson interval.
Lower-precision messages (FP16/BF16) are held to the FER criterion and report their per-edge error.
"""
import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I
from parity_rules import check_full

pytestmark = pytest.mark.gpu

MSG_TOL = 1e-4
NEAR_ZERO = 1e-3


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp, torch


def _groups(nd, c, kind, seed=7):
    code = nd.Code.from_inputs(c)
    if kind == "flood":
        g = nd.Groups.build(code, 1, 0.0, seed)
    elif kind == "gsbp":
        g = nd.Groups.build(code, 4, 0.0, seed)
    elif kind == "ndgsbp":
        g = nd.Groups.build(code, 4, 0.4, seed)
    elif kind == "ndgsbp12":
        g = nd.Groups.build(code, 12, 0.4, seed)
    elif kind == "layers_cyclic":
        g = nd.Groups.build(code, c.M // c.Z, 0.5, seed, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    elif kind == "layers_linear":
        g = nd.Groups.build(code, c.M // c.Z - 1, 0.5, seed, unit=nd.UNIT_LAYER)
    elif kind == "one_cn_per_group":
        # G = M: every group one CN (layered BP in the drawn CN order)
        g = nd.Groups.build(code, c.M, 0.0, seed)
    elif kind == "one_layer_per_group":
        g = nd.Groups.build(code, c.M // c.Z, 0.0, seed, unit=nd.UNIT_LAYER)
    elif kind == "ndgsbp_r07":
        # r > 0.5: Step 1 cannot draw r N_G CNs from G_{g-1} minus G_{g-2}; the window reading
        # takes the last o CNs of G_{g-1}
        g = nd.Groups.build(code, 4, 0.7, seed)
    elif kind == "layers_r07":
        g = nd.Groups.build(code, 4, 0.7, seed, unit=nd.UNIT_LAYER)
    else:
        raise ValueError(kind)
    return code, g


def _run(nd, torch, groups, c, llr, dtype=np.float32, want_msgs=False, stats=False, ref_bits=None,
         **pkw):
    dev = torch.device("cuda")
    F = llr.shape[0]
    W = (c.N + 31) // 32
    t = {np.float32: torch.float32, np.float64: torch.float64}.get(dtype)
    if t is None:
        t = dtype
        d_llr = torch.from_numpy(llr.astype(np.float32)).to(dev).to(t)
    else:
        d_llr = torch.from_numpy(llr.astype(dtype)).to(dev)
    p = nd.params_default(**pkw)
    out = dict(hard=torch.zeros((F, W), dtype=torch.int32, device=dev),
               iters=torch.zeros(F, dtype=torch.int32, device=dev),
               ok=torch.zeros(F, dtype=torch.uint8, device=dev),
               post=torch.zeros((F, c.N), dtype=torch.float32, device=dev))
    msgs = torch.zeros((F, c.E), dtype=torch.float32, device=dev) if want_msgs else None
    st = torch.zeros(nd.STATS_LEN, dtype=torch.int64, device=dev) if stats else None
    hist = torch.zeros(p.max_iter + 1, dtype=torch.int64, device=dev) if stats else None
    ws = torch.zeros(max(1, groups.workspace_size(p, F)), dtype=torch.uint8, device=dev)
    rb = None if ref_bits is None else torch.from_numpy(nd.pack_bits(ref_bits)).to(dev)
    nd.decode(groups, p, d_llr, ws, out["hard"], out["iters"], out["ok"], out["post"],
              messages=msgs, stats=st, iter_hist=hist, ref_bits=rb, ref_per_frame=ref_bits is not None and np.ndim(ref_bits) == 2)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["bits"] = nd.unpack_bits(out["hard"], c.N)
    res["plan"] = groups.plan(p, F).as_dict()
    if want_msgs:
        res["msgs"] = msgs.cpu().numpy()
    if stats:
        res["stats"] = st.cpu().numpy()
        res["hist"] = hist.cpu().numpy()
    return res


def _oracle(O, c, groups, llr, **kw):
    q = groups.query()
    return O.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], llr.astype(np.float32).astype(np.float64), **kw)


def _msg_err(gpu, ref):
    return float(np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), 1.0)))


# ----------------------------------------------------------------------------------------
# per-edge messages after k iterations
# ----------------------------------------------------------------------------------------
MSG_CASES = [
    ("gallager36_n1008", "ndgsbp", 1.5), ("gallager36_n1008", "gsbp", 1.5),
    ("gallager36_n1008", "flood", 1.5), ("gallager36_n1008", "ndgsbp12", 1.0),
    ("qc_n2304_r12", "layers_cyclic", 1.0), ("qc_n2304_r12", "layers_linear", 1.5),
    ("qc_n576_r12", "ndgsbp", 2.0), ("qc_n16200_r23", "layers_cyclic", 2.0),
    ("qc_n8192_r2732", "layers_cyclic", 3.5), ("qc_n2304_r34", "flood", 3.0),
    ("gallager36_n1008", "one_cn_per_group", 1.5), ("gallager36_n1008", "ndgsbp_r07", 1.5),
    ("qc_n576_r12", "one_layer_per_group", 2.0), ("qc_n2304_r12", "layers_r07", 1.5),
]


@pytest.mark.parametrize("name,kind,ebn0", MSG_CASES)
@pytest.mark.parametrize("k", [1, 2, 5])
def test_messages_after_k_iterations(env, oracle_mod, name, kind, ebn0, k):
    nd, torch = env
    c = I.code_by_name(name)
    F = 24 if c.N <= 2304 else 6
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=100 + k)
    code, g = _groups(nd, c, kind)
    gpu = _run(nd, torch, g, c, llr, want_msgs=True, max_iter=k, early_stop=0)
    ref = _oracle(oracle_mod, c, g, llr, max_iter=k, early_stop=False, want_c2v=True)
    err = _msg_err(gpu["msgs"], ref.c2v)
    assert err <= MSG_TOL, f"max relative message error {err:.3g}"
    post_err = np.max(np.abs(gpu["post"] - ref.total) / np.maximum(np.abs(ref.total), 1.0))
    assert post_err <= 4 * MSG_TOL
    assert (gpu["iters"] == k).all()


# ----------------------------------------------------------------------------------------
# full decodes with early stop
# ----------------------------------------------------------------------------------------
FULL_CASES = [
    ("gallager36_n1008", "ndgsbp", 1.5, 50), ("gallager36_n1008", "gsbp", 1.5, 50),
    ("gallager36_n1008", "flood", 1.5, 50), ("qc_n2304_r12", "layers_cyclic", 1.25, 25),
    ("qc_n2304_r12", "flood", 1.25, 50), ("qc_n1152_r23", "layers_cyclic", 2.5, 30),
    ("qc_n576_r12", "layers_cyclic", 2.0, 30),
    ("gallager36_n1008", "one_cn_per_group", 1.5, 50), ("gallager36_n1008", "ndgsbp_r07", 1.5, 50),
    ("qc_n576_r12", "one_layer_per_group", 2.0, 30), ("qc_n2304_r12", "layers_r07", 1.5, 25),
]


@pytest.mark.parametrize("name,kind,ebn0,imax", FULL_CASES)
def test_full_decode_matches_oracle(env, oracle_mod, name, kind, ebn0, imax):
    nd, torch = env
    c = I.code_by_name(name)
    F = 200
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=314)
    code, g = _groups(nd, c, kind)
    gpu = _run(nd, torch, g, c, llr, max_iter=imax)
    ref = _oracle(oracle_mod, c, g, llr, max_iter=imax)
    l64 = llr.astype(np.float32).astype(np.float64)
    check_full(f"{name}/{kind}", gpu["bits"], gpu["iters"], gpu["ok"], ref, l64,
               lambda x: _oracle(oracle_mod, c, g, x, max_iter=imax))
    # the same error-rate statistics
    fer_gpu = (gpu["bits"].any(axis=1)).mean()
    fer_ref = (ref.hard.any(axis=1)).mean()
    lo, hi = _clopper_pearson(int(round(fer_ref * F)), F)
    assert lo <= fer_gpu <= hi, (fer_gpu, fer_ref, lo, hi)
    H = c.dense().astype(np.int64)
    synd = ((gpu["bits"].astype(np.int64) @ H.T) % 2).any(axis=1)
    assert ((~synd).astype(np.uint8) == gpu["ok"]).all()
    assert gpu["iters"].min() >= 1 and gpu["iters"].max() <= imax


def _clopper_pearson(k, n, alpha=0.05):
    from scipy import stats
    lo = 0.0 if k == 0 else stats.beta.ppf(alpha / 2, k, n - k + 1)
    hi = 1.0 if k == n else stats.beta.ppf(1 - alpha / 2, k + 1, n - k)
    return lo, hi


def test_fer_ber_within_ci_c1(env, oracle_mod):
    """Gallager (3,6) n=1008, Eb/N0 1.5 dB, 500 frames, I_max 50: flooding, GSBP and NDGSBP
    (G=4, r=0.4) FER and BER of the GPU inside the oracle's 95% interval."""
    nd, torch = env
    c = I.code_by_name("gallager36_n1008")
    F = 500
    llr = I.channel_llr(c.N, F, 1.5, 0.5, seed=1008)
    for kind in ("flood", "gsbp", "ndgsbp"):
        code, g = _groups(nd, c, kind)
        gpu = _run(nd, torch, g, c, llr.astype(np.float64), dtype=np.float64, max_iter=50, stats=True)
        ref = _oracle(oracle_mod, c, g, llr, max_iter=50)
        fe_ref = int(ref.hard.any(axis=1).sum())
        lo, hi = _clopper_pearson(fe_ref, F)
        fer = gpu["stats"][nd.STAT_FRAME_ERRORS] / F
        assert lo <= fer <= hi, (kind, fer, fe_ref / F)
        be_ref = int(ref.hard.sum())
        blo, bhi = _clopper_pearson(be_ref, F * c.N)
        assert blo <= gpu["stats"][nd.STAT_BIT_ERRORS] / (F * c.N) <= bhi


# ----------------------------------------------------------------------------------------
# independence, determinism, variants, dtypes, edge cases
# ----------------------------------------------------------------------------------------

def test_frame_alone_equals_frame_in_batch(env):
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    llr = I.channel_llr(c.N, 300, 1.25, 0.5, seed=9)
    code, g = _groups(nd, c, "layers_cyclic")
    full = _run(nd, torch, g, c, llr, max_iter=25)
    again = _run(nd, torch, g, c, llr, max_iter=25)
    assert (full["post"] == again["post"]).all()
    for f in (0, 17, 299):
        one = _run(nd, torch, g, c, llr[f:f + 1], max_iter=25)
        assert (one["post"][0] == full["post"][f]).all()
        assert one["iters"][0] == full["iters"][f]
    sub = _run(nd, torch, g, c, llr[::-1].copy(), max_iter=25)
    assert (sub["post"][::-1] == full["post"]).all()


VARIANT_CASES = [("gallager36_n1008", "ndgsbp", False), ("qc_n2304_r12", "layers_cyclic", True),
                 ("qc_n2304_r12", "layers_linear", True), ("qc_n2304_r12", "flood", False),
                 ("qc_n576_r12", "flood", True), ("qc_n2304_r34", "layers_cyclic", True),
                 ("qc_n1152_r23", "layers_cyclic", True)]


@pytest.mark.parametrize("name,kind,qc", VARIANT_CASES)
@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_variants_and_block_sizes_agree_bitwise(env, name, kind, qc, msg):
    """Every kernel variant and launch shape computes the same arithmetic in the same order:
    the table-driven kernel with messages in shared or global memory, any block size, and the
    layered QC kernel give bit-identical posteriors."""
    nd, torch = env
    c = I.code_by_name(name)
    mdt = nd.F32 if msg == "f32" else nd.F16
    sched = nd.SCHEDULE_FLOOD if kind == "flood" else nd.SCHEDULE_GROUPS
    llr = I.channel_llr(c.N, 64, 1.25 if c.M * 2 == c.N else 3.0, I.design_rate(c), seed=77)
    code, g = _groups(nd, c, "layers_cyclic" if (kind == "flood" and c.Z) else kind)
    kw0 = dict(max_iter=20, msg_dtype=mdt, schedule=sched)
    base = _run(nd, torch, g, c, llr, variant=nd.VARIANT_SMEM, **kw0)
    assert base["plan"]["variant"] == nd.VARIANT_SMEM
    others = [dict(variant=nd.VARIANT_GLOBAL), dict(variant=nd.VARIANT_SMEM, block_threads=64),
              dict(variant=nd.VARIANT_GLOBAL, block_threads=128, ctas_per_sm=1)]
    if qc:
        others += [dict(variant=nd.VARIANT_QC), dict(variant=nd.VARIANT_QC_GLOBAL),
                   dict(variant=nd.VARIANT_QC_GLOBAL, ctas_per_sm=1)]
    for kw in others:
        other = _run(nd, torch, g, c, llr, **kw0, **kw)
        if kw["variant"] >= nd.VARIANT_QC:
            assert other["plan"]["variant"] == kw["variant"]
        assert (other["post"] == base["post"]).all(), kw
        assert (other["iters"] == base["iters"]).all()
        assert (other["bits"] == base["bits"]).all()
    auto = _run(nd, torch, g, c, llr, **kw0)
    assert (auto["post"] == base["post"]).all()
    if qc:
        assert auto["plan"]["variant"] == nd.VARIANT_QC


def test_qc_variant_rejected_when_not_layered(env):
    nd, torch = env
    c = I.code_by_name("gallager36_n1008")
    code, g = _groups(nd, c, "ndgsbp")
    with pytest.raises(nd.NdgsbpError) as e:
        g.plan(nd.params_default(variant=nd.VARIANT_QC), 10)
    assert e.value.status == nd.ERR_UNSUPPORTED


def test_llr_dtypes(env, oracle_mod):
    nd, torch = env
    c = I.code_by_name("gallager36_n1008")
    llr = I.channel_llr(c.N, 32, 1.75, 0.5, seed=5)
    code, g = _groups(nd, c, "ndgsbp")
    a = _run(nd, torch, g, c, llr, dtype=np.float32, max_iter=10, early_stop=0)
    b = _run(nd, torch, g, c, llr, dtype=np.float64, max_iter=10, early_stop=0)
    assert (a["post"] == b["post"]).all()
    h = _run(nd, torch, g, c, llr, dtype=torch.float16, max_iter=10)
    ref = _oracle(oracle_mod, c, g, llr, max_iter=10)
    assert (h["bits"].any(axis=1) == ref.hard.any(axis=1)).mean() > 0.9


def test_edge_cases(env, oracle_mod):
    nd, torch = env
    c = I.code_by_name("qc_n576_r12")
    code, g = _groups(nd, c, "layers_cyclic")
    p = nd.params_default(max_iter=5)
    dev = torch.device("cuda")
    # zero frames: a no-op that needs no workspace
    nd.decode(g, p, torch.zeros((0, c.N), device=dev), torch.zeros(1, dtype=torch.uint8, device=dev),
              torch.zeros((0, (c.N + 31) // 32), dtype=torch.int32, device=dev))
    # all-zero LLRs: bit 0 everywhere, the zero syndrome stops at l = 1 (Step 4)
    z = _run(nd, torch, g, c, np.zeros((3, c.N)), max_iter=5)
    assert not z["bits"].any() and (z["iters"] == 1).all() and z["ok"].all()
    # one iteration
    llr = I.channel_llr(c.N, 7, 1.0, 0.5, seed=3)
    one = _run(nd, torch, g, c, llr, max_iter=1, want_msgs=True)
    ref = _oracle(oracle_mod, c, g, llr, max_iter=1, want_c2v=True)
    assert _msg_err(one["msgs"], ref.c2v) <= MSG_TOL and (one["iters"] == 1).all()
    # ragged batch: frames not a multiple of the grid, more frames than CTAs
    plan = g.plan(p, 10**6)
    F = plan.grid + 13
    llr = I.channel_llr(c.N, F, 2.0, 0.5, seed=4)
    r = _run(nd, torch, g, c, llr, max_iter=30)
    sample = np.r_[0:5, F - 5:F]
    ref = _oracle(oracle_mod, c, g, llr[sample], max_iter=30)
    check_full("ragged tail", r["bits"][sample], r["iters"][sample], r["ok"][sample], ref,
               llr[sample].astype(np.float32).astype(np.float64),
               lambda x: _oracle(oracle_mod, c, g, x, max_iter=30))
    # errors are reported, not raised in the kernel
    with pytest.raises(nd.NdgsbpError):
        nd.decode(g, nd.params_default(max_iter=0), torch.zeros((1, c.N), device=dev),
                  torch.zeros(1024, dtype=torch.uint8, device=dev),
                  torch.zeros((1, 18), dtype=torch.int32, device=dev))
    with pytest.raises(nd.NdgsbpError) as e:
        nd.decode(g, p, torch.zeros((4, c.N), device=dev), torch.zeros(1, dtype=torch.uint8, device=dev),
                  torch.zeros((4, 18), dtype=torch.int32, device=dev))
    assert e.value.status == nd.ERR_WORKSPACE


def test_stats_epilogue(env):
    nd, torch = env
    c = I.code_by_name("qc_n1152_r23")
    cw = I.random_codeword(c, seed=11)
    F = 400
    llr = I.channel_llr(c.N, F, 2.0, I.design_rate(c), seed=12, codeword=cw)
    code, g = _groups(nd, c, "layers_cyclic")
    r = _run(nd, torch, g, c, llr, max_iter=20, stats=True, ref_bits=cw)
    err = r["bits"] ^ cw
    assert r["stats"][nd.STAT_FRAMES] == F
    assert r["stats"][nd.STAT_FRAME_ERRORS] == err.any(axis=1).sum()
    assert r["stats"][nd.STAT_BIT_ERRORS] == err.sum()
    assert r["stats"][nd.STAT_ITERATIONS] == r["iters"].sum()
    assert r["stats"][nd.STAT_UNSATISFIED] == (r["ok"] == 0).sum()
    assert r["stats"][nd.STAT_UNDETECTED] == (err.any(axis=1) & (r["ok"] == 1)).sum()
    assert (r["hist"] == np.bincount(r["iters"], minlength=21)).all()


def test_codeword_symmetry_gpu(env):
    """decode(L * (1 - 2c)) = decode(L) xor c on the GPU too (the arithmetic is sign-symmetric)."""
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    cw = I.random_codeword(c, seed=2)
    llr = I.channel_llr(c.N, 64, 1.25, 0.5, seed=13)
    code, g = _groups(nd, c, "layers_cyclic")
    a = _run(nd, torch, g, c, llr, max_iter=25)
    b = _run(nd, torch, g, c, llr * (1.0 - 2.0 * cw), max_iter=25)
    assert ((a["bits"] ^ cw) == b["bits"]).all() and (a["iters"] == b["iters"]).all()
    assert (a["post"] * (1.0 - 2.0 * cw) == b["post"]).all()


# ----------------------------------------------------------------------------------------
# channel generator
# ----------------------------------------------------------------------------------------

def test_philox_bit_exact(env, oracle_mod):
    nd, torch = env
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x89ABCDEF, 0x01234567)
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = torch.zeros_like(d_ctr)
    nd.philox4x32_10(d_ctr, key[0], key[1], out)
    got = out.cpu().numpy().view(np.uint32)
    want = np.array([oracle_mod.philox4x32_10(ctr[i], key) for i in range(len(ctr))])
    assert (got == want).all()


@pytest.mark.parametrize("name,kind,pkw", [("qc_n2304_r12", "layers_cyclic", dict()),
                                            ("qc_n2304_r12", "layers_cyclic", dict(variant=7)),
                                            ("qc_n8192_r2732", "layers_cyclic", dict()),
                                            ("gallager36_n1008", "ndgsbp", dict())])
def test_nonfinite_llrs_mark_frames_invalid(env, name, kind, pkw):
    """A frame whose LLRs hold a NaN or an infinity is not decoded: iteration count 0, syndrome
    flag 0, hard bits and posterior 0, counted in STAT_INVALID only; the other frames of the
    batch get their results as if decoded alone."""
    nd, torch = env
    c = I.code_by_name(name)
    F = 24
    llr = I.channel_llr(c.N, F, 2.0 if c.N <= 2304 else 3.3, I.design_rate(c), seed=808).astype(np.float32)
    bad = {3: np.nan, 7: np.inf, 11: -np.inf, 23: np.nan}
    dirty = llr.copy()
    for f, v in bad.items():
        dirty[f, (f * 37) % c.N] = v
    code, g = _groups(nd, c, kind)
    for dt in (np.float32, np.float64):
        r = _run(nd, torch, g, c, dirty, dtype=dt, stats=True, max_iter=20, **pkw)
        clean_idx = np.array([f for f in range(F) if f not in bad])
        alone = _run(nd, torch, g, c, llr[clean_idx], dtype=dt, stats=True, max_iter=20, **pkw)
        for f in bad:
            assert r["iters"][f] == 0 and r["ok"][f] == 0, f
            assert not r["bits"][f].any() and not r["post"][f].any(), f
        for k in ("iters", "ok", "hard", "post"):
            assert (r[k][clean_idx] == alone[k]).all(), k
        st = r["stats"]
        assert st[nd.STAT_INVALID] == len(bad) and st[nd.STAT_FRAMES] == F - len(bad)
        assert st[nd.STAT_ITERATIONS] == int(alone["iters"].sum())
        assert r["hist"][0] == 0 and r["hist"].sum() == F - len(bad)


def test_philox_matches_curand_host_generator(env):
    """The GPU generator equals cuRAND's host Philox4x32-10 (an implementation independent of
    this project and of the oracle) on the keys and counters of tests/curand_host.py."""
    import curand_host as CH
    nd, torch = env
    lib = CH.library()
    if lib is None:
        pytest.skip("cuRAND is not installed")
    for seed, j0 in CH.CASES:
        want = CH.blocks(lib, seed, j0, 64)
        ctr = np.array([CH.counter_of(j0 + i) for i in range(64)], dtype=np.uint32)
        d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
        out = torch.zeros_like(d_ctr)
        k = CH.key_of(seed)
        nd.philox4x32_10(d_ctr, k[0], k[1], out)
        assert (out.cpu().numpy().view(np.uint32) == want).all(), hex(seed)


def test_awgn_llr_unaligned_output_view(env):
    """An output that starts 4 or 8 bytes into a buffer (rows not 16-byte aligned) takes the
    element-store path and gets the same LLRs as an aligned buffer."""
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    code = nd.Code.from_inputs(c)
    F = 37
    ref = torch.zeros((F, c.N), dtype=torch.float32, device="cuda")
    nd.awgn_llr(code, F, 1.5, 0.5, 99, ref)
    for shift in (1, 2, 3):
        buf = torch.zeros(F * c.N + 4, dtype=torch.float32, device="cuda")
        view = buf[shift:shift + F * c.N].view(F, c.N)
        assert view.data_ptr() % 16 != 0
        nd.awgn_llr(code, F, 1.5, 0.5, 99, view)
        torch.cuda.synchronize()
        assert torch.equal(view, ref), shift
        assert float(buf[:shift].abs().sum()) == 0.0 and float(buf[shift + F * c.N:].abs().sum()) == 0.0
    # a pointer not aligned to its element is refused before any launch
    import ctypes
    raw = torch.zeros(F * c.N * 4 + 16, dtype=torch.uint8, device="cuda")
    st = nd._lib.ndgsbp_awgn_llr(code.handle, F, 1.5, 0.5, 99, None, 0, ctypes.c_void_p(raw.data_ptr() + 1),
                                 nd.F32, None)
    assert st == nd.ERR_INVALID


@pytest.mark.parametrize("name", ["qc_n2304_r12", "gallager36_n1008", "qc_n576_r12"])
def test_awgn_llr_matches_oracle(env, oracle_mod, name):
    nd, torch = env
    c = I.code_by_name(name)
    code = nd.Code.from_inputs(c)
    F = 300
    seed = 0x1234_5678_9ABC
    cw = I.random_codeword(c, seed=3)
    out = torch.zeros((F, c.N), dtype=torch.float32, device="cuda")
    nd.awgn_llr(code, F, 1.5, 0.5, seed, out, codeword_bits=torch.from_numpy(nd.pack_bits(cw)).cuda())
    torch.cuda.synchronize()
    ref = oracle_mod.awgn_llr(c.N, F, 1.5, 0.5, seed, codeword=cw)
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) < 2e-5
    half = torch.zeros((F, c.N), dtype=torch.float16, device="cuda")
    nd.awgn_llr(code, F, 1.5, 0.5, seed, half, codeword_bits=torch.from_numpy(nd.pack_bits(cw)).cuda())
    torch.cuda.synchronize()
    assert np.max(np.abs(half.float().cpu().numpy() - ref) / np.maximum(np.abs(ref), 1.0)) < 2e-3


# ----------------------------------------------------------------------------------------
# full size, bench launch configuration: sampled frames and invariants
# ----------------------------------------------------------------------------------------

def test_full_size_qc2304_sampled(env, oracle_mod):
    """65,536 frames of the n=2304 code, NDGSBP over 12 cyclic 2-layer windows, I_max 25, in the
    benchmark's launch configuration: sampled frames against the oracle, every frame's syndrome
    flag against its hard decisions."""
    nd, torch = env
    c = I.code_by_name("qc_n2304_r12")
    code, g = _groups(nd, c, "layers_cyclic")
    F = 65536
    dev = torch.device("cuda")
    host = I.channel_llr(c.N, F, 1.25, 0.5, seed=99, dtype=np.float32)
    llr = torch.from_numpy(host).to(dev)
    p = nd.params_default(max_iter=25)
    W = (c.N + 31) // 32
    hard = torch.zeros((F, W), dtype=torch.int32, device=dev)
    iters = torch.zeros(F, dtype=torch.int32, device=dev)
    ok = torch.zeros(F, dtype=torch.uint8, device=dev)
    ws = torch.zeros(g.workspace_size(p, F), dtype=torch.uint8, device=dev)
    nd.decode(g, p, llr, ws, hard, iters, ok)
    torch.cuda.synchronize()
    sample = np.random.default_rng(0).choice(F, 48, replace=False)
    host_llr = host[sample].astype(np.float64)
    q = g.query()
    ref = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], host_llr, 25)
    bits = nd.unpack_bits(hard[torch.from_numpy(sample).to(dev)], c.N)
    it = iters.cpu().numpy()
    check_full("n2304 65536-frame launch, sampled", bits, it[sample], ok.cpu().numpy()[sample], ref, host_llr,
               lambda x: oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], x, 25))
    # invariants on every frame
    allbits = nd.unpack_bits(hard, c.N)
    H = c.dense().astype(np.int64)
    synd_ok = ~(((allbits.astype(np.int64) @ H.T) % 2).any(axis=1))
    assert (synd_ok.astype(np.uint8) == ok.cpu().numpy()).all()
    assert it.min() >= 1 and it.max() <= 25


# ----------------------------------------------------------------------------------------
# tile kernel: lanes per CN, frames per CTA, large windows
# ----------------------------------------------------------------------------------------
TILE_CASES = [("qc_n2304_r12", "layers_cyclic", (1, 2), 1.25), ("qc_n576_r12", "flood", (1, 2, 4), 2.0),
              ("qc_n2304_r34", "layers_cyclic", (2, 4), 3.0), ("qc_n1152_r23", "layers_cyclic", (2, 4), 2.5),
              ("qc_n8192_r2732", "layers_cyclic", (4,), 3.5), ("qc_n16200_r23", "layers_cyclic", (2, 4), 2.0)]


@pytest.mark.parametrize("name,kind,lanes,ebn0", TILE_CASES)
def test_tile_kernel(env, oracle_mod, name, kind, lanes, ebn0):
    """One lane per CN reproduces the other kernels bit for bit; 2 or 4 lanes per CN combine the
    tanh product in another order and are held to the message tolerance against the oracle.
    Any number of frames per CTA gives the same result as one."""
    nd, torch = env
    c = I.code_by_name(name)
    F = 40 if c.N <= 2304 else 8
    sched = nd.SCHEDULE_FLOOD if kind == "flood" else nd.SCHEDULE_GROUPS
    code, g = _groups(nd, c, "layers_cyclic")
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=4242)
    q = g.query()
    if kind == "flood":
        ref_k = oracle_mod.flood_decode(c, llr.astype(np.float32).astype(np.float64), 2, early_stop=False,
                                        want_c2v=True)
        ref_full = oracle_mod.flood_decode(c, llr.astype(np.float32).astype(np.float64), 30)
    else:
        ref_k = _oracle(oracle_mod, c, g, llr, max_iter=2, early_stop=False, want_c2v=True)
        ref_full = _oracle(oracle_mod, c, g, llr, max_iter=30)
    l64 = llr.astype(np.float32).astype(np.float64)
    if kind == "flood":
        rerun = lambda x: oracle_mod.flood_decode(c, x, 30)   # noqa: E731
    else:
        rerun = lambda x: _oracle(oracle_mod, c, g, x, max_iter=30)   # noqa: E731
    for tpc in lanes:
        kw = dict(variant=nd.VARIANT_TILE, lanes_per_cn=tpc, schedule=sched)
        first = None
        for fpc in (1, 3, 16):
            r2 = _run(nd, torch, g, c, llr, want_msgs=True, max_iter=2, early_stop=0, frames_per_cta=fpc, **kw)
            assert r2["plan"]["variant"] == nd.VARIANT_TILE
            assert _msg_err(r2["msgs"], ref_k.c2v) <= MSG_TOL, (tpc, fpc)
            full = _run(nd, torch, g, c, llr, max_iter=30, frames_per_cta=fpc, **kw)
            check_full(f"{name} tile tpc={tpc} fpc={fpc}", full["bits"], full["iters"], full["ok"], ref_full, l64,
                       rerun)
            if first is None:
                first = full
            else:
                assert (full["post"] == first["post"]).all(), (tpc, fpc)
        if tpc == 1:
            base = _run(nd, torch, g, c, llr, max_iter=30, schedule=sched, variant=nd.VARIANT_SMEM)
            assert (first["post"] == base["post"]).all()
