"""Reduced-precision message storage (FP16, BF16) against the FP64 oracle (needs a GB300).

The kernels compute Eq. (1) in FP32 and round only the stored CN->VN messages; the posterior
absorbs the rounded values.  In the first flooding iteration every CN reads the exact channel
LLRs, so each message is an FP32-accurate value rounded once: its error is at most half an ulp of
the storage type (2^-11 relative for FP16, 2^-8 for BF16) plus the FP32 tolerance.  Grouped
schedules already feed rounded messages of earlier groups into later ones within the first
iteration, and later iterations compound that; there the per-edge error is stated (printed) and
bounded loosely, and the decisions are held to the error-rate criterion: FER inside the oracle's
95% Clopper-Pearson interval on the same frames, and an exact McNemar test on the frames where
only one of the two is in error (no systematic loss); FP32 storage also to the full parity rule.
"""
import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I

pytestmark = pytest.mark.gpu

HALF_ULP = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
LOOSE = {"f16": 2e-2, "bf16": 1e-1}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp, torch


def _layers(nd, c):
    code = nd.Code.from_inputs(c)
    return code, nd.Groups.build(code, c.M // c.Z, 0.5, 2304, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)


def _decode(nd, torch, g, c, llr, msg, want_msgs=False, **kw):
    dev = torch.device("cuda")
    F = llr.shape[0]
    p = nd.params_default(msg_dtype={"f32": nd.F32, "f16": nd.F16, "bf16": nd.BF16}[msg], **kw)
    d_llr = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).to(dev)
    hard = torch.zeros((F, (c.N + 31) // 32), dtype=torch.int32, device=dev)
    iters = torch.zeros(F, dtype=torch.int32, device=dev)
    ok = torch.zeros(F, dtype=torch.uint8, device=dev)
    msgs = torch.zeros((F, c.E), dtype=torch.float32, device=dev) if want_msgs else None
    ws = torch.zeros(g.workspace_size(p, F), dtype=torch.uint8, device=dev)
    nd.decode(g, p, d_llr, ws, hard, iters, ok, messages=msgs)
    torch.cuda.synchronize()
    return (nd.unpack_bits(hard, c.N), iters.cpu().numpy(), ok.cpu().numpy(),
            None if msgs is None else msgs.cpu().numpy())


def _cp(k, n, alpha=0.05):
    from scipy import stats
    lo = 0.0 if k == 0 else stats.beta.ppf(alpha / 2, k, n - k + 1)
    hi = 1.0 if k == n else stats.beta.ppf(1 - alpha / 2, k + 1, n - k)
    return lo, hi


@pytest.mark.parametrize("name", ["qc_n2304_r12", "qc_n16200_r23"])
@pytest.mark.parametrize("msg", ["f16", "bf16"])
@pytest.mark.parametrize("k", [1, 2, 5])
def test_low_precision_message_error(env, oracle_mod, name, msg, k):
    nd, torch = env
    c = I.code_by_name(name)
    F = 16 if c.N <= 2304 else 4
    ebn0 = 1.5 if c.N <= 2304 else 2.0
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=500 + k, dtype=np.float32)
    code, g = _layers(nd, c)
    _, _, _, msgs = _decode(nd, torch, g, c, llr, msg, want_msgs=True, max_iter=k, early_stop=0)
    q = g.query()
    ref = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], llr.astype(np.float64), k,
                                   early_stop=False, want_c2v=True)
    err = np.abs(msgs - ref.c2v) / np.maximum(np.abs(ref.c2v), 1.0)
    print(f"\n{name} {msg} NDGSBP k={k}: max per-edge error {err.max():.3e} (relative to max(|L|,1)), "
          f"mean {err.mean():.3e}")
    assert err.max() <= LOOSE[msg]
    if k == 1:
        # flooding, first iteration: one rounding of an FP32-accurate value
        _, _, _, fm = _decode(nd, torch, g, c, llr, msg, want_msgs=True, max_iter=1, early_stop=0,
                              schedule=nd.SCHEDULE_FLOOD)
        fref = oracle_mod.flood_decode(c, llr.astype(np.float64), 1, early_stop=False, want_c2v=True)
        ferr = np.abs(fm - fref.c2v) / np.maximum(np.abs(fref.c2v), 1.0)
        print(f"{name} {msg} flooding k=1: max per-edge error {ferr.max():.3e}")
        assert ferr.max() <= HALF_ULP[msg] * 1.01 + 1e-5


FER_CASES = [("qc_n2304_r12", 1.75, 20000), ("qc_n16200_r23", 1.85, 12000)]
_ORACLE = {}


def _oracle_once(oracle_mod, c, g, llr, name):
    """The oracle's decode of a case's frames, computed once for the three storage types."""
    if name not in _ORACLE:
        q = g.query()
        _ORACLE[name] = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], llr.astype(np.float64), 25)
    return _ORACLE[name]


def _mcnemar_p(b, c):
    """Exact two-sided McNemar test on the discordant pairs (b: oracle in error, GPU not; c: the
    reverse): the probability of a split at least this uneven if both are equally likely."""
    from scipy import stats
    n = b + c
    if n == 0:
        return 1.0
    return float(min(1.0, 2.0 * stats.binom.cdf(min(b, c), n, 0.5)))


@pytest.mark.parametrize("name,ebn0,F", FER_CASES)
@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_low_precision_fer_inside_oracle_ci(env, oracle_mod, name, ebn0, F, msg):
    """FP32/FP16/BF16 message storage against the FP64 oracle on the same frames (all-zero
    codeword, cyclic 2-layer NDGSBP, I_max 25): FER inside the oracle's 95% interval; the frames
    on which exactly one of the two is in error split evenly between the two directions (exact
    McNemar test, p >= 0.01: no systematic loss from the storage type); FP32 is also held to the
    full parity rule of tests/parity_rules.py."""
    nd, torch = env
    c = I.code_by_name(name)
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=9000 + int(ebn0 * 100), dtype=np.float32)
    code, g = _layers(nd, c)
    bits, iters, ok, _ = _decode(nd, torch, g, c, llr, msg, max_iter=25)
    ref = _oracle_once(oracle_mod, c, g, llr, name)
    e_ref = ref.hard.any(axis=1)
    e_gpu = bits.any(axis=1)
    fe_ref, fe = int(e_ref.sum()), int(e_gpu.sum())
    b, cc = int((e_ref & ~e_gpu).sum()), int((~e_ref & e_gpu).sum())
    lo, hi = _cp(fe_ref, F)
    p = _mcnemar_p(b, cc)
    print(f"\n{name} {msg} {ebn0} dB, {F} frames: FER gpu {fe / F:.2e} oracle {fe_ref / F:.2e} "
          f"CI [{lo:.2e}, {hi:.2e}]; discordant frames {b} (oracle only) / {cc} (GPU only), McNemar p {p:.3f}; "
          f"mean iterations gpu {iters.mean():.3f} oracle {ref.iters.mean():.3f}")
    assert lo <= fe / F <= hi
    assert p >= 0.01
    if msg == "f32":
        from parity_rules import check_full
        q = g.query()
        check_full(f"{name} fp32 {F} frames", bits, iters, ok, ref, llr.astype(np.float64),
                   lambda x: oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], x, 25))
