"""Reduced-precision message storage (FP16, BF16) against the FP64 oracle (needs a GB300).

The kernels compute Eq. (1) in FP32 and round only the stored CN->VN messages; the posterior
absorbs the rounded values.  In the first flooding iteration every CN reads the exact channel
LLRs, so each message is an FP32-accurate value rounded once: its error is at most half an ulp of
the storage type (2^-11 relative for FP16, 2^-8 for BF16) plus the FP32 tolerance.  Grouped
schedules already feed rounded messages of earlier groups into later ones within the first
iteration, and later iterations compound that; there the per-edge error is stated (printed) and
bounded loosely, and the decisions are held to the error-rate criterion: FER inside the oracle's
95% Clopper-Pearson interval on the same frames.
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


FER_CASES = [("qc_n2304_r12", 1.75, 12000), ("qc_n16200_r23", 1.9, 3000)]


@pytest.mark.parametrize("name,ebn0,F", FER_CASES)
@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_low_precision_fer_inside_oracle_ci(env, oracle_mod, name, ebn0, F, msg):
    """FER of FP32/FP16/BF16 message storage inside the FP64 oracle's 95% interval on the same
    frames (all-zero codeword, cyclic 2-layer NDGSBP, I_max 25)."""
    nd, torch = env
    c = I.code_by_name(name)
    llr = I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed=9000 + int(ebn0 * 100), dtype=np.float32)
    code, g = _layers(nd, c)
    bits, iters, ok, _ = _decode(nd, torch, g, c, llr, msg, max_iter=25)
    q = g.query()
    ref = oracle_mod.ndgsbp_decode(c, q["grp_ptr"], q["cn_idx"], llr.astype(np.float64), 25, want_total=False)
    fe_ref = int(ref.hard.any(axis=1).sum())
    fe = int(bits.any(axis=1).sum())
    lo, hi = _cp(fe_ref, F)
    print(f"\n{name} {msg} {ebn0} dB: FER gpu {fe / F:.2e} oracle {fe_ref / F:.2e} CI [{lo:.2e}, {hi:.2e}], "
          f"mean iterations gpu {iters.mean():.2f} oracle {ref.iters.mean():.2f}")
    assert lo <= fe / F <= hi
