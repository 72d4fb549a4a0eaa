"""ndgsbp_decode_static -- decoding without allocating device memory (GPU).

Some callers cannot allocate device memory at the moment they decode: a real-time receive loop
must not call cudaMalloc (it can synchronise the device and take unbounded time), and a process
whose device memory is already handed out by another allocator would see the allocation fail.
ndgsbp_decode_static serves them with scratch held in a static device array of the library.

These tests call it through the C ABI, twice in a row on different batches, and compare each
result with ndgsbp_decode (which takes a caller-allocated workspace) on the same frames.  The two
run the same kernels, so the tolerance is the one the parity tests use for identical
arithmetic: equality.  They also check the property the entry point exists for: after the
set-up (the plan and one first call), the device's free memory (cudaMemGetInfo) is the same
before and after the two calls.  The file is collected last so that a failure here does not
hide others.
"""
import ctypes

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
    lib = ctypes.CDLL(ndgsbp.library_path())
    fn = lib.ndgsbp_decode_static
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ndgsbp.Params), ctypes.c_void_p, ctypes.c_int32,
                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    return ndgsbp, torch, fn


def _outputs(torch, F, N, dev):
    W = (N + 31) // 32
    return (torch.full((F, W), -1, dtype=torch.int32, device=dev),
            torch.full((F,), -1, dtype=torch.int32, device=dev),
            torch.full((F,), 7, dtype=torch.uint8, device=dev),
            torch.full((F, N), float("nan"), dtype=torch.float32, device=dev))


def _static(nd, torch, fn, groups, params, llr, out=None):
    dev = llr.device
    hard, iters, ok, post = out if out is not None else _outputs(torch, llr.shape[0], groups.code.N, dev)
    stream = torch.cuda.current_stream().cuda_stream
    st = fn(groups.handle, ctypes.byref(params), ctypes.c_void_p(llr.data_ptr()), nd.F32, llr.shape[0],
            ctypes.c_void_p(hard.data_ptr()), ctypes.c_void_p(iters.data_ptr()), ctypes.c_void_p(ok.data_ptr()),
            ctypes.c_void_p(post.data_ptr()), ctypes.c_void_p(stream))
    return st, (hard, iters, ok, post)


def _workspace(nd, torch, groups, params, llr):
    dev = llr.device
    hard, iters, ok, post = _outputs(torch, llr.shape[0], groups.code.N, dev)
    ws = torch.zeros(groups.workspace_size(params, llr.shape[0]), dtype=torch.uint8, device=dev)
    nd.decode_plain(groups, params, llr, ws, hard, iters, ok, post)
    return hard, iters, ok, post


CASES = [
    # (code, grouping, params): QC kernel with messages in shared memory (scratch = counter only),
    # QC kernel and table-driven kernel with messages in per-CTA slots of the scratch array
    ("qc_n2304_r12", "layers", dict()),
    ("qc_n2304_r12", "layers", dict(variant=4, ctas_per_sm=1)),
    ("gallager36_n1008", "cn", dict(variant=2, ctas_per_sm=2)),
]


@pytest.mark.parametrize("name,kind,pkw", CASES)
def test_static_decode_matches_workspace_decode(env, name, kind, pkw):
    nd, torch, fn = env
    c = I.code_by_name(name)
    code = nd.Code.from_inputs(c)
    if kind == "layers":
        groups = nd.Groups.build(code, c.M // c.Z, 0.5, 2304, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    else:
        groups = nd.Groups.build(code, 4, 0.4, 7)
    params = nd.params_default(max_iter=25, **pkw)
    F = 3000
    dev = torch.device("cuda")
    llrs = [torch.from_numpy(I.channel_llr(c.N, F, ebn0, I.design_rate(c), seed, dtype=np.float32)).to(dev)
            for ebn0, seed in [(1.25, 11), (1.75, 12)]]
    outs = [_outputs(torch, F, c.N, dev) for _ in llrs]
    # set-up: the plan puts the grouping's tables on this device; the first call looks up the
    # static array's address and loads the kernel
    groups.plan(params, F)
    st, _ = _static(nd, torch, fn, groups, params, llrs[0])
    assert st == nd.OK, nd.last_error()
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for llr, out in zip(llrs, outs):
        st, _ = _static(nd, torch, fn, groups, params, llr, out)
        assert st == nd.OK, nd.last_error()
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before, f"device free memory changed by {free_before - free_after} bytes"
    for call, (llr, got) in enumerate(zip(llrs, outs)):
        want = _workspace(nd, torch, groups, params, llr)
        torch.cuda.synchronize()
        for g, w in zip(got, want):
            assert torch.equal(g, w), f"call {call + 1}: output differs from ndgsbp_decode"
        assert int(got[1].min()) >= 1 and int(got[1].max()) <= 25


def test_static_decode_refuses_what_it_cannot_do(env):
    nd, torch, fn = env
    c = I.code_by_name("qc_n2304_r12")
    code = nd.Code.from_inputs(c)
    dev = torch.device("cuda")
    llr = torch.zeros((64, c.N), dtype=torch.float32, device=dev)
    # tables not uploaded to the device yet: refused, nothing allocated
    fresh = nd.Groups.build(code, 12, 0.5, 5, unit=nd.UNIT_LAYER, flags=nd.GROUPS_CYCLIC)
    st, _ = _static(nd, torch, fn, fresh, nd.params_default(), llr)
    assert st == nd.ERR_INVALID and "ndgsbp_decode_plan" in nd.last_error()
    # scratch beyond the static array: messages of every resident CTA in global slots
    big = nd.params_default(variant=nd.VARIANT_QC_GLOBAL)
    plan = fresh.plan(big, 10**6)
    assert plan.workspace_bytes > nd.STATIC_SCRATCH_BYTES
    st, _ = _static(nd, torch, fn, fresh, big, torch.zeros((10**5, c.N), dtype=torch.float32, device=dev))
    assert st == nd.ERR_WORKSPACE and "static array" in nd.last_error()
