"""C-ABI library on the CPU: it loads, exports what include/ndgsbp.h declares, and its host-only
calls (code handles, group sizes, Step 1 grouping, layout statistics) agree with the oracle.
No compute call is made here (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nd():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(ndgsbp_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol(nd):
    declared = _declared_functions()
    assert len(declared) >= 15
    lib = ctypes.CDLL(nd.library_path())
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared call
    assert declared <= set(nd.DECLARED_SYMBOLS), declared - set(nd.DECLARED_SYMBOLS)
    assert nd.version().startswith("ndgsbp")


def test_code_create_validation(nd):
    c = I.code_by_name("qc_n576_r12")
    code = nd.Code.from_inputs(c)
    info = code.info()
    assert info["M"] == c.M and info["N"] == c.N and info["E"] == c.E and info["lift_Z"] == c.Z
    assert info["max_row_degree"] == c.row_degrees().max()
    assert info["max_col_degree"] == c.col_degrees().max()
    with pytest.raises(nd.NdgsbpError) as e:
        nd.Code([0, 2], [1, 1], 1, 4)             # repeated column
    assert e.value.status == nd.ERR_INVALID and "repeated" in str(e.value)
    with pytest.raises(nd.NdgsbpError):
        nd.Code([0, 2], [1, 7], 1, 4)             # column out of range
    with pytest.raises(nd.NdgsbpError):
        nd.Code([0, 2, 1], [0, 1], 2, 4)          # row_ptr decreasing
    with pytest.raises(nd.NdgsbpError):
        nd.Code(c.row_ptr, c.col_idx, c.M, c.N, 5)  # M not a multiple of Z


def test_group_sizes_match_oracle(nd, oracle_mod):
    for M in (4, 12, 252, 504, 1152):
        for G in (1, 2, 3, 4, 12):
            if G > M:
                continue
            for r in (0.0, 0.2, 0.4, 0.5, 0.7):
                try:
                    want = oracle_mod.group_sizes(M, G, r)
                except ValueError:
                    with pytest.raises(nd.NdgsbpError):
                        nd.group_sizes(M, G, r)
                    continue
                assert nd.group_sizes(M, G, r) == (want[0], want[1])
    assert nd.group_sizes(252, 12, 0.4) == (34, 14)
    with pytest.raises(nd.NdgsbpError):
        nd.group_sizes(10, 2, 1.0)


CASES = [
    ("gallager36_n1008", 4, 0.4, 0, 0), ("gallager36_n1008", 1, 0.0, 0, 0),
    ("gallager36_n1008", 12, 0.4, 0, 0), ("gallager36_n1008", 4, 0.0, 0, 0),
    ("gallager36_n1008", 5, 0.7, 0, 0), ("qc_n2304_r12", 12, 0.5, 1, 1),
    ("qc_n2304_r12", 11, 0.5, 1, 0), ("qc_n2304_r12", 6, 0.0, 1, 0),
    ("qc_n576_r12", 12, 0.5, 1, 3), ("qc_n16200_r23", 15, 0.5, 1, 1),
]


@pytest.mark.parametrize("name,G,r,layer,flags", CASES)
def test_groups_build_matches_oracle(nd, oracle_mod, name, G, r, layer, flags):
    c = I.code_by_name(name)
    code = nd.Code.from_inputs(c)
    unit = c.Z if layer else 1
    for seed in (0, 1, 12345, 2**63 + 7):
        g = nd.Groups.build(code, G, r, seed, unit=nd.UNIT_LAYER if layer else nd.UNIT_CN, flags=flags)
        q = g.query()
        gp, gc = oracle_mod.groups(c.M, G, r, seed, unit=unit, cyclic=bool(flags & 1),
                                   natural=bool(flags & 2))
        assert (q["grp_ptr"] == gp).all() and (q["cn_idx"] == gc).all()
        assert q["cn_updates_per_iter"] == len(gc)
        deg = c.row_degrees()
        assert q["edge_updates_per_iter"] == int(deg[gc].sum())
        assert abs(q["cocsg"] - oracle_mod.cocsg(c, gp, gc)) < 1e-12


def test_groups_from_lists_validation(nd):
    c = I.fig1_code(5)
    code = nd.Code.from_inputs(c)
    g = nd.Groups.from_lists(code, [0, 2, 4, 6], [0, 1, 1, 2, 2, 3])
    q = g.query()
    assert q["G"] == 3 and list(q["cn_idx"]) == [0, 1, 1, 2, 2, 3]
    with pytest.raises(nd.NdgsbpError):
        nd.Groups.from_lists(code, [0, 2], [0, 0])        # CN twice in a group
    with pytest.raises(nd.NdgsbpError):
        nd.Groups.from_lists(code, [0, 1], [9])           # CN out of range
    with pytest.raises(nd.NdgsbpError):
        nd.Groups.build(code, 2, 0.2, 0, unit=nd.UNIT_LAYER)   # no lift size


def test_params_default(nd):
    p = nd.params_default()
    assert p.max_iter == 50 and p.early_stop == 1 and abs(p.llr_max - 20.0) < 1e-6
    assert p.msg_dtype == nd.F32 and p.schedule == nd.SCHEDULE_GROUPS


def test_bit_packing_roundtrip(nd):
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2, size=(5, 77)).astype(np.uint8)
    assert (nd.unpack_bits(nd.pack_bits(bits), 77) == bits).all()


@pytest.mark.parametrize("name,G", [("gallager36_n1008", 1), ("gallager36_n1008", 7), ("qc_n2304_r12", 5),
                                    ("qc_n576_r12", 576)])
def test_vgroups_build_matches_oracle(nd, oracle_mod, name, G):
    """VN groups of the vertical schedule: Step 1's draw over the N VNs with r = 0 (the oracle's
    own grouping over N units), a partition of the VNs."""
    c = I.code_by_name(name)
    code = nd.Code.from_inputs(c)
    for seed, natural in ((0, False), (99, False), (2**63 + 7, False), (5, True)):
        v = nd.VGroups.build(code, G, seed, flags=nd.GROUPS_NATURAL if natural else 0)
        q = v.query()
        gp, gv = oracle_mod.groups(c.N, G, 0.0, seed, unit=1, natural=natural)
        assert q["G"] == G and (q["grp_ptr"] == gp).all() and (q["grp_vn"] == gv).all()
        assert sorted(q["grp_vn"].tolist()) == list(range(c.N))
        col = c.col_degrees()
        assert q["max_group_edges"] == max(int(col[gv[gp[g]:gp[g + 1]]].sum()) for g in range(G))


def test_vgroups_validation(nd):
    c = I.fig1_code(5)
    code = nd.Code.from_inputs(c)
    N = c.N
    v = nd.VGroups.from_lists(code, [0, 2, N], list(range(N))[::-1])
    assert v.query()["G"] == 2
    for gp, gv in (([0, N], [0] * N),                        # repeated VN
                   ([0, 0, N], list(range(N))),               # empty group
                   ([0, N - 1], list(range(N - 1))),          # VN missing
                   ([0, N], [N] + list(range(1, N)))):        # out of range
        with pytest.raises(nd.NdgsbpError) as e:
            nd.VGroups.from_lists(code, gp, gv + [0] * (N - len(gv)))
        assert e.value.status == nd.ERR_INVALID
    with pytest.raises(nd.NdgsbpError):
        nd.VGroups.build(code, N + 1, 0)
    with pytest.raises(nd.NdgsbpError):
        nd.VGroups.build(code, 2, 0, flags=nd.GROUPS_CYCLIC)
