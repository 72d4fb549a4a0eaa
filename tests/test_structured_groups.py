"""Structure-aware grouping (NDGSBP_GROUPS_STRUCTURED): the library's groups equal the oracle's
independent construction, keep Step 1's structure (group 1 and the overlaps), and raise the
CoCSG l of Sec. II-A over random Step 1 groups."""
import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I


@pytest.fixture(scope="module")
def nd():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp


@pytest.mark.parametrize("G,r,seed", [(4, 0.4, 7), (12, 0.4, 2024), (12, 0.0, 5), (36, 0.25, 11)])
def test_structured_groups_match_oracle_and_raise_cocsg(nd, oracle_mod, G, r, seed):
    c = I.code_by_name("gallager36_n1008")
    code = nd.Code.from_inputs(c)
    gs = nd.Groups.build(code, G, r, seed, flags=nd.GROUPS_STRUCTURED)
    q = gs.query()
    gp, gc = oracle_mod.groups_structured(c, G, r, seed)
    np.testing.assert_array_equal(q["grp_ptr"], gp)
    np.testing.assert_array_equal(q["cn_idx"], gc)
    # Step 1's structure: group 1 is the random group 1, each overlap is the last o of the previous
    rnd_p, rnd_c = oracle_mod.groups(c.M, G, r, seed)
    np.testing.assert_array_equal(gc[:gp[1]], rnd_c[:rnd_p[1]])
    NG, o, fresh = oracle_mod.group_sizes(c.M, G, r)
    for g in range(1, G):
        cur, prev = gc[gp[g]:gp[g + 1]], gc[gp[g - 1]:gp[g]]
        np.testing.assert_array_equal(cur[:o], prev[len(prev) - o:])
    assert len(set(gc.tolist())) == c.M
    l_s = oracle_mod.cocsg(c, gp, gc)
    l_r = oracle_mod.cocsg(c, rnd_p, rnd_c)
    print(f"\nG={G} r={r}: CoCSG structured {l_s:.1f} vs random {l_r:.1f}")
    assert l_s > l_r
    assert q["cocsg"] == pytest.approx(l_s)


def test_structured_flag_validation(nd):
    c = I.code_by_name("qc_n576_r12")
    code = nd.Code.from_inputs(c)
    for kw in (dict(unit=nd.UNIT_LAYER), dict(flags=nd.GROUPS_STRUCTURED | nd.GROUPS_CYCLIC)):
        kw.setdefault("flags", nd.GROUPS_STRUCTURED)
        with pytest.raises(nd.NdgsbpError) as e:
            nd.Groups.build(code, 12, 0.5, 1, **kw)
        assert e.value.status == nd.ERR_INVALID
