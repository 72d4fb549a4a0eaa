"""Groupings cycled by iteration (ndgsbp_groups_build_cycled): grouping k is Step 1 with seed
seed + k, equal to the oracle's independent draw."""
import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I


@pytest.fixture(scope="module")
def nd():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp


@pytest.mark.parametrize("name,unit,G,r,flags", [("gallager36_n1008", "cn", 12, 0.4, 0),
                                                  ("qc_n2304_r12", "layer", 12, 0.5, "cyclic")])
def test_cycled_groupings_match_oracle(nd, oracle_mod, name, unit, G, r, flags):
    c = I.code_by_name(name)
    code = nd.Code.from_inputs(c)
    u = nd.UNIT_LAYER if unit == "layer" else nd.UNIT_CN
    fl = nd.GROUPS_CYCLIC if flags == "cyclic" else 0
    g = nd.Groups.build(code, G, r, 77, unit=u, flags=fl, n_groupings=4)
    gs = g.groupings()
    assert len(gs) == 4
    q = g.query()
    np.testing.assert_array_equal(q["grp_ptr"], gs[0][0])
    for k, (gp, gc) in enumerate(gs):
        rp, rc = oracle_mod.groups(c.M, G, r, 77 + k, unit=c.Z if unit == "layer" else 1, cyclic=fl != 0)
        np.testing.assert_array_equal(gp, rp)
        np.testing.assert_array_equal(gc, rc)
    assert any((gs[0][1] != gs[k][1]).any() for k in range(1, 4))
    with pytest.raises(nd.NdgsbpError):
        nd.Groups.build(code, G, r, 77, unit=u, flags=fl, n_groupings=0)
