"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage or fact it relies on.  Together they are chosen so that a plausible
mistake in the oracle (a dropped term in Eq. (1) or (2), a wrong sign, reading a message updated
within the same group, a wrong overlap choice in Step 1) fails at least one of them; the
mutation tests at the end plant such mistakes in a copy of the oracle and check that they do.
"""
import json
import os

import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------------------------------
# Printed values (Sec. II-A, Sec. IV)
# ----------------------------------------------------------------------------------------

def test_printed_group_sizes(oracle_mod):
    for case in _load("printed_values.json")["group_sizes"]:
        NG, o, fresh = oracle_mod.group_sizes(case["M"], case["G"], case["r"])
        assert NG == case["N_G"], case["where"]


def test_printed_budget(oracle_mod):
    for case in _load("printed_values.json")["budget"]:
        it = oracle_mod.budget_iters(case["M"], case["G"], case["N_G"], case["r"], case["I_max"])
        assert it == case["iters"], case["where"]


def test_size_relation_counts(oracle_mod):
    """G N_G - (G-1) N_G r = M: the group entries number M plus one overlap per later group."""
    for M in (17, 252, 504, 1000):
        for G in (1, 2, 4, 12):
            for r in (0.0, 0.25, 0.4, 0.5):
                NG, o, fresh = oracle_mod.group_sizes(M, G, r)
                assert fresh.sum() == M
                assert fresh[0] == NG
                gp, gc = oracle_mod.groups(M, G, r, seed=M * 31 + G)
                assert gp[-1] == M + (G - 1) * o
                # N_G is the smallest integer with G N_G - (G-1) N_G r >= M
                assert G * NG - (G - 1) * NG * r >= M - 1e-9
                if NG > 1 and G > 1:
                    assert G * (NG - 1) - (G - 1) * (NG - 1) * r < M


def test_group_size_errors(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.group_sizes(10, 11, 0.2)
    with pytest.raises(ValueError):
        oracle_mod.group_sizes(10, 2, 1.0)
    with pytest.raises(ValueError):
        oracle_mod.group_sizes(10, 2, -0.1)
    with pytest.raises(ValueError):
        oracle_mod.group_sizes(10, 3, 0.5, cyclic=True)   # 3 does not divide 10


# ----------------------------------------------------------------------------------------
# Step 1 (Sec. II-C)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("M,G,r", [(60, 4, 0.4), (504, 4, 0.4), (252, 12, 0.4), (50, 5, 0.0),
                                   (40, 3, 0.5), (40, 3, 0.7), (30, 1, 0.3)])
def test_step1_structure(oracle_mod, M, G, r):
    NG, o, fresh = oracle_mod.group_sizes(M, G, r)
    for seed in range(5):
        gp, gc = oracle_mod.groups(M, G, r, seed=seed)
        groups = [list(gc[gp[g]:gp[g + 1]]) for g in range(G)]
        assert sorted(set(gc.tolist())) == list(range(M))          # every CN is grouped
        assert len(groups[0]) == NG
        seen = set(groups[0])
        for g in range(1, G):
            assert len(set(groups[g])) == len(groups[g])
            ov, new = groups[g][:o], groups[g][o:]
            assert ov == groups[g - 1][len(groups[g - 1]) - o:]    # r N_G CNs from G_{g-1}
            assert len(new) == fresh[g] and not (set(new) & seen)   # the rest are unused CNs
            if g >= 2 and o <= fresh[g - 1]:
                assert not (set(ov) & set(groups[g - 2]))           # drawn from G_{g-1}\G_{g-2}
            seen |= set(new)
        if r == 0.0:
            assert len(gc) == M                                     # r = 0: a partition (GSBP)


def test_step1_random_choice_uniform(oracle_mod):
    """'randomly' in Step 1: every CN is equally likely to open G_1, and every CN of G_1 equally
    likely to be carried into G_2 (chi-square over 3000 seeds)."""
    from scipy import stats
    M, G, r = 20, 3, 0.4
    NG, o, fresh = oracle_mod.group_sizes(M, G, r)
    in_g1 = np.zeros(M)
    carried = np.zeros(M)
    trials = 3000
    for seed in range(trials):
        gp, gc = oracle_mod.groups(M, G, r, seed=seed + 1000)
        g1 = gc[gp[0]:gp[1]]
        in_g1[g1] += 1
        carried[gc[gp[1]:gp[1] + o]] += 1
    assert stats.chisquare(in_g1).pvalue > 1e-4
    assert stats.chisquare(carried).pvalue > 1e-4
    assert np.isclose(carried.sum() / in_g1.sum(), o / NG)


def test_step1_seeded(oracle_mod):
    a = oracle_mod.groups(504, 4, 0.4, seed=11)
    b = oracle_mod.groups(504, 4, 0.4, seed=11)
    c = oracle_mod.groups(504, 4, 0.4, seed=12)
    assert (a[1] == b[1]).all() and not (a[1] == c[1]).all()


def test_step1_cyclic_layers(oracle_mod):
    """Cyclic windows of 2 layers at overlap 1 over 12 layers: each layer is in two groups,
    consecutive groups (and the last and first) share one layer."""
    Z = 4
    gp, gc = oracle_mod.groups(12 * Z, 12, 0.5, seed=3, unit=Z, cyclic=True)
    layers = [sorted(set(int(c) // Z for c in gc[gp[g]:gp[g + 1]])) for g in range(12)]
    assert all(len(l) == 2 for l in layers)
    assert np.bincount([x for l in layers for x in l], minlength=12).tolist() == [2] * 12
    for g in range(12):
        assert len(set(layers[g]) & set(layers[(g + 1) % 12])) == 1
    # units expand to whole layers
    for g in range(12):
        cns = gc[gp[g]:gp[g + 1]]
        assert len(cns) == 2 * Z


def test_cocsg_bound(oracle_mod):
    """CoCSG of Sec. II-B: l >= (M/N) N_G r as printed; for a regular code each of the o d_c
    edges of the overlap CNs lands on a VN of degree d_v, so l >= o N / M as well."""
    code = I.code_by_name("gallager36_n1008")
    for r in (0.2, 0.4):
        NG, o, _ = oracle_mod.group_sizes(code.M, 4, r)
        gp, gc = oracle_mod.groups(code.M, 4, r, seed=5)
        l = oracle_mod.cocsg(code, gp, gc)
        assert l >= code.M / code.N * NG * r
        assert l >= o * code.N / code.M


# ----------------------------------------------------------------------------------------
# Reductions (Sec. II-A definitions of BP, GSBP and the layered limit)
# ----------------------------------------------------------------------------------------

def _llr(code, frames, ebn0, seed):
    return I.channel_llr(code.N, frames, ebn0, I.design_rate(code), seed)


def test_one_group_is_flooding(oracle_mod):
    code = I.code_by_name("gallager36_n1008")
    llr = _llr(code, 24, 1.5, seed=21)
    gp, gc = oracle_mod.groups(code.M, 1, 0.0, seed=0)
    a = oracle_mod.ndgsbp_decode(code, gp, gc, llr, 30, want_c2v=True)
    b = oracle_mod.flood_decode(code, llr, 30, want_c2v=True)
    assert (a.iters == b.iters).all() and (a.hard == b.hard).all() and (a.synd_ok == b.synd_ok).all()
    assert np.abs(a.total - b.total).max() < 1e-8
    assert np.abs(a.c2v - b.c2v).max() < 1e-8


def test_one_cn_per_group_is_layered(oracle_mod):
    code = I.code_by_name("qc_n576_r12")
    llr = _llr(code, 16, 2.0, seed=22)
    gp, gc = oracle_mod.groups(code.M, code.M, 0.0, seed=0, natural=True)
    assert (gc == np.arange(code.M)).all()
    a = oracle_mod.ndgsbp_decode(code, gp, gc, llr, 20, want_c2v=True)
    b = oracle_mod.layered_decode(code, llr, 20, want_c2v=True)
    assert (a.iters == b.iters).all() and (a.hard == b.hard).all()
    assert np.abs(a.total - b.total).max() < 1e-8
    assert np.abs(a.c2v - b.c2v).max() < 1e-8


@pytest.mark.parametrize("G,r,cyc,layers", [(4, 0.0, False, False), (4, 0.4, False, False),
                                            (12, 0.4, False, False), (12, 0.5, True, True)])
def test_explicit_messages_equal_posterior_form(oracle_mod, G, r, cyc, layers):
    """Eq. (2) written with explicit VN->CN messages and the posterior form give the same
    decoder for any groups, disjoint (GSBP) or overlapping (NDGSBP)."""
    code = I.code_by_name("qc_n576_r12") if layers else I.code_by_name("gallager36_n1008")
    unit = code.Z if layers else 1
    llr = _llr(code, 16, 1.5, seed=23)
    gp, gc = oracle_mod.groups(code.M, G, r, seed=9, unit=unit, cyclic=cyc)
    a = oracle_mod.ndgsbp_decode(code, gp, gc, llr, 25, want_c2v=True)
    b = oracle_mod.group_posterior_decode(code, gp, gc, llr, 25, want_c2v=True)
    assert (a.iters == b.iters).all() and (a.hard == b.hard).all()
    assert np.abs(a.total - b.total).max() < 1e-8
    assert np.abs(a.c2v - b.c2v).max() < 1e-8


def test_regrouping_with_identical_groupings(oracle_mod):
    code = I.code_by_name("gallager36_n1008")
    llr = _llr(code, 8, 1.5, seed=24)
    gp, gc = oracle_mod.groups(code.M, 4, 0.4, seed=2)
    a = oracle_mod.ndgsbp_decode(code, gp, gc, llr, 20)
    b = oracle_mod.ndgsbp_decode(code, np.stack([gp, gp, gp]), gc, llr, 20)
    assert (a.total == b.total).all()


# ----------------------------------------------------------------------------------------
# Exactness on cycle-free graphs (brute-force bitwise MAP)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_tree_posteriors_equal_map(oracle_mod, seed):
    code = I.tree_code(14, seed=seed)
    rng = np.random.default_rng(seed)
    llr = rng.normal(0.8, 1.2, size=(6, code.N))
    ref = oracle_mod.brute_force_map(code, llr)
    kw = dict(llr_max=0.0, early_stop=False)
    res = [oracle_mod.flood_decode(code, llr, 40, **kw),
           oracle_mod.layered_decode(code, llr, 40, **kw)]
    for G, r in ((1, 0.0), (2, 0.0), (3, 0.0), (3, 0.4), (4, 0.5)):
        if G > code.M:
            continue
        gp, gc = oracle_mod.groups(code.M, G, r, seed=seed)
        res.append(oracle_mod.ndgsbp_decode(code, gp, gc, llr, 40, **kw))
    for r_ in res:
        assert np.abs(r_.total - ref).max() < 1e-9


# ----------------------------------------------------------------------------------------
# Vertical (VN-group) shuffled BP, the other serial schedule of Sec. I
# ----------------------------------------------------------------------------------------

def test_vertical_one_group_is_flooding(oracle_mod):
    """All VNs in one group: every CN message of the iteration comes from the previous
    iteration's VN messages, i.e. the textbook flooding decoder."""
    code = I.code_by_name("gallager36_n1008")
    llr = _llr(code, 16, 1.5, seed=41)
    a = oracle_mod.vertical_decode(code, [0, code.N], np.arange(code.N), llr, 25, want_c2v=True)
    b = oracle_mod.flood_decode(code, llr, 25, want_c2v=True)
    assert (a.iters == b.iters).all() and (a.hard == b.hard).all()
    assert np.abs(a.total - b.total).max() < 1e-8 and np.abs(a.c2v - b.c2v).max() < 1e-8


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_vertical_tree_posteriors_equal_map(oracle_mod, seed):
    """On cycle-free graphs every VN-group schedule converges to the bitwise-MAP LLRs."""
    code = I.tree_code(14, seed=seed)
    rng = np.random.default_rng(100 + seed)
    llr = rng.normal(0.8, 1.2, size=(6, code.N))
    ref = oracle_mod.brute_force_map(code, llr)
    for G in (1, 2, 5, code.N):
        gp, gv = oracle_mod.groups(code.N, G, 0.0, seed=seed)
        r = oracle_mod.vertical_decode(code, gp, gv, llr, 60, llr_max=0.0, early_stop=False)
        assert np.abs(r.total - ref).max() < 1e-9, G


def _vertical_expected_deps(code, groups):
    """Channel values each CN->VN message of iteration 1 depends on, from the schedule's
    definition alone: the message into VN n from CN m, formed in n's sub-iteration, reads the
    other VNs n' of m; n' contributes {n'} if its group comes at or after n's (not yet updated),
    else {n'} plus everything its other CNs sent it in its own sub-iteration."""
    gof = {}
    for g, vs in enumerate(groups):
        for v in vs:
            gof[v] = g
    rows = [list(code.col_idx[code.row_ptr[m]:code.row_ptr[m + 1]]) for m in range(code.M)]
    cols = [[m for m in range(code.M) if n in rows[m]] for n in range(code.N)]
    deps = {}
    for g, vs in enumerate(groups):
        for n in vs:
            for m in cols[n]:
                d = set()
                for n2 in rows[m]:
                    if n2 == n:
                        continue
                    d.add(n2)
                    if gof[n2] < g:
                        for m2 in cols[n2]:
                            if m2 != m:
                                d |= deps[(m2, n2)]
                deps[(m, n)] = d
    return deps


@pytest.mark.parametrize("seed", [3, 8])
def test_vertical_influence_sets(oracle_mod, seed):
    """The order of the VN groups, pinned by which channel values reach each CN->VN message in
    the first iteration: perturbing L_j moves message (m, n) exactly when the schedule's
    definition says it reads L_j (a VN of an earlier group carries what it received; a VN of the
    same or a later group only its channel value)."""
    rng = np.random.default_rng(seed)
    N, M = 12, 6
    # a random sparse code: every VN on 1-2 CNs, every CN on >= 2 VNs
    H = np.zeros((M, N), np.uint8)
    for n in range(N):
        for m in rng.choice(M, size=int(rng.integers(1, 3)), replace=False):
            H[m, n] = 1
    for m in range(M):
        while H[m].sum() < 2:
            H[m, int(rng.integers(0, N))] = 1
    code = I.code_from_rows([list(np.nonzero(H[m])[0]) for m in range(M)], N, name=f"vsbp_s{seed}")
    perm = rng.permutation(N)
    groups = [[int(v) for v in perm[i::3]] for i in range(3)]
    gp = np.cumsum([0] + [len(g) for g in groups])
    gv = np.concatenate([np.array(g) for g in groups])
    llr = rng.normal(1.0, 1.0, size=(1, N))
    kw = dict(llr_max=0.0, early_stop=False, want_c2v=True)
    base = oracle_mod.vertical_decode(code, gp, gv, llr, 1, **kw).c2v[0]
    deps = _vertical_expected_deps(code, groups)
    for j in range(N):
        pert = llr.copy()
        pert[0, j] += 1e-3
        moved = np.abs(oracle_mod.vertical_decode(code, gp, gv, pert, 1, **kw).c2v[0] - base) > 1e-12
        for m in range(code.M):
            for e in range(code.row_ptr[m], code.row_ptr[m + 1]):
                n = int(code.col_idx[e])
                assert moved[e] == (j in deps[(m, n)]), (j, m, n)


# ----------------------------------------------------------------------------------------
# Fig. 1 message sets (Sec. II-A)
# ----------------------------------------------------------------------------------------

def _influence(oracle_mod, code, groups_1based, after, vn0):
    """Channel values m_j that reached VN vn0's total LLR after `after` sub-iterations, found by
    perturbing each L_j and watching the oracle's posterior (no clipping, generic LLRs)."""
    gp = [0]
    gc = []
    for g in groups_1based:
        gc += [c - 1 for c in g]
        gp.append(len(gc))
    gp = np.asarray(gp, np.int32)
    gc = np.asarray(gc, np.int32)
    rng = np.random.default_rng(7)
    base = rng.uniform(0.6, 1.4, size=code.N) * rng.choice([-1, 1], size=code.N)
    frames = np.tile(base, (code.N + 1, 1))
    for j in range(code.N):
        frames[j + 1, j] += 0.05
    res = oracle_mod.ndgsbp_decode(code, gp, gc, frames, 10, llr_max=0.0, early_stop=False,
                                   stop_after_subiters=after)
    d = np.abs(res.total[1:, vn0] - res.total[0, vn0])
    return sorted(j + 1 for j in range(code.N) if j != vn0 and d[j] > 1e-12)


@pytest.mark.parametrize("x", [1, 3, 5, 7])
def test_fig1_message_sets(oracle_mod, x):
    code = I.fig1_code(x)
    for case in _load("fig1_influence.json")["cases"]:
        got = _influence(oracle_mod, code, case["groups"], case["after_subiters"], case["vn"] - 1)
        assert got == case["receives"], (case, got)


# ----------------------------------------------------------------------------------------
# Symmetry, ties, stopping (Sec. II-C Step 4, Sec. III all-zero assumption)
# ----------------------------------------------------------------------------------------

def test_codeword_symmetry(oracle_mod):
    """decode(L * (1 - 2c)) = decode(L) xor c for any codeword c, exactly."""
    code = I.code_by_name("gallager36_n1008")
    cw = I.random_codeword(code, seed=5)
    assert cw.any()
    H = code.dense().astype(np.int64)
    assert not ((H @ cw) % 2).any()
    llr = _llr(code, 12, 1.5, seed=25)
    gp, gc = oracle_mod.groups(code.M, 4, 0.4, seed=3)
    a = oracle_mod.ndgsbp_decode(code, gp, gc, llr, 30)
    b = oracle_mod.ndgsbp_decode(code, gp, gc, llr * (1.0 - 2.0 * cw), 30)
    assert (a.iters == b.iters).all() and (a.synd_ok == b.synd_ok).all()
    assert ((a.hard ^ cw) == b.hard).all()
    assert (a.total * (1.0 - 2.0 * cw) == b.total).all()


def test_zero_llr_decides_zero(oracle_mod):
    """Step 4 a): d_n = 0 when the total LLR is exactly 0; the all-zero word passes at l = 1."""
    code = I.code_by_name("qc_n576_r12")
    gp, gc = oracle_mod.groups(code.M, 4, 0.4, seed=1)
    r = oracle_mod.ndgsbp_decode(code, gp, gc, np.zeros((2, code.N)), 10)
    assert not r.hard.any() and (r.iters == 1).all() and r.synd_ok.all()


def test_stop_rule(oracle_mod):
    code = I.code_by_name("gallager36_n1008")
    llr = _llr(code, 40, 1.25, seed=26)
    gp, gc = oracle_mod.groups(code.M, 4, 0.4, seed=3)
    a = oracle_mod.ndgsbp_decode(code, gp, gc, llr, 15)
    assert a.iters.min() >= 1 and a.iters.max() <= 15
    assert (a.synd_ok[a.iters < 15] == 1).all()
    b = oracle_mod.ndgsbp_decode(code, gp, gc, llr, 15, early_stop=False)
    assert (b.iters == 15).all()
    # the syndrome flag agrees with the reported hard decisions
    H = code.dense().astype(np.int64)
    ok = ~((b.hard.astype(np.int64) @ H.T) % 2).any(axis=1)
    assert (ok == b.synd_ok.astype(bool)).all()


# ----------------------------------------------------------------------------------------
# Channel (Sec. II-C) and the Philox generator
# ----------------------------------------------------------------------------------------

def test_awgn_llr_statistics(oracle_mod):
    from scipy import stats
    N, F, ebn0, R = 1000, 400, 1.5, 0.5
    s2 = I.sigma2_from_ebn0(ebn0, R)
    L = oracle_mod.awgn_llr(N, F, ebn0, R, seed=99)
    # L = 2 (1 + sigma z) / sigma^2: mean 2/sigma^2, variance 4/sigma^2
    assert abs(L.mean() - 2 / s2) < 4 * np.sqrt(4 / s2 / L.size)
    assert abs(L.var() / (4 / s2) - 1) < 0.01
    z = (L * s2 / 2 - 1) / np.sqrt(s2)
    assert stats.kstest(z.ravel()[:200000], "norm").pvalue > 1e-4
    # neighbours within a Philox block and across frames are uncorrelated
    assert abs(np.corrcoef(z[:, 0::4].ravel(), z[:, 1::4].ravel())[0, 1]) < 0.01
    assert abs(np.corrcoef(z[:-1].ravel(), z[1:].ravel())[0, 1]) < 0.01
    # a 1 bit is sent as -1
    cw = np.zeros(N, np.uint8)
    cw[::3] = 1
    L1 = oracle_mod.awgn_llr(N, F, ebn0, R, seed=99, codeword=cw)
    assert np.allclose(L1[:, cw == 0], L[:, cw == 0])
    assert abs(L1[:, cw == 1].mean() + 2 / s2) < 0.05 * 2 / s2


def test_philox_matches_curand_host_generator(oracle_mod):
    """The oracle's Philox4x32-10 (Salmon et al., SC'11) equals cuRAND's host implementation of
    the same generator, block for block, over keys and counters that exercise every key bit and
    counter words 0-2 (see tests/curand_host.py).  A wrong multiplier, Weyl constant, round count
    or word order fails here."""
    import curand_host as CH
    lib = CH.library()
    if lib is None:
        pytest.skip("cuRAND is not installed")
    for seed, j0 in CH.CASES:
        got = CH.blocks(lib, seed, j0, 8)
        for i in range(8):
            want = oracle_mod.philox4x32_10(CH.counter_of(j0 + i), CH.key_of(seed))
            assert (want == got[i]).all(), (hex(seed), j0 + i, want, got[i])
    # counter 0 under key 0: the generator's very first block
    assert [hex(x) for x in oracle_mod.philox4x32_10([0, 0, 0, 0], [0, 0])] == \
        [hex(x) for x in CH.blocks(lib, 0, 0, 1)[0]]


def test_philox_properties(oracle_mod):
    key = [0x1234, 0x5678]
    outs = np.array([oracle_mod.philox4x32_10([i, 0, 0, 0], key) for i in range(4096)])
    bits = np.unpackbits(outs.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005
    assert len(set(map(tuple, outs.tolist()))) == 4096
    # avalanche: one flipped counter bit changes about half of the 128 output bits
    a = oracle_mod.philox4x32_10([7, 8, 9, 10], key)
    flips = []
    for w in range(4):
        for b in range(32):
            ctr = [7, 8, 9, 10]
            ctr[w] ^= 1 << b
            o = oracle_mod.philox4x32_10(ctr, key)
            flips.append(np.unpackbits((a ^ o).view(np.uint8)).sum())
    assert 56 < np.mean(flips) < 72 and min(flips) > 30
    assert not (oracle_mod.philox4x32_10([1, 2, 3, 4], [0, 0]) ==
                oracle_mod.philox4x32_10([1, 2, 3, 4], [0, 1])).all()


# ----------------------------------------------------------------------------------------
# Planted mistakes: each mutant of the C oracle must fail at least one pin above
# ----------------------------------------------------------------------------------------

MUTANTS = {
    # Eq. (1): include the edge itself in the product
    "cn_self_included": ("            if (j != k) prod *= th[j];", "            prod *= th[j];"),
    # Eq. (1): drop the factor 2 in front of atanh
    "cn_missing_factor2": ("c2v[b + k] = clip(2.0 * atanh(prod), c->llr_max);",
                           "c2v[b + k] = clip(atanh(prod), c->llr_max);"),
    # Eq. (2): drop the channel value L_n
    "vn_missing_channel": ("                    double s = L[n];\n                    for (int j = c->col_ptr[n]",
                           "                    double s = 0.0;\n                    for (int j = c->col_ptr[n]"),
    # Step 2: VN update only for the first CN of the group (a dropped term in the union)
    "vn_union_truncated": ("                    if (!mark[n]) { mark[n] = 1; touched[nt++] = n; }",
                           "                    if (!mark[n] && i == gp[g]) { mark[n] = 1; touched[nt++] = n; }"),
    # Step 1: take the overlap from the front of the previous group instead of its new part
    "overlap_from_front": ("for (int j = prev_len - o; j < prev_len; ++j) units[w++] = units[prev_begin + j];",
                           "for (int j = 0; j < o; ++j) units[w++] = units[prev_begin + j];"),
    # channel generator: a wrong Weyl increment, and counter words 1 and 3 swapped in a round
    "philox_weyl": ("W1 = 0xBB67AE85u;", "W1 = 0xBB67AE86u;"),
    "philox_word_swap": ("uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;", "uint32_t n0 = (uint32_t)(p1 >> 32) ^ c3 ^ k0;"),
    # vertical schedule: a VN's own edge included in its outgoing sum (Eq. (2))
    "vertical_own_edge": ("                        if (a2 != a) s += c2v[c->col_edge[a2]];",
                          "                        s += c2v[c->col_edge[a2]];"),
}


def _pins_pass(oracle_mod):
    """Run a compact set of the pins above; return False at the first failure."""
    try:
        test_tree_posteriors_equal_map(oracle_mod, 1)
        for x in (1, 7):
            test_fig1_message_sets(oracle_mod, x)
        test_step1_structure(oracle_mod, 60, 4, 0.4)
        test_one_group_is_flooding(oracle_mod)
        test_philox_matches_curand_host_generator(oracle_mod)
        test_vertical_one_group_is_flooding(oracle_mod)
        test_vertical_influence_sets(oracle_mod, 3)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(oracle_mod, tmp_path, name):
    old, new = MUTANTS[name]
    src = oracle_mod.source_text()
    assert src.count(old) == 1, name
    path = oracle_mod.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    with oracle_mod.swapped_library(path):
        assert not _pins_pass(oracle_mod), f"mutant {name} passed every pin"
    assert _pins_pass(oracle_mod)
