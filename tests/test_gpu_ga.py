"""The FP64 GA recursion on the GPU (ndgsbp_ga_flood) against the oracle's (oracle/ga.py) and
Table I (needs a GB300).  The two sides integrate Eq. (14) by different rules (trapezoidal on
the GPU, Gauss-Hermite in the oracle), so iteration counts are compared away from the threshold,
where a 1e-12 difference in Phi cannot move the step at which mu_c passes the cap."""
import numpy as np
import pytest

from oracle import ga
from paper_1202_1060_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ENSEMBLES = [({3: 1.0}, {6: 1.0}, 0.5, 1.163), ({4: 1.0}, {6: 1.0}, 1 / 3, 1.730)]


@pytest.fixture(scope="module")
def nd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1202_1060_gb300 import ndgsbp
    return ndgsbp


@pytest.mark.parametrize("lam,rho,R,printed", ENSEMBLES)
def test_gpu_ga_thresholds_table1(nd, lam, rho, R, printed):
    t_gpu = nd.ga_flood_threshold(lam, rho, R, phi_kind=nd.GA_PHI_CLOSED, lo_db=0.5, hi_db=3.0, tol_db=1e-4)
    t_or = ga.threshold(lambda e: ga.flood_ga(e, lam, rho, R, kind="approx"), lo=0.5, hi=3.0, tol=1e-4)
    print(f"\nGA threshold (closed-form Phi): GPU {t_gpu:.5f} dB, oracle {t_or:.5f} dB, printed {printed}")
    assert abs(t_gpu - t_or) <= 3e-4
    assert abs(t_gpu - printed) <= 1.2e-3


@pytest.mark.parametrize("kind", ["exact", "approx"])
def test_gpu_ga_matches_oracle_recursion(nd, kind):
    lam, rho, R = {3: 1.0}, {6: 1.0}, 0.5
    pk = nd.GA_PHI_EXACT if kind == "exact" else nd.GA_PHI_CLOSED
    snr = np.array([0.8, 1.0, 1.1, 1.25, 1.4, 1.6, 2.0])
    cv, it, mu = nd.ga_flood(lam, rho, R, snr, phi_kind=pk)
    for k, e in enumerate(snr):
        c, i, m = ga.flood_ga(float(e), lam, rho, R, kind=kind)
        assert cv[k] == c, e
        assert it[k] == i, (e, it[k], i)
        if not c:
            assert mu[k] == pytest.approx(m, rel=1e-9)
    t_gpu = nd.ga_flood_threshold(lam, rho, R, phi_kind=pk, lo_db=0.5, hi_db=3.0, tol_db=2e-4)
    t_or = ga.threshold(lambda e: ga.flood_ga(e, lam, rho, R, kind=kind), lo=0.5, hi=3.0, tol=2e-4)
    assert abs(t_gpu - t_or) <= 5e-4


def test_gpu_ga_irregular_profile(nd):
    """The edge-perspective profile of the n=2304 QC code (VN degrees {2,3,6}, CN degrees {6,7})."""
    prof = I.degree_profile(I.code_by_name("qc_n2304_r12"))
    lam, rho = prof["lambda"], prof["rho"]
    snr = np.array([0.0, 0.5, 1.0, 1.5, 2.0])
    cv, it, mu = nd.ga_flood(lam, rho, 0.5, snr, phi_kind=nd.GA_PHI_EXACT)
    for k, e in enumerate(snr):
        c, i, m = ga.flood_ga(float(e), lam, rho, 0.5)
        assert (cv[k], it[k]) == (c, i), e


# ----------------------------------------------------------------------------------------
# group schedules (GSBP r = 0, NDGSBP r > 0): Eqs. (4)-(17)
# ----------------------------------------------------------------------------------------
GROUP_CASES = [(4, 0.0), (12, 0.0), (4, 0.4), (12, 0.4), (36, 0.4)]


@pytest.mark.parametrize("G,r", GROUP_CASES)
def test_gpu_group_ga_matches_oracle(nd, G, r):
    """Converged flags, iteration counts (away from the threshold, where rounding cannot move the
    step at which mu_c passes the cap) and fixed points of the group recursion equal the oracle's
    (closed-form Phi, the form of Table I)."""
    lam, rho, R = {3: 1.0}, {6: 1.0}, 0.5
    snr = np.array([0.8, 1.0, 1.1, 1.3, 1.6, 2.0])
    cv, it, mu = nd.ga_groups(lam, rho, R, G, r, snr, phi_kind=nd.GA_PHI_CLOSED)
    for k, e in enumerate(snr):
        c, i, m = ga.group_ga(float(e), lam, rho, R, G, r, kind="approx")
        assert cv[k] == c, (G, r, e)
        assert it[k] == i, (G, r, e, it[k], i)
        assert mu[k] == pytest.approx(m, rel=1e-9 if not c else 1e-6)


@pytest.mark.parametrize("G", [12, 36])
def test_gpu_group_ga_irregular_profile(nd, G):
    """The group recursion on the n=2304 QC code's profile (VN degrees {2,3,6}, CN degrees {6,7}),
    r = 0.4: 19 class-b weight terms per group, so G = 12 reads them from the per-point table and
    G = 36 (665 terms) computes them in the loop; both equal the oracle."""
    prof = I.degree_profile(I.code_by_name("qc_n2304_r12"))
    lam, rho = prof["lambda"], prof["rho"]
    snr = np.array([0.3, 0.6, 1.2, 2.0])
    cv, it, mu = nd.ga_groups(lam, rho, 0.5, G, 0.4, snr, phi_kind=nd.GA_PHI_CLOSED)
    for k, e in enumerate(snr):
        c, i, m = ga.group_ga(float(e), lam, rho, 0.5, G, 0.4, kind="approx")
        assert (cv[k], it[k]) == (c, i), (G, e, it[k], i)
        assert mu[k] == pytest.approx(m, rel=1e-9 if not c else 1e-6)


def test_gpu_group_ga_exact_phi(nd):
    """The exact Eq. (14) (trapezoidal on the GPU, Gauss-Hermite in the oracle) on points well
    above and below the threshold, G = 4, r = 0.4."""
    lam, rho, R = {3: 1.0}, {6: 1.0}, 0.5
    snr = np.array([0.9, 1.8])
    cv, it, mu = nd.ga_groups(lam, rho, R, 4, 0.4, snr, phi_kind=nd.GA_PHI_EXACT)
    for k, e in enumerate(snr):
        c, i, m = ga.group_ga(float(e), lam, rho, R, 4, 0.4, kind="exact")
        assert (cv[k], it[k]) == (c, i), e
        if not c:
            assert mu[k] == pytest.approx(m, rel=1e-9)


@pytest.mark.parametrize("lam,rho,R,printed", ENSEMBLES)
def test_gpu_group_thresholds_equal_flooding(nd, lam, rho, R, printed):
    """Table I: BP, GSBP and NDGSBP share the GA threshold (1.163 dB for (3,6), 1.730 dB for
    (4,6)); the GPU's group thresholds agree with its flooding threshold and the printed value."""
    t_flood = nd.ga_flood_threshold(lam, rho, R, phi_kind=nd.GA_PHI_CLOSED, lo_db=0.5, hi_db=3.0, tol_db=1e-3)
    for G, r in ((4, 0.0), (4, 0.4), (12, 0.4)):
        t = nd.ga_groups_threshold(lam, rho, R, G, r, phi_kind=nd.GA_PHI_CLOSED, lo_db=0.5, hi_db=3.0, tol_db=1e-3)
        print(f"\nGA threshold G={G} r={r}: {t:.4f} dB (flooding {t_flood:.4f}, printed {printed})")
        assert abs(t - t_flood) <= 2e-3 and abs(t - printed) <= 3e-3


def test_gpu_group_ga_iteration_ordering(nd):
    """Table I's ordering of the iterations to error-free decoding just above the threshold:
    NDGSBP < GSBP < BP, and fewer with more groups (the counts themselves depend on the stop
    criterion the paper leaves open)."""
    lam, rho, R = {3: 1.0}, {6: 1.0}, 0.5
    e = np.array([1.20])
    _, it_bp, _ = nd.ga_flood(lam, rho, R, e, phi_kind=nd.GA_PHI_CLOSED)
    its = {}
    for G, r in ((4, 0.0), (12, 0.0), (4, 0.4), (12, 0.4)):
        cv, it, _ = nd.ga_groups(lam, rho, R, G, r, e, phi_kind=nd.GA_PHI_CLOSED)
        assert cv[0]
        its[(G, r)] = int(it[0])
    print("\nGA iterations at 1.20 dB: BP", int(it_bp[0]), its)
    assert its[(4, 0.4)] < its[(4, 0.0)] < it_bp[0]
    assert its[(12, 0.4)] < its[(12, 0.0)] < it_bp[0]
    assert its[(12, 0.0)] <= its[(4, 0.0)] and its[(12, 0.4)] <= its[(4, 0.4)]
