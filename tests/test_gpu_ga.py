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
