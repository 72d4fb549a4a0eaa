"""Gaussian-approximation (GA) convergence analysis of Sec. III, in FP64 -- test infrastructure.

This module is part of the oracle: only tests/, __graft_entry__.smoke() and bench.py's CPU legs
use it.  It shares no code with the CUDA library.

Sec. III models every message as a consistent Gaussian N(mu, 2 mu) and tracks only its mean
(all-zero codeword, BPSK 0 -> +1, mu0 = E{L_n} = 2 / sigma^2):

* ``phi(mu)`` is Eq. (14), Phi(mu) = 1 - E[tanh(T/2)] with T ~ N(mu, 2 mu).  It is evaluated
  as E[2 / (1 + e^T)] -- the same quantity, since 1 - tanh(t/2) = 2 / (1 + e^t), without the
  cancellation of 1 - tanh near 1 -- by 320-node Gauss-Hermite quadrature (T = mu + 2 sqrt(mu) x;
  within 1e-12 of adaptive quadrature up to mu = 10).
  Phi(0) = 1 and Phi decreases to 0.
* ``phi_approx`` is the closed-form approximation of Phi used by the GA analysis the paper
  builds on (its reference [Chung'01]): exp(-0.4527 mu^0.86 + 0.0218) for mu < 10 and
  sqrt(pi / mu) e^(-mu/4) (1 - 10 / (7 mu)) above.  Table I's thresholds are those of this form
  (1.162 and 1.730 dB); the exact Eq. (14) gives 1.191 dB for the (3,6) ensemble.
* ``phi_inv`` inverts either form on [0, inf) by bisection.
* ``cn_mean`` is Eqs. (15)-(16): the mean of a CN's output from the VN means mu_v,i and the
  edge-perspective degree fractions lambda_i, rho_j (Sec. II-B).
* ``flood_ga`` is the standard BP recursion: every VN sums the channel mean and the other
  i - 1 CN means of the previous iteration (Eq. (4) with all other CNs in class a).
* ``group_ga`` is Eqs. (4)-(17) for G groups with overlap ratio r (r = 0: GSBP), in the reading
  stated at the function.
* ``threshold`` is the smallest Eb/N0 at which the recursion drives mu_c to infinity (error-free
  decoding, the end of Sec. III), found by bisection.

Table I of the paper prints the GA thresholds 1.163 dB ((3,6), R = 1/2) and 1.730 dB ((4,6),
R = 1/3) and states that BP, GSBP and NDGSBP share them; the iteration counts it prints depend on
an unstated "error-free" criterion and are not reproduced (only their ordering is checked).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.hermite import hermgauss
from scipy.special import expit

_GH_X, _GH_W = hermgauss(320)
_GH_W = _GH_W / math.sqrt(math.pi)

MU_CAP = 60.0          # a CN mean above this keeps growing: error-free (Phi(60) ~ 3e-7)


def phi(mu):
    """Eq. (14) for scalar or array mu >= 0."""
    mu = np.asarray(mu, dtype=np.float64)
    out = np.ones_like(mu)
    pos = mu > 0
    m = mu[pos][..., None]
    t = m + 2.0 * np.sqrt(m) * _GH_X
    out[pos] = (2.0 * expit(-t)) @ _GH_W
    return out if out.ndim else float(out)


def phi_approx(mu: float) -> float:
    """The closed-form approximation of Eq. (14) of the cited GA analysis (module docstring)."""
    if mu <= 0.0:
        return 1.0
    if mu < 10.0:
        return math.exp(-0.4527 * mu ** 0.86 + 0.0218)
    return math.sqrt(math.pi / mu) * math.exp(-mu / 4.0) * (1.0 - 10.0 / (7.0 * mu))


PHI = {"exact": lambda m: float(phi(m)), "approx": phi_approx}


def phi_inv(p: float, kind: str = "exact") -> float:
    """The mu >= 0 with Phi(mu) = p (p in (0, 1]), by bisection; Phi decreases (the closed form
    starts at e^0.0218 > 1, so p near 1 maps near 0)."""
    f = PHI[kind]
    if p >= 1.0 and kind == "exact":
        return 0.0
    lo, hi = 0.0, 200.0
    if f(hi) >= p:
        return hi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > p:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-13 * max(1.0, hi):
            break
    return 0.5 * (lo + hi)


def cn_mean(mu_v: dict, lam: dict, rho: dict, kind: str = "exact") -> float:
    """Eqs. (15)-(16): mu_c = sum_j rho_j Phi^-1(1 - (1 - sum_i lambda_i Phi(mu_v,i))^(j-1))."""
    f = PHI[kind]
    s = sum(lam[i] * f(mu_v[i]) for i in lam)
    return sum(rho[j] * phi_inv(1.0 - (1.0 - s) ** (j - 1), kind) for j in rho)


def sigma2(ebn0_db: float, rate: float) -> float:
    """sigma^2 = 1 / (2 R 10^(Eb/N0 / 10)) (BPSK, unit symbol energy)."""
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def flood_ga(ebn0_db: float, lam: dict, rho: dict, rate: float, max_iter: int = 20000, kind: str = "exact"):
    """Standard BP recursion.  Returns (converged, iterations, final mu_c)."""
    mu0 = 2.0 / sigma2(ebn0_db, rate)
    mu_c = 0.0
    for it in range(1, max_iter + 1):
        mu_v = {i: mu0 + (i - 1) * mu_c for i in lam}
        new = cn_mean(mu_v, lam, rho, kind)
        if new >= MU_CAP:
            return True, it, new
        if abs(new - mu_c) <= 1e-12 * max(1.0, new):
            return False, it, new
        mu_c = new
    return False, max_iter, mu_c


def group_ga(ebn0_db: float, lam: dict, rho: dict, rate: float, G: int, r: float, max_iter: int = 20000,
             kind: str = "exact"):
    """Eqs. (4)-(17) for G groups with overlap ratio r.  Returns (converged, iterations, mu_c).

    Reading (the printed equations refer to means of the current sub-iteration on both sides):
    at sub-iteration g of iteration l, a VN's other i - 1 CNs are of class d (fraction x for
    g = 1 and y for g > 1, Eqs. (10)-(11)), class b (z, Eq. (12); none for g = 1) or class a
    (the rest, not updated yet in this iteration: mean mu_c^(l-1)).  Eq. (8) averages mu_v,i,p,q
    with the weights omega of Eq. (9); since mu_v,i,p,q is linear in (p, q) this is
    mu0 + (i - 1)(y mu_d + z mu_b + (1 - y - z) mu_a).  The CNs of the current group hold the
    messages of their previous update: a class-b CN the output of group g - 1 in this iteration,
    a fresh CN that of its group in iteration l - 1.  So in Eqs. (6)-(7) the term mu_c^{g,(l)}
    of the current group is taken from iteration l - 1, and for g = 1 mu_d is group 1's fresh
    output of iteration l - 1.  Class-c CNs output Eq. (15)-(16) from these mu_v; class-b CNs
    from mu_v' with p >= 1 (the weights of Eq. (9) restricted to p >= 1 and renormalised).
    Eq. (17) gives the iteration's mean.
    """
    mu0 = 2.0 / sigma2(ebn0_db, rate)
    D = G - (G - 1) * r
    x = 1.0 / D
    z = r / D
    mu_c = 0.0
    prev_cc = [0.0] * (G + 1)     # class-c output of each group in the previous iteration
    for it in range(1, max_iter + 1):
        cc = [0.0] * (G + 1)
        cb = [0.0] * (G + 1)
        for g in range(1, G + 1):
            if g == 1:
                mu_d, frac_d, frac_b, mu_b = prev_cc[1], x, 0.0, 0.0
            else:
                if r < 0.5:
                    acc = cc[1] + prev_cc[g] + sum((r / (1 - r)) * cb[k] + ((1 - 2 * r) / (1 - r)) * cc[k]
                                                   for k in range(2, g))
                else:
                    acc = cc[1] + prev_cc[g] + sum(cb[k] for k in range(2, g))
                mu_d, frac_d, frac_b = acc / g, g * (1 - r) / D, z
                mu_b = cc[g - 1] if g - 1 == 1 or r < 0.5 else cb[g - 1]
            frac_a = max(0.0, 1.0 - frac_d - frac_b)
            mu_a = mu_c
            mean_other = frac_d * mu_d + frac_b * mu_b + frac_a * mu_a
            mu_v = {i: mu0 + (i - 1) * mean_other for i in lam}
            cc[g] = cn_mean(mu_v, lam, rho, kind)
            if g > 1 and r > 0:
                # p >= 1: at least one class-d neighbour among the i - 1
                mu_vp = {}
                for i in lam:
                    n = i - 1
                    tot, acc_mu = 0.0, 0.0
                    for p in range(1, n + 1):
                        for q in range(0, n - p + 1):
                            w = math.comb(n, p) * math.comb(n - p, q) * frac_d ** p * frac_b ** q * \
                                max(0.0, 1 - frac_d - frac_b) ** (n - p - q)
                            tot += w
                            acc_mu += w * (mu0 + p * mu_d + q * mu_b + (n - p - q) * mu_a)
                    mu_vp[i] = acc_mu / tot if tot > 0 else mu_v[i]
                cb[g] = cn_mean(mu_vp, lam, rho, kind)
            else:
                cb[g] = cc[g]
        new = (r / D) * cb[G] + ((G - G * r) / D) * cc[G]
        if new >= MU_CAP:
            return True, it, new
        if abs(new - mu_c) <= 1e-12 * max(1.0, new):
            return False, it, new
        mu_c = new
        prev_cc = cc
    return False, max_iter, mu_c


def threshold(run, lo: float = 0.0, hi: float = 3.0, tol: float = 1e-4) -> float:
    """Smallest Eb/N0 (dB) in [lo, hi] at which run(ebn0) converges, by bisection."""
    if not run(hi)[0]:
        raise ValueError("no convergence at the upper end")
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if run(mid)[0]:
            hi = mid
        else:
            lo = mid
    return hi
