"""A host model of how the GA kernels invert the closed-form Phi (ga_phi_inv_closed in
csrc/ga.cu), held against the oracle's plain bisection (oracle/ga.py phi_inv, kind "approx").

The kernel takes the bisection's decisions far from the root r from r itself (closed form below
mu = 10, Newton's method on log Phi above), starts five levels above the bisection's last level,
and lets the warp's 31 lanes evaluate the next five levels' midpoints at once; the band where the
closed form jumps up at mu = 10, p near Phi(0+) and brackets with an end within delta of r go
through the whole bisection.  The claim is that it returns the one-level bisection's value bit
for bit.  This model repeats those steps in Python (math.log / math.pow in place of CUDA's) and
compares with the oracle on values of p spread over every case.
"""
import math
import random

from oracle import ga

PHI = ga.phi_approx
P_LEFT = math.exp(-0.4527 * 10.0 ** 0.86 + 0.0218)                            # Phi(10-)
P_RIGHT = math.sqrt(math.pi / 10.0) * math.exp(-10.0 / 4.0) * (1.0 - 10.0 / 70.0)  # Phi(10)
P_ZERO = math.exp(0.0218)                                                       # Phi(0+)


def _tree(p, lo, hi, steps, evals):
    """Five bisection levels per round: node j (heap order) evaluated by lane j - 1."""
    while steps < 200:
        ball = 0
        for lane in range(31):
            j = lane + 1
            l, h = lo, hi
            for b in range(j.bit_length() - 2, -1, -1):
                m = 0.5 * (l + h)
                if (j >> b) & 1:
                    l = m
                else:
                    h = m
            if PHI(0.5 * (l + h)) > p:
                ball |= 1 << lane
        evals[0] += 1
        node = 1
        for _ in range(5):
            if steps >= 200:
                break
            m = 0.5 * (lo + hi)
            if (ball >> (node - 1)) & 1:
                lo, node = m, 2 * node + 1
            else:
                hi, node = m, 2 * node
            steps += 1
            if hi - lo <= 1e-13 * max(1.0, hi):
                return 0.5 * (lo + hi)
    return 0.5 * (lo + hi)


def _seeded(p, evals):
    if PHI(200.0) >= p:
        return 200.0
    left = P_RIGHT * (1 + 1e-9) < p < P_ZERO * (1 - 1e-9)
    if not left and not p < P_LEFT * (1 - 1e-9):
        return _tree(p, 0.0, 200.0, 0, evals)
    lp = math.log(p)
    if left:
        r = ((0.0218 - lp) / 0.4527) ** (1.0 / 0.86)
    else:
        r = min(200.0, max(10.0, -4.0 * lp))
        for _ in range(6):
            g = math.log(math.sqrt(math.pi / r) * (1.0 - 10.0 / (7.0 * r))) - r / 4.0 - lp
            dg = -0.5 / r - 0.25 + (10.0 / (7.0 * r * r)) / (1.0 - 10.0 / (7.0 * r))
            r = min(200.0, max(10.0, r - g / dg))
    k = math.ceil(math.log2(200.0 / (1e-13 * max(1.0, r)))) - 2
    for _ in range(8):
        w = math.ldexp(200.0, -k)
        if w <= 1e-13 * max(1.0, w * math.floor(r / w) + w):
            break
        k += 1
    else:
        return _tree(p, 0.0, 200.0, 0, evals)
    k -= 5
    w = math.ldexp(200.0, -k)
    lo = w * math.floor(r / w)
    hi = lo + w
    d = 4e-14 * max(1.0, r)
    if lo <= r < hi and (lo == 0.0 or r - lo > d) and (hi == 200.0 or hi - r > d):
        return _tree(p, lo, hi, k, evals)
    return _tree(p, 0.0, 200.0, 0, evals)


def test_seeded_bisection_equals_plain_bisection():
    rng = random.Random(2)
    ps = ([rng.random() for _ in range(1500)]
          + [math.exp(-rng.uniform(0.0, 50.0)) for _ in range(1500)]
          + [rng.uniform(0.0384, 0.0395) for _ in range(300)]          # around the jump at mu = 10
          + [1.0, 1.01, 1.03, 1e-300, 0.0, -1.0, 2e-8, P_LEFT, P_RIGHT, P_ZERO, PHI(200.0)])
    evals = [0]
    bad = [p for p in ps if _seeded(p, evals) != ga.phi_inv(p, "approx")]
    assert not bad, bad[:5]
    # the point of it: about two rounds of evaluations instead of the plain loop's ~48
    assert evals[0] / len(ps) < 2.5
