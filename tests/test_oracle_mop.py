"""Pins of the oracle's Metric-of-Promise K-Best (Eq. mop and the K-Best text).

K-Best keeps n survivors per level. For this separable, non-negative metric
(with a tie order that is consistent under extension) it returns exactly the n
smallest of all 9^K position vectors; the brute-force sort below checks that,
and hand-derived golden lists check the metric itself.
"""
import itertools
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "mop.txt")


def brute_topn(w, n):
    K = len(w)
    rows = []
    for ks in itertools.product(range(9), repeat=K):
        m = 0.0
        for l in range(K):            # left to right, as the partial metrics accumulate
            m = m + float(w[l]) * ks[l]
        code = sum(ks[l] << (4 * l) for l in range(K))
        rows.append((m, code))
    rows.sort()
    return rows[:n]


def read_gold():
    cases = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, tail = line.split(":")
        codes, mets = tail.split("|")
        h = head.split()
        K, n = int(h[0]), int(h[1])
        w = [float(v) for v in h[2:2 + K]]
        cases.append((K, n, w, [int(c) for c in codes.split()], [float(m) for m in mets.split()]))
    return cases


@pytest.mark.parametrize("case", read_gold(), ids=lambda c: f"K{c[0]}n{c[1]}")
def test_mop_golden(orc, case):
    K, n, w, codes, mets = case
    got_c, got_m = orc.mop_kbest(np.array(w), n)
    assert got_c.tolist() == codes
    assert np.allclose(got_m, mets)


@pytest.mark.parametrize("K", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 5, 16, 64, 200])
def test_kbest_equals_brute_force(orc, K, n):
    rng = np.random.default_rng(K * 1000 + n)
    for _ in range(3):
        w = rng.exponential(1.0, size=K)
        got_c, got_m = orc.mop_kbest(w, n)
        ref = brute_topn(w, n)
        assert got_c.tolist() == [c for _, c in ref]
        assert np.allclose(got_m, [m for m, _ in ref], rtol=1e-14, atol=1e-14)


def test_kbest_all_vectors_and_ties(orc):
    # n = 9^K returns every position vector once; equal weights (an orthogonal
    # channel) create many exact ties, resolved by the code order.
    for w in ([1.0, 1.0, 1.0], [0.75, 0.75, 2.25]):   # dyadic: sums exact
        got_c, got_m = orc.mop_kbest(np.array(w), 729)
        ref = brute_topn(w, 729)
        assert len(set(got_c.tolist())) == 729
        assert got_c.tolist() == [c for _, c in ref]
    got_c, _ = orc.mop_kbest(np.array([1.0, 2.0]), 500)   # n > 9^K
    assert len(got_c) == 81


def test_kbest_sorted_and_scale_free(orc):
    rng = np.random.default_rng(9)
    w = rng.exponential(1.0, size=16)
    c1, m1 = orc.mop_kbest(w, 256)
    assert np.all(np.diff(m1) >= 0)
    assert c1[0] == 0 and m1[0] == 0.0
    c2, m2 = orc.mop_kbest(w * 3.5, 256)          # H -> H/sqrt(3.5) scales every weight
    assert c1.tolist() == c2.tolist()
    # every prefix of a selected vector is itself selected (closure of K-Best)
    s = set(c1.tolist())
    for c in c1.tolist():
        for l in range(16):
            trunc = c & ~(0xF << (4 * l))
            # lowering one digit to 0 can only lower the metric
            assert trunc in s
