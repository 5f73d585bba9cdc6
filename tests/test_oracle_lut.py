"""Pins of the oracle's region-LUT DEMAP (Section III-A-2: the position of the
effective point relative to its nearest lattice point addresses a table of
neighbour orders; Alg. 2's DEMAP step), under the reading stated in
tests/golden/lut.txt: 9 cells x 8 octants, each list the exact distance order
from the octant centroid.

Independent references: hand-derived golden lists, the exact ranking at the
region centroids (FP64 distances, a different code path), symmetry, and the
exhaustive minimum when all 9^K paths are searched.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2602_12098_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lut.txt")


def _golden():
    for ln in open(GOLDEN):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        lhs, rhs = ln.split(":")
        re, im = (float(v) for v in lhs.split())
        yield complex(re, im), [int(v) for v in rhs.split()]


def test_golden_lists(orc):
    for s, want in _golden():
        assert list(orc.rank9_lut(s)) == want, s


def _centroid(region):
    cell, octn = divmod(region, 8)
    n0 = complex(cell // 3 - 1, cell % 3 - 1)
    a, b = (1 / 3, 1 / 6) if octn & 4 else (1 / 6, 1 / 3)
    return n0 + complex(a if octn & 1 else -a, b if octn & 2 else -b)


def test_lists_are_distance_orders_at_the_centroids(orc):
    """Every region's list is a permutation of the 9 points, sorted by the
    FP64 distance from the region's centroid (the exact ranking there, up to
    ties), and a point at the centroid falls in that region."""
    for r in range(72):
        lst = list(orc.lut_order(r))
        assert sorted(lst) == list(range(9))
        c = _centroid(r)
        assert list(orc.rank9_lut(c)) == lst
        pts = [complex(a // 3 - 1, a % 3 - 1) for a in lst]
        d = [abs(c - p) ** 2 for p in pts]
        assert all(d[i] <= d[i + 1] + 1e-12 for i in range(8)), (r, d)
        ex = list(orc.rank9(c))
        de = sorted(abs(c - complex(a // 3 - 1, a % 3 - 1)) ** 2 for a in ex)
        assert np.allclose(sorted(d), de)


def test_first_entry_is_the_nearest_point(orc):
    rng = np.random.default_rng(7)
    for s in rng.uniform(-2.5, 2.5, 400) + 1j * rng.uniform(-2.5, 2.5, 400):
        assert orc.rank9_lut(s)[0] == orc.rank9(s)[0]


def _region(s):
    n0 = complex((s.real > 0.5) - (s.real <= -0.5), (s.imag > 0.5) - (s.imag <= -0.5))
    d = s - n0
    octn = int(d.real > 0) | (int(d.imag > 0) << 1) | (int(abs(d.real) > abs(d.imag)) << 2)
    return int(((n0.real + 1) * 3 + (n0.imag + 1)) * 8 + octn)


def test_mirror_symmetry(orc):
    """Negating Re s_hat mirrors the region and its list: rank by rank the
    mirrored points are as far from the mirrored centroid (ties may swap,
    since ties go to the smaller alphabet index)."""
    mir = [3 * (2 - a // 3) + a % 3 for a in range(9)]
    pt = [complex(a // 3 - 1, a % 3 - 1) for a in range(9)]
    rng = np.random.default_rng(8)
    for s in rng.uniform(-1.9, 1.9, 200) + 1j * rng.uniform(-1.9, 1.9, 200):
        sm = complex(-s.real, s.imag)
        if abs(abs(s.real) - abs(s.imag)) < 1e-9 or abs(abs(s.real) - 0.5) < 1e-9:
            continue
        a = orc.rank9_lut(s)
        b = orc.rank9_lut(sm)
        cb = _centroid(_region(sm))
        da = [abs(cb - pt[mir[v]]) ** 2 for v in a]
        db = [abs(cb - pt[v]) ** 2 for v in b]
        assert np.allclose(da, db), s


@pytest.mark.parametrize("K,M", [(2, 2), (3, 3)])
def test_all_paths_reach_the_minimum_with_the_lut(orc, K, M):
    """With all 9^K paths every bounded perturbation is a candidate (each list
    is a bijection), so the LUT DEMAP also finds the exhaustive minimum."""
    qam = 16
    rng = W.rng_for(97, K)
    C, S = 6, 3
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    off = W.vec_offsets_uniform(C, S)
    out = orc.precode_batch(H, sym, off, qam, 9 ** K, demap="lut")
    tau = orc.default_tau(qam)
    for v in range(C * S):
        f = orc.factor_channel(H[v // S].astype(np.complex128), 1)
        vl = orc.qam_points(qam, sym[v])[f["user_of_level"]]
        g_bf, _ = orc.brute_min(f["Rt"], vl, tau)
        assert abs(out["gamma"][v] - g_bf) <= 1e-9 * g_bf


def test_lut_paths_between_optimum_and_zf(orc):
    K = M = 6
    qam, n = 64, 64
    rng = W.rng_for(98, 0)
    H = W.channels(rng, 20, K, M)
    sym = W.symbols(rng, 40, K, qam)
    off = W.vec_offsets_uniform(20, 2)
    lut = orc.precode_batch(H, sym, off, qam, n, demap="lut")
    tau = orc.default_tau(qam)
    for v in range(40):
        Hc = H[v // 2].astype(np.complex128)
        s = orc.qam_points(qam, sym[v])
        g_zf = float(np.real(s.conj() @ np.linalg.inv(Hc @ Hc.conj().T) @ s))
        f = orc.factor_channel(Hc, 1)
        g_opt = orc.sphere_min(f["Rt"], s[f["user_of_level"]], tau)[0]
        assert g_opt * (1 - 1e-9) <= lut["gamma"][v] <= g_zf * (1 + 1e-9)
