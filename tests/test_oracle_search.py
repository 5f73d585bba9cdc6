"""Pins of the oracle's DEMAP ranking, parallel search (Alg. 2) and precoded output.

Independent references used here: hand-derived golden orderings, numpy brute
force over the bounded alphabet, a textbook nearest-plane (SIC) rounding on a
numpy Cholesky factor, closed forms (K = 1), the receiver's modulo of
Eq. (postproc), and metamorphic relations of the lattice problem.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2602_12098_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "rank9.txt")


def read_rank_gold():
    out = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b = line.split(":")
        sr, si = (float(v) for v in a.split())
        out.append((complex(sr, si), [int(v) for v in b.split()]))
    return out


@pytest.mark.parametrize("case", read_rank_gold(), ids=lambda c: str(c[0]))
def test_rank9_golden(orc, case):
    s, order = case
    assert orc.rank9(s).tolist() == order


def test_rank9_is_sorted_permutation(orc):
    rng = np.random.default_rng(1)
    for _ in range(500):
        s = complex(*rng.uniform(-2.5, 2.5, 2))
        o = orc.rank9(s)
        assert sorted(o.tolist()) == list(range(9))
        d = [abs(s - orc.alphabet_point(a)) ** 2 for a in o]
        assert all(d[i] <= d[i + 1] for i in range(8))


def numpy_factor(H, ul):
    """U from numpy: conj-transpose of the Cholesky factor of inv(G) in level order."""
    Hp = H[ul]
    return np.linalg.cholesky(np.linalg.inv(Hp @ Hp.conj().T)).conj().T


def gamma_np(U, v, tau, t):
    z = U @ (v - tau * t)
    return float(np.real(np.vdot(z, z)))


def all_t(K):
    pts = np.array([complex(a // 3 - 1, a % 3 - 1) for a in range(9)])
    for idx in itertools.product(range(9), repeat=K):
        yield pts[list(idx)]


def setup_problem(orc, rng, K, M, qam):
    H = (rng.standard_normal((K, M)) + 1j * rng.standard_normal((K, M))) / np.sqrt(2)
    f = orc.factor_channel(H, 1)
    ul = f["user_of_level"]
    s_user = orc.qam_points(qam, rng.integers(0, qam, K))
    return H, f, ul, s_user, s_user[ul]


@pytest.mark.parametrize("K,M,qam", [(2, 2, 16), (2, 3, 64), (3, 3, 4), (3, 4, 16)])
def test_all_paths_give_the_exact_bounded_minimum(orc, K, M, qam):
    """n = 9^K: each level's 9 ranks map to 9 distinct points, so the MoP paths
    cover every perturbation and the search returns the exact minimum."""
    rng = np.random.default_rng(K * 31 + M + qam)
    tau = orc.default_tau(qam)
    for _ in range(6):
        H, f, ul, s_user, v = setup_problem(orc, rng, K, M, qam)
        codes, _ = orc.mop_kbest(f["w"], 9 ** K)
        r = orc.search_vector(f["Rt"], f["Qbar"], M, v, tau, codes, want_all=True)
        U = numpy_factor(H, ul)
        gs = [gamma_np(U, v, tau, t) for t in all_t(K)]
        assert np.isclose(r["gamma"], min(gs), rtol=1e-10)
        # the candidate metrics are a permutation of all 9^K brute-force values
        # (plus the zero candidate, which repeats one of them)
        assert np.allclose(np.sort(r["d"][1:]), np.sort(gs), rtol=1e-9)


def test_sphere_and_brute_minimum(orc):
    rng = np.random.default_rng(11)
    for K in (2, 3, 4):
        for _ in range(4):
            H, f, ul, s_user, v = setup_problem(orc, rng, K, K, 16)
            g_se, t_se = orc.sphere_min(f["Rt"], v, 8.0)
            g_bf, t_bf = orc.brute_min(f["Rt"], v, 8.0)
            U = numpy_factor(H, ul)
            if K <= 3:
                assert np.isclose(g_bf, min(gamma_np(U, v, 8.0, t) for t in all_t(K)), rtol=1e-10)
            assert np.isclose(g_se, g_bf, rtol=1e-12)
            assert np.isclose(gamma_np(U, v, 8.0, t_se), g_se, rtol=1e-9)


@pytest.mark.parametrize("K,qam", [(4, 16), (8, 64), (16, 256)])
def test_single_path_is_clamped_babai(orc, K, qam):
    """n = 1 selects p = (1,...,1): nearest symbol per level = successive
    nearest-plane rounding clamped to {-1,0,1}; the zero candidate competes."""
    rng = np.random.default_rng(K + qam)
    tau = orc.default_tau(qam)
    for _ in range(8):
        H, f, ul, s_user, v = setup_problem(orc, rng, K, K, qam)
        U = numpy_factor(H, ul)
        t = np.zeros(K, dtype=complex)
        for l in range(K - 1, -1, -1):               # textbook SIC on numpy's U
            y = (U[l, l:] @ v[l:] - tau * (U[l, l + 1:] @ t[l + 1:])) / (U[l, l] * tau)
            t[l] = np.clip(np.round(y.real), -1, 1) + 1j * np.clip(np.round(y.imag), -1, 1)
        g_babai = gamma_np(U, v, tau, t)
        g_zero = gamma_np(U, v, tau, np.zeros(K))
        r = orc.search_vector(f["Rt"], f["Qbar"], K, v, tau, np.array([0], dtype=np.uint64))
        assert np.isclose(r["gamma"], min(g_babai, g_zero), rtol=1e-10)
        if g_babai < g_zero * (1 - 1e-9):
            assert np.allclose(r["t"], t)


@pytest.mark.parametrize("K,qam,n", [(8, 64, 64), (16, 256, 256)])
def test_gamma_ordering_opt_vp_zf(orc, K, qam, n):
    rng = np.random.default_rng(K * n)
    tau = orc.default_tau(qam)
    for _ in range(4):
        H, f, ul, s_user, v = setup_problem(orc, rng, K, K, qam)
        codes, _ = orc.mop_kbest(f["w"], n)
        r = orc.search_vector(f["Rt"], f["Qbar"], K, v, tau, codes, want_all=True)
        g_zf = float(np.real(s_user.conj() @ np.linalg.inv(H @ H.conj().T) @ s_user))
        g_opt, _ = orc.sphere_min(f["Rt"], v, tau)
        assert np.isclose(r["d"][0], g_zf, rtol=1e-9)     # candidate 0 is ZF
        assert g_opt <= r["gamma"] * (1 + 1e-12) and r["gamma"] <= g_zf * (1 + 1e-12)
        assert r["best"] == int(np.argmin(r["d"]))


def test_single_user_closed_form(orc):
    """K = 1: every QAM point lies in the fundamental tau-square, so t = 0,
    gamma = |v|^2 / |h|^2 and x = conj(h) v / (|h| |v|)."""
    rng = np.random.default_rng(2)
    for M in (1, 4):
        for qam in (4, 16, 256):
            h = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) / np.sqrt(2)
            idx = rng.integers(0, qam, (3, 1)).astype(np.uint8)
            out = orc.precode_batch(h[None, None, :], idx, np.array([0, 3]), qam, 9)
            for k in range(3):
                v = orc.qam_point(qam, int(idx[k, 0]))
                assert np.all(out["l"][k] == 0)
                assert np.isclose(out["gamma"][k], abs(v) ** 2 / np.linalg.norm(h) ** 2, rtol=1e-6)
                xe = h.conj() * v / (np.linalg.norm(h) * abs(v))
                assert np.allclose(out["x"][k], xe, atol=1e-6)


def run_batch(orc, H, sym, qam, n, S):
    C = H.shape[0]
    off = np.arange(C + 1, dtype=np.int32) * S
    return orc.precode_batch(H, sym, off, qam, n)


@pytest.mark.parametrize("K,M,qam,n", [(4, 4, 16, 16), (4, 8, 64, 32), (8, 8, 64, 64)])
def test_pipeline_invariants(orc, K, M, qam, n):
    """||x|| = 1 (P_T = 1), H x sqrt(gamma) = s + tau l, and the receiver's modulo
    (Eq. postproc) gives back s exactly in the noiseless case."""
    rng = W.rng_for(50, K * 100 + M)
    C, S = 6, 5
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    out = run_batch(orc, H, sym, qam, n, S)
    tau = orc.default_tau(qam)
    assert np.all(out["status"] == 0)
    for v in range(C * S):
        c = v // S
        s = orc.qam_points(qam, sym[v])
        lv = out["l"][v, :, 0] + 1j * out["l"][v, :, 1]
        x = out["x"][v]
        assert np.isclose(np.linalg.norm(x), 1.0, atol=1e-12)
        y = H[c].astype(np.complex128) @ x * np.sqrt(out["gamma"][v])
        assert np.allclose(y, s + tau * lv, atol=1e-9)
        assert np.allclose(orc.centered_mod(y, tau), s, atol=1e-9)
        assert np.all(np.abs(out["l"][v]) <= 1)


def test_metamorphic_relations(orc):
    """cH, e^{j theta} H and H V (V unitary) leave the lattice problem unchanged:
    same l; gamma / c^2; x, e^{-j theta} x and V^H x respectively."""
    K, M, qam, n, S = 8, 8, 64, 64, 4
    rng = W.rng_for(51, 0)
    C = 4
    H = W.channels(rng, C, K, M).astype(np.complex128)
    sym = W.symbols(rng, C * S, K, qam)
    base = run_batch(orc, H, sym, qam, n, S)
    c = 2.0                                   # power-of-two scale keeps float32 H exact
    o1 = run_batch(orc, H * c, sym, qam, n, S)
    assert np.array_equal(o1["l"], base["l"])
    assert np.allclose(o1["gamma"] * c ** 2, base["gamma"], rtol=1e-9)
    assert np.allclose(o1["x"], base["x"], atol=1e-9)
    th = 0.7
    Hr = (H * np.exp(1j * th)).astype(np.complex64)
    o2 = run_batch(orc, Hr, sym, qam, n, S)
    agree = np.all(o2["l"] == base["l"], axis=(1, 2))
    assert agree.mean() > 0.9                 # float32 rounding of the rotated H may flip near-ties
    assert np.allclose(o2["x"][agree], base["x"][agree] * np.exp(-1j * th), atol=2e-5)
    Z = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    V, _ = np.linalg.qr(Z)
    Hv = (H @ V).astype(np.complex64)
    o3 = run_batch(orc, Hv, sym, qam, n, S)
    agree = np.all(o3["l"] == base["l"], axis=(1, 2))
    assert agree.mean() > 0.9
    assert np.allclose(o3["x"][agree], base["x"][agree] @ V.conj(), atol=2e-5)
    assert np.allclose(o3["gamma"][agree], base["gamma"][agree], rtol=2e-5)


def test_user_permutation_equivariance(orc):
    K, M, qam, n, S = 6, 8, 16, 32, 3
    rng = W.rng_for(52, 0)
    H = W.channels(rng, 3, K, M)
    sym = W.symbols(rng, 9, K, qam)
    base = run_batch(orc, H, sym, qam, n, S)
    pi = rng.permutation(K)
    o = run_batch(orc, np.ascontiguousarray(H[:, pi]), np.ascontiguousarray(sym[:, pi]), qam, n, S)
    assert np.array_equal(o["l"], base["l"][:, pi])
    assert np.allclose(o["gamma"], base["gamma"], rtol=1e-9)
    assert np.allclose(o["x"], base["x"], atol=1e-9)


def test_bad_channels_give_zero_outputs(orc):
    rng = W.rng_for(53, 0)
    H = W.channels(rng, 3, 4, 4)
    H[1, 2] = H[1, 0]
    H[2, 0, 0] = np.inf
    sym = W.symbols(rng, 6, 4, 16)
    out = run_batch(orc, H, sym, 16, 16, 2)
    assert out["status"].tolist() == [0, 2, 1]
    assert np.all(out["x"][2:] == 0) and np.all(out["gamma"][2:] == 0)


# --------------------------------------------------------------------------
# The path digit of level l drives level l. Eq. (mop) scores digit p_l with
# the weight |Rt_ll|^2 of level l, and DEMAP in Alg. 2 applies that same digit
# at level l. The tests below rebuild every candidate in numpy from those
# definitions, at budgets 1 < n < 9^K, where the binding decides the result.

def numpy_candidates(U, v, tau, codes):
    """t and d = ||U (v - tau t)||^2 of the zero candidate and every path, level
    by level from level K: effective point of Eq. (17) on numpy's factor U,
    DEMAP = the digit-th entry of the 9 points sorted by (squared distance,
    alphabet index), the digit taken from nibble l of the code."""
    K = U.shape[0]
    pts = np.array([complex(a // 3 - 1, a % 3 - 1) for a in range(9)])
    ts = [np.zeros(K, dtype=complex)]
    for code in codes:
        t = np.zeros(K, dtype=complex)
        for l in range(K - 1, -1, -1):
            s_hat = (U[l, l:] @ v[l:] - tau * (U[l, l + 1:] @ t[l + 1:])) / (U[l, l] * tau)
            dist = np.abs(s_hat - pts) ** 2
            order = np.lexsort((np.arange(9), dist))
            t[l] = pts[order[(int(code) >> (4 * l)) & 15]]
        ts.append(t)
    return ts, np.array([gamma_np(U, v, tau, t) for t in ts])


@pytest.mark.parametrize("K,M,qam,n", [(3, 3, 16, 50), (3, 4, 64, 200), (4, 4, 16, 16), (4, 4, 16, 300)])
def test_digit_of_level_l_drives_level_l(orc, K, M, qam, n):
    rng = np.random.default_rng(7000 + 10 * K + n)
    tau = orc.default_tau(qam)
    for _ in range(6):
        H, f, ul, s_user, v = setup_problem(orc, rng, K, M, qam)
        U = numpy_factor(H, ul)
        w = np.abs(np.diag(U)) ** 2
        codes, met = orc.mop_kbest(f["w"], n)
        # Eq. (mop): nibble l of a code is scored by the weight of level l
        nib = np.array([[(int(c) >> (4 * l)) & 15 for l in range(K)] for c in codes])
        assert np.allclose(nib @ w, met, rtol=1e-9, atol=1e-12)
        # Alg. 2: the same nibble picks the DEMAP rank at level l
        ts, d = numpy_candidates(U, v, tau, codes)
        r = orc.search_vector(f["Rt"], f["Qbar"], M, v, tau, codes, want_all=True)
        assert np.allclose(r["d"], d, rtol=1e-9)
        kb = int(np.argmin(d))
        assert r["best"] == kb and np.allclose(r["t"], ts[kb])


@pytest.mark.parametrize("K,M,qam,n", [(3, 3, 16, 50), (4, 4, 16, 16)])
def test_pipeline_and_fixed_search_bind_digits_to_levels(orc, K, M, qam, n):
    """The batch pipeline, in floating point and as the fixed-point search with
    53-bit words (no rounding that matters), picks the numpy-built argmin."""
    rng = W.rng_for(96, 10 * K + n)
    C, S = 4, 5
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    tau = orc.default_tau(qam)
    outs = [run_batch(orc, H, sym, qam, n, S),
            orc.precode_batch(H, sym, W.vec_offsets_uniform(C, S), qam, n, frac_bits=40, word_bits=53)]
    for c in range(C):
        f = orc.factor_channel(H[c], n)
        ul = f["user_of_level"]
        U = numpy_factor(H[c].astype(np.complex128), ul)
        for k in range(S):
            vi = c * S + k
            v = orc.qam_points(qam, sym[vi])[ul]
            ts, d = numpy_candidates(U, v, tau, f["codes"])
            kb = int(np.argmin(d))
            for out in outs:
                # the chosen candidate is the minimum; an exact tie (the zero
                # candidate against an all-zero path) may go either way, by the
                # order of the sums
                kc = int(out["best"][vi])
                assert kc == kb or np.isclose(d[kc], d[kb], rtol=1e-13, atol=0)
                assert np.isclose(out["gamma"][vi], d[kb], rtol=1e-9)
                lv = out["l"][vi, :, 0] + 1j * out["l"][vi, :, 1]
                assert np.allclose(lv[ul], -ts[kc])


GOLD_SEARCH = os.path.join(os.path.dirname(__file__), "golden", "search_k2.txt")


def read_search_gold():
    cases = []
    for line in open(GOLD_SEARCH):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = dict(kv.split("=", 1) for kv in line.split(";"))
        Rt = np.array([complex(s) for s in f["Rt"].split()]).reshape(2, 2)
        v = np.array([complex(s) for s in f["v"].split()])
        codes = np.array([int(s) for s in f["codes"].split()], dtype=np.uint64)
        d = np.array([float(s) for s in f["d"].split()])
        t = np.array([complex(s) for s in f["t"].split()])
        cases.append((Rt, v, float(f["tau"]), codes, d, int(f["best"]), t))
    return cases


@pytest.mark.parametrize("case", read_search_gold())
def test_search_golden_two_levels(orc, case):
    Rt, v, tau, codes, d, best, t = case
    w = np.abs(np.diag(Rt)) ** 2
    got_codes, _ = orc.mop_kbest(w, len(codes))
    assert got_codes.tolist() == codes.tolist()
    r = orc.search_vector(Rt, np.eye(2), 2, v, tau, codes, want_all=True)
    assert np.allclose(r["d"], d, rtol=1e-12)
    assert r["best"] == best and np.allclose(r["t"], t)
