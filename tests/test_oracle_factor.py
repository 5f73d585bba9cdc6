"""Pins of the oracle's QAM map and sorted RQ (Alg. 1 + Section IV-B reversal).

Each check compares the oracle with something it does not contain: closed
forms, numpy/LAPACK routines (inverse, Cholesky, least squares) or an
independent restatement of the ordering rule by explicit projections.
"""
import numpy as np
import pytest

from paper_2602_12098_gb300 import workloads as W


def rand_h(rng, K, M):
    return (rng.standard_normal((K, M)) + 1j * rng.standard_normal((K, M))) / np.sqrt(2)


def test_qam_map_closed_form(orc):
    # 16-QAM: unit spacing 2 -> {+-1, +-3}^2 and tau = 8 (the benchmark configuration)
    pts = np.array([orc.qam_point(16, i) for i in range(16)])
    assert set(np.unique(pts.real)) == {-3.0, -1.0, 1.0, 3.0}
    assert set(np.unique(pts.imag)) == {-3.0, -1.0, 1.0, 3.0}
    assert len(set(pts.tolist())) == 16
    assert orc.default_tau(16) == 8.0
    for q in (4, 16, 64, 256):
        p = np.array([orc.qam_point(q, i) for i in range(q)])
        assert len(set(p.tolist())) == q                       # bijective
        assert np.allclose(np.mean(np.abs(p) ** 2), 2 * (q - 1) / 3)   # E|s|^2 closed form
        m = int(np.sqrt(q))
        assert np.all(np.abs(p.real) <= m - 1) and np.all(np.abs(p.real) % 2 == 1)
        # every point lies inside the fundamental region of the tau-lattice
        assert np.all(np.abs(p.real) < orc.default_tau(q) / 2)


@pytest.mark.parametrize("K,M", [(1, 1), (2, 3), (4, 4), (4, 8), (8, 8), (12, 16), (16, 16)])
def test_isrqd_is_inverse_gram_factor(orc, K, M):
    rng = np.random.default_rng(100 + 7 * K + M)
    for _ in range(5):
        H = rand_h(rng, K, M)
        rc, ul, R, Q = orc.isrqd(H)
        assert rc == 0
        assert sorted(ul.tolist()) == list(range(K))
        Hp = H[ul]
        # upper triangular, positive real diagonal
        assert np.allclose(np.tril(R, -1), 0)
        assert np.all(np.abs(np.diag(R).imag) < 1e-14) and np.all(np.diag(R).real > 0)
        # H_perm = R Q, with orthonormal rows of Q (first M columns carry H)
        assert np.allclose(R @ Q[:, :M], Hp, atol=1e-12)
        assert np.allclose(Q @ Q.conj().T, np.eye(K), atol=1e-12)
        U = orc.tri_inv_upper(R)
        assert np.allclose(R @ U, np.eye(K), atol=1e-12)
        # (H H^H)^-1 = U^H U in level order (numpy inverse)
        Ginv = np.linalg.inv(Hp @ Hp.conj().T)
        assert np.allclose(U.conj().T @ U, Ginv, rtol=1e-9, atol=1e-11)
        # uniqueness: U is the conjugate transpose of LAPACK's Cholesky factor of Ginv
        Uc = np.linalg.cholesky(Ginv).conj().T
        assert np.allclose(U, Uc, rtol=1e-8, atol=1e-10)
        # precoding matrix Q^H U = H^+ (numpy pseudo-inverse), Eq. viper_rq1
        P = Q[:, :M].conj().T @ U
        assert np.allclose(P, np.linalg.pinv(Hp), atol=1e-10)


def greedy_order_by_projection(H):
    """Min-norm-first rule restated with explicit least-squares projections.

    At each step pick the not-yet-placed row whose distance to the span of the
    rows already placed is smallest (ties: smallest index); the first pick is
    the deepest tree level. Returns (user_of_level, residual norms per level).
    """
    K = H.shape[0]
    chosen, res = [], []
    for _ in range(K):
        best, bestn = None, None
        for j in range(K):
            if j in chosen:
                continue
            h = H[j]
            if chosen:
                B = H[chosen].T                          # M x c
                coef, *_ = np.linalg.lstsq(B, h, rcond=None)
                r = h - B @ coef
            else:
                r = h
            n = np.linalg.norm(r)
            if bestn is None or n < bestn - 1e-13:
                best, bestn = j, n
        chosen.append(best)
        res.append(bestn)
    return np.array(chosen[::-1]), np.array(res[::-1])


@pytest.mark.parametrize("K,M", [(3, 3), (4, 4), (6, 8), (8, 8), (16, 16)])
def test_isrqd_order_matches_projection_rule(orc, K, M):
    rng = np.random.default_rng(7 * K + M)
    for _ in range(5):
        H = W.channels(rng, 1, K, M, "kron", 0.5, 0.2)[0].astype(np.complex128)
        rc, ul, R, Q = orc.isrqd(H)
        order, res = greedy_order_by_projection(H)
        assert rc == 0
        assert ul.tolist() == order.tolist()
        assert np.allclose(np.diag(R).real, res, rtol=1e-9)


def test_isrqd_weakest_row_at_last_level(orc):
    # Alg. 1 picks the min-norm row first; the reversal puts it at level K,
    # where the tree search starts, with R_KK = its norm.
    rng = np.random.default_rng(3)
    H = rand_h(rng, 5, 6)
    H[2] *= 0.1
    rc, ul, R, Q = orc.isrqd(H)
    assert ul[-1] == 2
    assert np.isclose(R[-1, -1].real, np.linalg.norm(H[2]))


def test_isrqd_identity_ties_by_user_index(orc):
    rc, ul, R, Q = orc.isrqd(np.eye(4))
    assert rc == 0
    assert ul.tolist() == [3, 2, 1, 0]
    assert np.allclose(R, np.eye(4))


@pytest.mark.parametrize("K,M,lam", [(4, 4, 0.3), (8, 4, 0.5), (6, 6, 1.0)])
def test_regularised_inverse_from_q2(orc, K, M, lam):
    """Eq. invr: lambda I = Rbar Qbar_2 gives Rbar^-1 = Qbar_2 / lambda, and the
    regularised factor equals the RZF inverse (H H^H + lambda^2 I)^-1 (overloaded K > M too)."""
    rng = np.random.default_rng(int(10 * lam) + K)
    H = rand_h(rng, K, M)
    rc, ul, R, Q = orc.isrqd(H, lam)
    assert rc == 0
    U = orc.tri_inv_upper(R)
    Q2 = Q[:, M:]
    # level order: Qbar_2's column for user u, level l sits at column ul[l]
    U_from_q2 = Q2[:, ul] / lam
    assert np.allclose(U, U_from_q2, atol=1e-10)
    Hp = H[ul]
    assert np.allclose(U.conj().T @ U, np.linalg.inv(Hp @ Hp.conj().T + lam ** 2 * np.eye(K)),
                       atol=1e-10)


def test_isrqd_singular_and_nonfinite(orc):
    rng = np.random.default_rng(5)
    H = rand_h(rng, 4, 4)
    H[3] = H[1] * (0.5 - 0.25j)
    rc, *_ = orc.isrqd(H)
    assert rc == 2
    H = rand_h(rng, 4, 4)
    H[0, 2] = np.nan
    rc, *_ = orc.isrqd(H)
    assert rc == 1
