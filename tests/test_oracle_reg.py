"""Pins of the oracle's regularised (Tikhonov) path: Alg. 2 "Regularize &
factorize" with lambda > 0, Hbar = [H lambda*I] (Section III-A-1), including
overloaded channels (more users than antennas, Section V).

Independent references: numpy's inverse of H H^H + lambda^2 I (the RZF
equivalence of Section III-A-1), a numpy brute force over all bounded
perturbations, and the lambda -> 0 limit.
"""
import itertools

import numpy as np
import pytest

from paper_2602_12098_gb300 import workloads as W


def _batch(orc, H, sym, qam, n, lam):
    C, K, M = H.shape
    S = sym.shape[0] // C
    off = W.vec_offsets_uniform(C, S)
    return off, orc.precode_batch(H, sym, off, qam, n, lam=lam)


def _user_points(orc, qam, sym_row):
    return orc.qam_points(qam, sym_row).astype(np.complex128)


@pytest.mark.parametrize("K,M,qam,n,lam", [(4, 4, 16, 16, 0.3), (8, 4, 4, 64, 0.5), (6, 6, 64, 40, 1.2)])
def test_rzf_direction_and_gamma(orc, K, M, qam, n, lam):
    """x sqrt(gamma) = H^H (H H^H + lam^2 I)^-1 (s + tau l) on the antennas, and
    gamma = u^H (H H^H + lam^2 I)^-1 u (the full ||w||^2 of Alg. 2)."""
    rng = W.rng_for(90, K * 10 + M)
    C, S = 6, 3
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    off, out = _batch(orc, H, sym, qam, n, lam)
    assert np.all(out["status"] == 0)
    tau = orc.default_tau(qam)
    for v in range(C * S):
        c = v // S
        Hc = H[c].astype(np.complex128)
        A = np.linalg.inv(Hc @ Hc.conj().T + lam * lam * np.eye(K))
        l = out["l"][v].astype(np.float64)
        u = _user_points(orc, qam, sym[v]) + tau * (l[:, 0] + 1j * l[:, 1])
        g = float(np.real(u.conj() @ A @ u))
        assert abs(out["gamma"][v] - g) <= 1e-9 * g
        y = Hc.conj().T @ (A @ u)
        assert np.allclose(out["x"][v] * np.sqrt(out["gamma"][v]), y, rtol=0, atol=1e-9 * np.linalg.norm(y))
        # the regularisation keeps part of the power off the antennas
        assert np.linalg.norm(out["x"][v]) < 1.0


@pytest.mark.parametrize("K,M,lam", [(2, 2, 0.4), (3, 2, 0.7), (3, 3, 0.2)])
def test_all_paths_reach_regularised_minimum(orc, K, M, lam):
    """n = 9^K: gamma is the brute-force minimum of u^H (H H^H + lam^2 I)^-1 u
    over every bounded perturbation (numpy enumeration)."""
    qam = 16
    rng = W.rng_for(91, K * 10 + M)
    C, S = 4, 2
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    off, out = _batch(orc, H, sym, qam, 9 ** K, lam)
    tau = orc.default_tau(qam)
    alph = [complex(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)]
    for v in range(C * S):
        Hc = H[v // S].astype(np.complex128)
        A = np.linalg.inv(Hc @ Hc.conj().T + lam * lam * np.eye(K))
        s = _user_points(orc, qam, sym[v])
        best = min(float(np.real((s + tau * np.array(t)).conj() @ A @ (s + tau * np.array(t))))
                   for t in itertools.product(alph, repeat=K))
        assert abs(out["gamma"][v] - best) <= 1e-9 * best


def test_lambda_to_zero_is_the_unregularised_path(orc):
    K = M = 5
    qam, n = 64, 50
    rng = W.rng_for(92, 0)
    H = W.channels(rng, 8, K, M)
    sym = W.symbols(rng, 8 * 2, K, qam)
    _, a = _batch(orc, H, sym, qam, n, 0.0)
    _, b = _batch(orc, H, sym, qam, n, 1e-7)
    assert np.array_equal(a["l"], b["l"])
    assert np.allclose(a["gamma"], b["gamma"], rtol=1e-8)
    assert np.allclose(a["x"], b["x"], atol=1e-7)


def test_overloaded_needs_lambda(orc):
    rng = W.rng_for(93, 0)
    H = W.channels(rng, 2, 6, 3)
    sym = W.symbols(rng, 2, 6, 4)
    with pytest.raises(ValueError):
        _batch(orc, H, sym, 4, 8, 0.0)
    _, out = _batch(orc, H, sym, 4, 8, 0.5)
    assert np.all(out["status"] == 0) and np.all(np.isfinite(out["x"])) and np.all(out["gamma"] > 0)
