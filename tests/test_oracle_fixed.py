"""Pins of the oracle's fixed-point search (Section IV, Precision and Numerical
Accuracy: signed 16-bit words, 8..13 fractional bits), under the reading
stated in the oracle: the level residuals in units of tau and the normalised
entries U~ = Rt_mk / Rt_mm are held as words with F fractional bits (round
half to even, saturation; the starting residuals formed from the rounded
entries), the PEDs, gamma and x are exact.

Independent references: the floating-point search (a wide word makes the
quantisation vanish), and numpy brute force over every bounded perturbation
of the quantised metric written in closed form (matrix form for unsaturated
words; the one saturating update of K = 2 for tiny words).
"""
import itertools

import numpy as np
import pytest

from paper_2602_12098_gb300 import workloads as W

ALPH = [complex(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)]


def _run(orc, H, sym, S, qam, n, **kw):
    C = H.shape[0]
    return orc.precode_batch(H, sym, W.vec_offsets_uniform(C, S), qam, n, **kw)


@pytest.mark.parametrize("K,M,qam,n", [(4, 4, 16, 16), (8, 8, 64, 64), (12, 12, 256, 96)])
def test_wide_word_is_the_float_search(orc, K, M, qam, n):
    """53-bit words with 40 fractional bits: rounding moves every value by
    < 2^-41 and nothing saturates, so the result is the floating-point search."""
    rng = W.rng_for(95, K)
    C, S = 6, 4
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    a = _run(orc, H, sym, S, qam, n)
    b = _run(orc, H, sym, S, qam, n, frac_bits=40, word_bits=53)
    assert np.array_equal(a["l"], b["l"]) and np.array_equal(a["best"], b["best"])
    assert np.allclose(a["gamma"], b["gamma"], rtol=1e-12, atol=0)
    assert np.allclose(a["x"], b["x"], rtol=0, atol=1e-12)


def _level_data(orc, Hc, sym_row, qam, n):
    f = orc.factor_channel(Hc, n)
    assert f["status"] == 0
    ul = np.asarray(f["user_of_level"])
    U = np.asarray(f["Rt"], dtype=np.complex128)          # upper triangular, level order
    v = orc.qam_points(qam, sym_row).astype(np.complex128)[ul]
    return ul, U, v


def _q(z, F, word):
    """Words with F fractional bits: round half to even, saturate (numpy)."""
    lim = 2.0 ** (word - 1) - 1
    re = np.clip(np.round(np.real(z) * 2.0 ** F), -lim, lim)
    im = np.clip(np.round(np.imag(z) * 2.0 ** F), -lim, lim)
    return (re + 1j * im) / 2.0 ** F


def _t_of(out, v, ul, K):
    l = out["l"][v].astype(np.float64)
    l = l[:, 0] + 1j * l[:, 1]                  # user order
    return -l[ul]                               # t = -l in level order


# F = 2 with 16-QAM puts b'_K = s_K / tau = +-1/8, +-3/8 exactly halfway between
# words, so rounding half away from zero (or towards it) changes the metric.
@pytest.mark.parametrize("K,M,qam,F", [(2, 2, 16, 2), (2, 3, 64, 8), (3, 3, 16, 11), (3, 4, 256, 6), (3, 3, 16, 2)])
def test_all_paths_minimise_the_quantised_metric(orc, K, M, qam, F):
    """n = 9^K: the chosen t minimises sum_l w_l tau^2 |b_q,l - (U~_q t)_l|^2 over
    all 9^K bounded t, with U~_q the unit upper matrix of quantised entries and
    b_q = q(U~_q v / tau) (no saturation at these sizes); gamma
    is the exact ||U (v - tau t)||^2 of that t."""
    word = 16
    rng = W.rng_for(96, K * 100 + F)
    C, S = 5, 3
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    tau = orc.default_tau(qam)
    out = _run(orc, H, sym, S, qam, 9 ** K, frac_bits=F, word_bits=word)
    lim = (2.0 ** (word - 1) - 1) / 2.0 ** F
    T = np.array(list(itertools.product(ALPH, repeat=K)), dtype=np.complex128)   # [9^K, K]
    for v in range(C * S):
        ul, U, vl = _level_data(orc, H[v // S], sym[v], qam, 9 ** K)
        d = np.diag(U)
        Ut = U / d[:, None]
        Uq = np.triu(_q(Ut, F, word), 1) + np.eye(K)
        bq = _q(Uq @ vl / tau, F, word)
        R = bq[None, :] - T @ (Uq - np.eye(K)).T        # residuals r'_l(t), all levels at once
        assert np.all(np.abs(R.real) < lim) and np.all(np.abs(R.imag) < lim)
        w = np.abs(d) ** 2 * tau * tau
        met = (np.abs(R - T) ** 2) @ w
        t = _t_of(out, v, ul, K)
        chosen = float((np.abs((bq - (Uq - np.eye(K)) @ t) - t) ** 2) @ w)
        assert chosen <= met.min() * (1 + 1e-12) + 1e-300
        g = float(np.sum(np.abs(U @ (vl - tau * t)) ** 2))
        assert abs(out["gamma"][v] - g) <= 1e-10 * g


@pytest.mark.parametrize("qam,F,word", [(16, 2, 3), (64, 1, 3), (256, 2, 4)])
def test_saturating_words_two_users(orc, qam, F, word):
    """Tiny words saturate b' and the one column update of K = 2:
    metric(t) = w_1 |b_q,1 - t_1|^2 + w_0 |sat(b_q,0 - U~_q,01 t_1) - t_0|^2,
    minimised over all 81 t by the n = 81 search."""
    K = 2
    rng = W.rng_for(97, qam + F)
    C, S = 12, 4
    H = W.channels(rng, C, K, K)
    sym = W.symbols(rng, C * S, K, qam)
    tau = orc.default_tau(qam)
    out = _run(orc, H, sym, S, qam, 81, frac_bits=F, word_bits=word)
    lim = (2.0 ** (word - 1) - 1) / 2.0 ** F
    n_sat = 0
    for v in range(C * S):
        ul, U, vl = _level_data(orc, H[v // S], sym[v], qam, 81)
        d = np.diag(U)
        Ut = U / d[:, None]
        uq = _q(Ut[0, 1], F, word)
        bq = _q(np.array([vl[0] + uq * vl[1], vl[1]]) / tau, F, word)
        w = np.abs(d) ** 2 * tau * tau

        def metric(t0, t1):
            r0 = bq[0] - uq * t1
            r0s = np.clip(r0.real, -lim, lim) + 1j * np.clip(r0.imag, -lim, lim)
            return w[1] * abs(bq[1] - t1) ** 2 + w[0] * abs(r0s - t0) ** 2, r0s != r0

        best = min(metric(t0, t1)[0] for t0 in ALPH for t1 in ALPH)
        n_sat += sum(bool(metric(t0, t1)[1]) for t0 in ALPH for t1 in ALPH)
        t = _t_of(out, v, ul, K)
        assert metric(t[0], t[1])[0] <= best * (1 + 1e-12) + 1e-300
        g = float(np.sum(np.abs(U @ (vl - tau * t)) ** 2))
        assert abs(out["gamma"][v] - g) <= 1e-10 * g
    assert n_sat > 0     # the saturating branch was exercised
