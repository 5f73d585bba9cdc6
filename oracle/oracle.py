"""Python face of the FP64 CPU oracle (test infrastructure only).

The arithmetic lives in ``oracle.c`` (plain C, FP64); this module compiles it
with gcc on first use, loads it with ctypes and marshals numpy arrays. It also
holds the numpy-level linear baselines (ZF, MMSE) and the receiver of
Eq. (postproc) used for the symbol-error-rate comparison.

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py`` (CPU baseline and the
``--impl reference`` arm) may import this module. The CUDA library never does.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (OpenMP when gcc supports it)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    tmp = _SO + f".{os.getpid()}.tmp"
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    try:
        subprocess.run(base[:-1] + ["-fopenmp", base[-1]], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.orc_qam_point.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            L.orc_isrqd.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ip, dp, dp]
            L.orc_isrqd.restype = ctypes.c_int
            L.orc_tri_inv_upper.argtypes = [ctypes.c_int, dp, dp]
            L.orc_mop_kbest.argtypes = [ctypes.c_int, dp, ctypes.c_int, u64p, dp]
            L.orc_mop_kbest.restype = ctypes.c_int
            L.orc_rank9.argtypes = [ctypes.c_double, ctypes.c_double, ip]
            L.orc_rank9_lut.argtypes = [ctypes.c_double, ctypes.c_double, ip]
            L.orc_lut_order.argtypes = [ctypes.c_int, ip]
            L.orc_search_vector.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, dp,
                                            ctypes.c_double, ctypes.c_int, u64p, ip, dp, dp, ip, dp]
            L.orc_precode_batch.argtypes = ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int]
                                            + [ctypes.c_void_p] * 8
                                            + [ctypes.c_int])
            L.orc_precode_batch.restype = ctypes.c_int
            L.orc_brute_min.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ip]
            L.orc_brute_min.restype = ctypes.c_double
            L.orc_sphere_min.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ip]
            L.orc_sphere_min.restype = ctypes.c_double
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _cplx_in(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


# --------------------------------------------------------------------------
# Thin wrappers, one per C function.

def qam_point(qam: int, idx: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_qam_point(qam, int(idx), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def qam_points(qam: int, idx) -> np.ndarray:
    idx = np.asarray(idx)
    table = np.array([qam_point(qam, i) for i in range(qam)])
    return table[idx]


def default_tau(qam: int) -> float:
    """tau = 2*sqrt(Q) for the odd-integer grid (a reading, see oracle.c)."""
    return 2.0 * float(np.sqrt(qam))


def isrqd(H, lam: float = 0.0):
    """Alg. 1 + index reversal. Returns (status, user_of_level, R, Qbar)."""
    H = _cplx_in(H)
    K, M = H.shape
    ul = np.zeros(K, dtype=np.intc)
    R = np.zeros((K, K), dtype=np.complex128)
    Q = np.zeros((K, M + K), dtype=np.complex128)
    rc = lib().orc_isrqd(K, M, _p(H), float(lam), _p(ul, ctypes.c_int), _p(R), _p(Q))
    return rc, ul.astype(np.int64), R, Q


def tri_inv_upper(R) -> np.ndarray:
    R = _cplx_in(R)
    K = R.shape[0]
    out = np.zeros((K, K), dtype=np.complex128)
    lib().orc_tri_inv_upper(K, _p(R), _p(out))
    return out


def mop_kbest(w, n: int):
    """MoP K-Best. Returns (codes uint64[n'], metric float64[n'])."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    K = w.shape[0]
    codes = np.zeros(n, dtype=np.uint64)
    met = np.zeros(n, dtype=np.float64)
    got = lib().orc_mop_kbest(K, _p(w), int(n), _p(codes, ctypes.c_uint64), _p(met))
    if got < 0:
        raise ValueError("bad MoP arguments")
    return codes[:got], met[:got]


def rank9_lut(s_hat: complex) -> np.ndarray:
    """Region-LUT DEMAP order (alphabet indices) for the effective point."""
    order = np.zeros(9, dtype=np.intc)
    lib().orc_rank9_lut(float(np.real(s_hat)), float(np.imag(s_hat)), _p(order, ctypes.c_int))
    return order


def lut_order(region: int) -> np.ndarray:
    """The neighbour list of LUT region 0..71."""
    order = np.zeros(9, dtype=np.intc)
    lib().orc_lut_order(int(region), _p(order, ctypes.c_int))
    return order


def rank9(s_hat: complex) -> np.ndarray:
    order = np.zeros(9, dtype=np.intc)
    lib().orc_rank9(float(np.real(s_hat)), float(np.imag(s_hat)), _p(order, ctypes.c_int))
    return order.astype(np.int64)


def alphabet_point(a: int) -> complex:
    return complex(a // 3 - 1, a % 3 - 1)


def code_digits(code: int, K: int) -> list:
    """p_l - 1 per level (level index 0..K-1) of a packed path code."""
    return [(int(code) >> (4 * l)) & 15 for l in range(K)]


def search_vector(Rt, Qbar, M: int, v_level, tau: float, codes, want_all: bool = False):
    """Alg. 2 post-processing for one vector. Returns dict with t, gamma, x, best, d."""
    Rt = _cplx_in(Rt)
    Qbar = _cplx_in(Qbar)
    v = _cplx_in(v_level)
    codes = np.ascontiguousarray(np.asarray(codes, dtype=np.uint64))
    K = Rt.shape[0]
    Mq = Qbar.shape[1]
    n = codes.shape[0]
    t = np.zeros(2 * K, dtype=np.intc)
    g = ctypes.c_double()
    x = np.zeros(M, dtype=np.complex128)
    b = ctypes.c_int()
    d = np.zeros(n + 1, dtype=np.float64) if want_all else None
    lib().orc_search_vector(K, M, _p(Rt), _p(Qbar), Mq, _p(v), float(tau), n,
                            _p(codes, ctypes.c_uint64), _p(t, ctypes.c_int), ctypes.byref(g),
                            _p(x), ctypes.byref(b), _p(d) if d is not None else None)
    tt = t[0::2].astype(np.int64) + 1j * t[1::2].astype(np.int64)
    return {"t": tt, "gamma": g.value, "x": x, "best": b.value, "d": d}


def brute_min(Rt, v_level, tau: float):
    Rt = _cplx_in(Rt)
    v = _cplx_in(v_level)
    K = Rt.shape[0]
    t = np.zeros(2 * K, dtype=np.intc)
    g = lib().orc_brute_min(K, _p(Rt), _p(v), float(tau), _p(t, ctypes.c_int))
    return g, t[0::2] + 1j * t[1::2]


def sphere_min(Rt, v_level, tau: float):
    Rt = _cplx_in(Rt)
    v = _cplx_in(v_level)
    K = Rt.shape[0]
    t = np.zeros(2 * K, dtype=np.intc)
    g = lib().orc_sphere_min(K, _p(Rt), _p(v), float(tau), _p(t, ctypes.c_int))
    return g, t[0::2] + 1j * t[1::2]


def max_threads() -> int:
    return int(lib().orc_max_threads())


# --------------------------------------------------------------------------
# Per-channel factor bundle and the whole pipeline.

def factor_channel(H, n_paths: int, lam: float = 0.0):
    """Alg. 2 pre-processing of one channel (Regularize & factorize, MoP paths).

    Returns dict(status, user_of_level, R, Rt (= U), Qbar, w, codes, metric).
    """
    rc, ul, R, Q = isrqd(H, lam)
    out = {"status": rc, "user_of_level": ul, "R": R, "Qbar": Q}
    if rc != 0:
        return out
    Rt = tri_inv_upper(R)
    w = np.abs(np.diag(Rt)) ** 2
    codes, met = mop_kbest(w, n_paths)
    out.update(Rt=Rt, w=w, codes=codes, metric=met)
    return out


def precode_batch(H, sym_idx, vec_off, qam: int, n_paths: int, tau: float | None = None,
                  nthreads: int = 1, lam: float = 0.0, demap: str = "exact", frac_bits: int = 0,
                  word_bits: int = 16):
    """Whole pipeline (factor + MoP + search + x) over channels.

    frac_bits > 0 runs the fixed-point search (Section IV) with word_bits-bit
    values, frac_bits of them fractional; 0 is the floating-point search.

    H        complex64 [C, K, M]
    sym_idx  uint8 [V, K] (user order)
    vec_off  int32 [C+1]
    Returns dict(x complex128 [V, M], l int8 [V, K, 2], gamma [V], best [V], status [C]).
    """
    H = np.ascontiguousarray(np.asarray(H, dtype=np.complex64))
    C, K, M = H.shape
    sym_idx = np.ascontiguousarray(np.asarray(sym_idx, dtype=np.uint8))
    vec_off = np.ascontiguousarray(np.asarray(vec_off, dtype=np.int32))
    V = int(vec_off[-1])
    assert sym_idx.shape == (V, K)
    tau = default_tau(qam) if tau is None else float(tau)
    x = np.zeros((V, M), dtype=np.complex128)
    l = np.zeros((V, K, 2), dtype=np.int8)
    gamma = np.zeros(V, dtype=np.float64)
    best = np.zeros(V, dtype=np.int32)
    status = np.zeros(C, dtype=np.uint8)
    rc = lib().orc_precode_batch(K, M, qam, tau, float(lam), {"exact": 0, "lut": 1}[demap], int(frac_bits),
                                 int(word_bits), int(n_paths), C,
                                 H.ctypes.data, vec_off.ctypes.data, sym_idx.ctypes.data,
                                 x.ctypes.data, l.ctypes.data, gamma.ctypes.data,
                                 best.ctypes.data, status.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the batch arguments")
    return {"x": x, "l": l, "gamma": gamma, "best": best, "status": status}


# --------------------------------------------------------------------------
# Linear baselines and the receiver (Section II), for the SER comparison.

def zf_precode(H, s):
    """ZF: x = H^+ s / ||H^+ s|| (the zero-perturbation candidate)."""
    H = np.asarray(H, dtype=np.complex128)
    P = H.conj().T @ np.linalg.inv(H @ H.conj().T)
    y = P @ s
    g = float(np.real(np.vdot(y, y)))
    return y / np.sqrt(g), g


def mmse_matrix(H, sigma2: float):
    """G_MMSE = H^H (H H^H + alpha I)^-1 with alpha = sigma^2 N_R (Eq. 2 and text)."""
    H = np.asarray(H, dtype=np.complex128)
    K = H.shape[0]
    return H.conj().T @ np.linalg.inv(H @ H.conj().T + sigma2 * K * np.eye(K))


def qam_energy(qam: int) -> float:
    """E|s|^2 of the odd-integer grid: 2 (Q - 1) / 3."""
    return 2.0 * (qam - 1) / 3.0


def centered_mod(a, tau: float):
    """mod[a]_tau per real component, centred: a - tau*floor(a/tau + 1/2) (Eq. postproc)."""
    a = np.asarray(a)
    re = a.real - tau * np.floor(a.real / tau + 0.5)
    im = a.imag - tau * np.floor(a.imag / tau + 0.5)
    return re + 1j * im


def qam_slice(qam: int, y):
    """Nearest QAM index to each complex sample (per real dimension)."""
    m = int(round(np.sqrt(qam)))
    y = np.asarray(y)
    kr = np.clip(np.round((y.real + (m - 1)) / 2.0), 0, m - 1).astype(np.int64)
    ki = np.clip(np.round((y.imag + (m - 1)) / 2.0), 0, m - 1).astype(np.int64)
    return ki * m + kr
