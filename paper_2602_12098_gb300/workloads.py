"""Seeded synthetic workloads shaped like the paper's (inputs only).

This module produces channels, QAM symbol indices and batch layouts. It holds
none of the precoder's arithmetic, and both the CUDA path's tests/benchmark
and the FP64 oracle draw their inputs from here, so the two sides see the same
bytes.

Shapes follow the paper's evaluation setup (Table I: 30 kHz SCS, 14-symbol
0.5 ms slots, N_T, N_R in [4, 16], QPSK..256-QAM, i.i.d. Rayleigh; Section V:
100 MHz = 273 RB x 12 = 3276 subcarriers). There is no dataset: every input is
drawn from numpy's PCG64 with a fixed seed.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 2602_12098
SYMBOLS_PER_SLOT = 14
SUBCARRIERS_PER_RB = 12


@dataclasses.dataclass(frozen=True)
class Workload:
    """One channels x symbols precoding batch of a single (K, M, Q, n) shape."""
    name: str
    K: int
    M: int
    qam: int
    n_paths: int
    subcarriers: int
    symbols: int
    channel: str = "iid"          # "iid" or "kron"
    rho_ap: float = 0.0
    rho_u: float = 0.0
    per_rb: bool = False          # one channel per 12-subcarrier RB
    seed_offset: int = 0

    @property
    def n_channels(self) -> int:
        if self.per_rb:
            return -(-self.subcarriers // SUBCARRIERS_PER_RB)
        return self.subcarriers

    @property
    def n_vectors(self) -> int:
        return self.subcarriers * self.symbols


# The three single-shape workloads of the evaluation (uneven batches and the
# serving loop are built from these shapes by the helpers further down).
SMALL_4x4 = Workload("4x4 16-QAM, 64 subcarriers x 1 symbol, 16 paths, iid",
                     K=4, M=4, qam=16, n_paths=16, subcarriers=64, symbols=1,
                     channel="iid", seed_offset=0)
RB_8x8 = Workload("8x8 64-QAM, 1638 subcarriers x 14 symbols, per-RB channel, 64 paths, iid",
                  K=8, M=8, qam=64, n_paths=64, subcarriers=1638, symbols=14,
                  channel="iid", per_rb=True, seed_offset=1)
SLOT_16x16 = Workload("16x16 256-QAM, 3276 subcarriers x 14 symbols (100 MHz slot), 256 paths, "
                      "Kronecker rho_ap=0.5 rho_u=0.2",
                      K=16, M=16, qam=256, n_paths=256, subcarriers=3276, symbols=14,
                      channel="kron", rho_ap=0.5, rho_u=0.2, seed_offset=2)
WORKLOADS = {"small_4x4": SMALL_4x4, "rb_8x8": RB_8x8, "slot_16x16": SLOT_16x16}

# The shapes of the paper's accelerator throughput table (Table II: K = M in
# {4, 8, 12, 16}, 16-QAM), here as whole 100 MHz slots with 8 paths, iid.
PAPER_POINTS = [Workload(f"{k}x{k} 16-QAM, 3276 subcarriers x 14 symbols, 8 paths, iid", K=k, M=k, qam=16,
                         n_paths=8, subcarriers=3276, symbols=14, channel="iid", seed_offset=6)
                for k in (4, 8, 12, 16)]


def rng_for(seed_offset: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for a workload (base seed + offset) and a sub-stream."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + seed_offset, stream]))


def exp_corr(n: int, rho: float) -> np.ndarray:
    """Exponential correlation matrix [R]_ij = rho^|i-j|."""
    idx = np.arange(n)
    return rho ** np.abs(idx[:, None] - idx[None, :])


def _psd_sqrt(R: np.ndarray) -> np.ndarray:
    w, V = np.linalg.eigh(R)
    return (V * np.sqrt(np.clip(w, 0.0, None))) @ V.conj().T


def channels(rng: np.random.Generator, C: int, K: int, M: int, model: str = "iid",
             rho_ap: float = 0.0, rho_u: float = 0.0) -> np.ndarray:
    """C Rayleigh channels H ~ CN(0, 1) entries, complex64 [C, K, M].

    model "kron": H = R_u^(1/2) H_w R_ap^(1/2) with exponential correlation.
    """
    Hw = (rng.standard_normal((C, K, M)) + 1j * rng.standard_normal((C, K, M))) / np.sqrt(2.0)
    if model == "kron":
        Ru = _psd_sqrt(exp_corr(K, rho_u))
        Ra = _psd_sqrt(exp_corr(M, rho_ap))
        Hw = Ru[None] @ Hw @ Ra[None]
    elif model != "iid":
        raise ValueError(f"unknown channel model {model!r}")
    return np.ascontiguousarray(Hw.astype(np.complex64))


def symbols(rng: np.random.Generator, V: int, K: int, qam: int) -> np.ndarray:
    """Uniform QAM indices, uint8 [V, K] (user order)."""
    return np.ascontiguousarray(rng.integers(0, qam, size=(V, K), dtype=np.int64).astype(np.uint8))


def vec_offsets_uniform(C: int, S: int) -> np.ndarray:
    return (np.arange(C + 1, dtype=np.int64) * S).astype(np.int32)


def vec_offsets_per_rb(subcarriers: int, symbols_per_slot: int) -> np.ndarray:
    """Channel = one 12-subcarrier RB; vectors of RB r are its subcarriers x symbols.

    The vector order is RB-major, so a channel's vectors are contiguous.
    """
    C = -(-subcarriers // SUBCARRIERS_PER_RB)
    off = [0]
    for r in range(C):
        sc = min(SUBCARRIERS_PER_RB, subcarriers - r * SUBCARRIERS_PER_RB)
        off.append(off[-1] + sc * symbols_per_slot)
    return np.asarray(off, dtype=np.int32)


@dataclasses.dataclass
class Batch:
    H: np.ndarray          # complex64 [C, K, M]
    sym: np.ndarray        # uint8 [V, K]
    vec_off: np.ndarray    # int32 [C+1]
    workload: Workload


def make_batch(w: Workload, slot: int = 0, subcarriers: int | None = None) -> Batch:
    """The seeded inputs of workload w (optionally truncated to fewer subcarriers).

    slot selects an independent draw (a later slot of the same cell).
    """
    sc = w.subcarriers if subcarriers is None else int(subcarriers)
    if w.per_rb:
        off = vec_offsets_per_rb(sc, w.symbols)
    else:
        off = vec_offsets_uniform(sc, w.symbols)
    C = off.shape[0] - 1
    rng = rng_for(w.seed_offset, 2 * slot)
    H = channels(rng, C, w.K, w.M, w.channel, w.rho_ap, w.rho_u)
    rng_s = rng_for(w.seed_offset, 2 * slot + 1)
    sym = symbols(rng_s, int(off[-1]), w.K, w.qam)
    return Batch(H=H, sym=sym, vec_off=off, workload=w)


# ---------------------------------------------------------------------------
# Uneven batch: many problems of mixed (K x M, Q, n_paths), each one channel
# with 14 symbols (one subcarrier over one slot).

UNEVEN_SHAPES = [(4, 8), (8, 16), (12, 16), (16, 16)]
UNEVEN_QAMS = [16, 64, 256]
UNEVEN_PATHS = [16, 64, 256, 1024]


@dataclasses.dataclass
class Problem:
    K: int
    M: int
    qam: int
    n_paths: int
    H: np.ndarray          # complex64 [K, M]
    sym: np.ndarray        # uint8 [S, K]


def uneven_problems(n_problems: int, symbols_per_problem: int = SYMBOLS_PER_SLOT,
                    seed_offset: int = 3) -> list:
    """Problems with (K x M, Q, n) drawn uniformly from the mixed-shape grid."""
    rng = rng_for(seed_offset, 0)
    out = []
    for _ in range(n_problems):
        K, M = UNEVEN_SHAPES[int(rng.integers(len(UNEVEN_SHAPES)))]
        qam = UNEVEN_QAMS[int(rng.integers(len(UNEVEN_QAMS)))]
        n = UNEVEN_PATHS[int(rng.integers(len(UNEVEN_PATHS)))]
        H = channels(rng, 1, K, M, "iid")[0]
        sym = symbols(rng, symbols_per_problem, K, qam)
        out.append(Problem(K, M, qam, n, H, sym))
    return out


# ---------------------------------------------------------------------------
# Serving: Poisson job arrivals per 0.5 ms slot, each job one cell's slot.

SERVE_KS = [4, 8, 12, 16]
SERVE_QAMS = [16, 64, 256]


@dataclasses.dataclass
class Job:
    job_id: int
    arrival_us: float
    K: int
    M: int
    qam: int
    n_paths: int
    subcarriers: int
    symbols: int
    seed: int


def poisson_jobs(n_slots: int, mean_per_slot: float = 4.0, slot_us: float = 500.0,
                 subcarriers: int = 3276, symbols_per_slot: int = SYMBOLS_PER_SLOT,
                 n_paths: int = 64, M: int = 16, seed_offset: int = 4) -> list:
    """Job list with exponential inter-arrival times (mean slot_us / mean_per_slot)."""
    rng = rng_for(seed_offset, 0)
    t = 0.0
    jobs = []
    horizon = n_slots * slot_us
    while True:
        t += float(rng.exponential(slot_us / mean_per_slot))
        if t >= horizon:
            break
        K = SERVE_KS[int(rng.integers(len(SERVE_KS)))]
        qam = SERVE_QAMS[int(rng.integers(len(SERVE_QAMS)))]
        jobs.append(Job(len(jobs), t, K, M, qam, n_paths, subcarriers, symbols_per_slot,
                        seed=int(rng.integers(1 << 31))))
    return jobs


def job_inputs(job: Job):
    """(H complex64 [C,K,M], sym uint8 [V,K]) of a serving job, one channel per subcarrier."""
    rng = np.random.Generator(np.random.PCG64([BASE_SEED + 5, job.seed]))
    H = channels(rng, job.subcarriers, job.K, job.M, "iid")
    sym = symbols(rng, job.subcarriers * job.symbols, job.K, job.qam)
    return H, sym


@dataclasses.dataclass
class PackedProblems:
    """Problems of an uneven batch packed into flat arrays (one device copy each).

    Element offsets of problem i: H_off[i] (complex64), sym_off[i] (uint8 rows
    of K), x_off[i] (complex64), l_off[i] (int8), g_off[i] (float32).
    """
    K: np.ndarray
    M: np.ndarray
    qam: np.ndarray
    n_paths: np.ndarray
    S: np.ndarray
    H: np.ndarray          # complex64 [sum K*M]
    sym: np.ndarray        # uint8 [sum S*K]
    H_off: np.ndarray
    sym_off: np.ndarray
    x_off: np.ndarray
    l_off: np.ndarray
    g_off: np.ndarray
    x_size: int
    l_size: int
    g_size: int


def pack_problems(problems: list) -> PackedProblems:
    K = np.array([p.K for p in problems], dtype=np.int64)
    M = np.array([p.M for p in problems], dtype=np.int64)
    S = np.array([p.sym.shape[0] for p in problems], dtype=np.int64)

    def offsets(sizes):
        o = np.zeros(len(sizes) + 1, dtype=np.int64)
        np.cumsum(sizes, out=o[1:])
        return o

    H_off = offsets(K * M)
    sym_off = offsets(S * K)
    x_off = offsets(S * M)
    l_off = offsets(S * K * 2)
    g_off = offsets(S)
    H = np.concatenate([p.H.reshape(-1) for p in problems]).astype(np.complex64)
    sym = np.concatenate([p.sym.reshape(-1) for p in problems]).astype(np.uint8) if S.sum() else \
        np.zeros(0, dtype=np.uint8)
    return PackedProblems(K=K, M=M, qam=np.array([p.qam for p in problems]), n_paths=np.array([p.n_paths for p in problems]),
                          S=S, H=H, sym=sym, H_off=H_off[:-1], sym_off=sym_off[:-1], x_off=x_off[:-1],
                          l_off=l_off[:-1], g_off=g_off[:-1], x_size=int(x_off[-1]), l_size=int(l_off[-1]),
                          g_size=int(g_off[-1]))
