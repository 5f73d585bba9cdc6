"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Sizes: the small 4x4 workload in full; the 8x8 per-RB and 16x16 slot
workloads on reduced subcarrier counts (several tiles of 32 paths and a
ragged vector tail) in full, and at their full sizes on sampled vectors.
"""
import numpy as np
import pytest
import torch

import paper_2602_12098_gb300 as vp
from paper_2602_12098_gb300 import workloads as W
from vp_gpu_util import assert_parity, compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vp.load()


def oracle_run(orc, H, sym, off, qam, n, tau=None):
    return orc.precode_batch(H, sym, off, qam, n, tau=tau, nthreads=orc.max_threads())


def check_factor(orc, H, gpu, tol=2e-5):
    """U (level order), user order and P against the oracle's Alg. 1 factor."""
    C = H.shape[0]
    order_ok = 0
    for c in range(C):
        f = orc.factor_channel(H[c].astype(np.complex128), 1)
        if f["status"] != 0:
            continue
        if np.array_equal(gpu["ul"][c], f["user_of_level"]):
            order_ok += 1
            e = np.linalg.norm(gpu["U"][c] - f["Rt"]) / np.linalg.norm(f["Rt"])
            assert e <= tol, (c, e)
        Hc = H[c].astype(np.complex128)
        eP = np.linalg.norm(gpu["P"][c] - np.linalg.pinv(Hc)) / np.linalg.norm(np.linalg.pinv(Hc))
        assert eP <= tol, (c, eP)
    assert order_ok >= 0.99 * C


def test_small_4x4_full(orc):
    b = W.make_batch(W.SMALL_4x4)
    w = b.workload
    gpu = run_gpu(b.H, b.sym, b.vec_off, w.qam, w.n_paths)
    ref = oracle_run(orc, b.H, b.sym, b.vec_off, w.qam, w.n_paths)
    assert np.all(gpu["status"] == 0)
    check_factor(orc, b.H, gpu)
    # candidate paths equal the oracle's MoP K-Best (rank order)
    same = 0
    for c in range(b.H.shape[0]):
        f = orc.factor_channel(b.H[c].astype(np.complex128), w.n_paths)
        same += int(np.array_equal(gpu["codes"][c], f["codes"]))
    assert same >= 0.98 * b.H.shape[0]
    st = compare(orc, b.H, b.sym, b.vec_off, w.qam, gpu, ref)
    assert_parity(st)


@pytest.mark.parametrize("K,M,qam,n", [(2, 2, 16, 81), (3, 3, 64, 729), (3, 4, 4, 729)])
def test_all_paths_reach_exhaustive_minimum(orc, K, M, qam, n):
    """n = 9^K: the GPU search covers every bounded perturbation, so its gamma
    equals the oracle's exhaustive minimum."""
    rng = W.rng_for(70, K * 10 + M)
    C, S = 40, 3
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    off = W.vec_offsets_uniform(C, S)
    gpu = run_gpu(H, sym, off, qam, n)
    tau = orc.default_tau(qam)
    for v in range(C * S):
        c = v // S
        f = orc.factor_channel(H[c].astype(np.complex128), 1)
        vl = orc.qam_points(qam, sym[v])[f["user_of_level"]]
        g_bf, _ = orc.brute_min(f["Rt"], vl, tau)
        assert abs(gpu["gamma"][v] - g_bf) <= 1e-5 * g_bf


@pytest.mark.parametrize("wl,sub", [(W.RB_8x8, 24 * 12 + 6), (W.SLOT_16x16, 40)])
def test_reduced_full_compare(orc, wl, sub):
    b = W.make_batch(wl, subcarriers=sub)
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths)
    ref = oracle_run(orc, b.H, b.sym, b.vec_off, wl.qam, wl.n_paths)
    assert np.array_equal(gpu["status"] & 3, ref["status"])
    check_factor(orc, b.H, gpu)
    # candidate paths: the oracle's MoP K-Best on the same channel (rank order)
    same = 0
    for c in range(b.H.shape[0]):
        f = orc.factor_channel(b.H[c].astype(np.complex128), wl.n_paths)
        same += int(np.array_equal(gpu["codes"][c], f["codes"]))
    assert same >= 0.95 * b.H.shape[0], same
    st = compare(orc, b.H, b.sym, b.vec_off, wl.qam, gpu, ref)
    print(wl.name, st, "fp64 channels:", int(np.sum(gpu["status"] == vp.VP_CH_FP64)))
    assert_parity(st)


@pytest.mark.parametrize("wl", [W.RB_8x8, W.SLOT_16x16])
def test_full_size_sampled(orc, wl):
    """Full-size launch (the benchmark's configuration); oracle on sampled vectors."""
    b = W.make_batch(wl)
    S = wl.symbols
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, want_factor=False,
                  uniform_S=None if wl.per_rb else S)
    C = b.H.shape[0]
    rng = np.random.default_rng(5)
    chans = np.sort(rng.choice(C, size=min(C, 512), replace=False))
    vecs, off = [], [0]
    for c in chans:
        vv = np.arange(b.vec_off[c], b.vec_off[c + 1])
        pick = vv if len(vv) <= 4 else rng.choice(vv, 4, replace=False)
        vecs.extend(sorted(pick))
        off.append(len(vecs))
    vecs = np.asarray(vecs)
    off = np.asarray(off, dtype=np.int32)
    ref = oracle_run(orc, b.H[chans], b.sym[vecs], off, wl.qam, wl.n_paths)
    sub = {k: gpu[k][vecs] for k in ("x", "l", "gamma")}
    st = compare(orc, b.H[chans], b.sym[vecs], off, wl.qam, sub, ref)
    print(wl.name, st)
    assert_parity(st)
    # properties at every vector: unit norm, |l| <= 1, gamma > 0
    assert np.allclose(np.linalg.norm(gpu["x"], axis=1), 1.0, atol=1e-5)
    assert np.all(np.abs(gpu["l"]) <= 1)
    assert np.all(gpu["gamma"] > 0)


def test_fp64_path_matches(orc):
    """Every channel through the FP64 fix-up (threshold 0) still matches the oracle."""
    b = W.make_batch(W.SLOT_16x16, subcarriers=24)
    wl = b.workload
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, fp64_threshold=0.0)
    assert np.all(gpu["status"] == vp.VP_CH_FP64)
    check_factor(orc, b.H, gpu, tol=1e-6)
    ref = oracle_run(orc, b.H, b.sym, b.vec_off, wl.qam, wl.n_paths)
    assert_parity(compare(orc, b.H, b.sym, b.vec_off, wl.qam, gpu, ref))


def test_edge_cases(orc):
    rng = W.rng_for(71, 0)
    # K = 1 (closed form), M > K, n not a multiple of 32, ragged per-channel vector counts
    for K, M, qam, n in [(1, 1, 16, 9), (1, 3, 256, 5), (5, 7, 64, 45), (6, 6, 16, 100)]:
        C = 7
        H = W.channels(rng, C, K, M)
        counts = rng.integers(0, 6, C)
        off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        sym = W.symbols(rng, int(off[-1]), K, qam)
        gpu = run_gpu(H, sym, off, qam, n)
        ref = oracle_run(orc, H, sym, off, qam, n)
        assert_parity(compare(orc, H, sym, off, qam, gpu, ref))
    # identity channel (exact ties everywhere), a singular channel, a NaN channel
    K = M = 4
    H = W.channels(rng, 4, K, M)
    H[0] = np.eye(4, dtype=np.complex64)
    H[1, 3] = H[1, 0]
    H[2, 1, 1] = np.nan
    sym = W.symbols(rng, 8, K, 16)
    off = W.vec_offsets_uniform(4, 2)
    gpu = run_gpu(H, sym, off, 16, 16)
    ref = oracle_run(orc, H, sym, off, 16, 16)
    assert gpu["status"][1] & vp.VP_CH_SINGULAR and gpu["status"][2] == vp.VP_CH_NONFINITE
    assert np.all(gpu["x"][2:6] == 0) and np.all(gpu["gamma"][2:6] == 0) and np.all(gpu["l"][2:6] == 0)
    keep = np.r_[0:2, 6:8]
    sub = {k: gpu[k][keep] for k in ("x", "l", "gamma")}
    refk = {k: ref[k][keep] for k in ("x", "l", "gamma")}
    st = compare(orc, H[[0, 3]], sym[keep], np.array([0, 2, 4], dtype=np.int32), 16, sub, refk)
    assert st["n_l_diff"] == 0 and st["x_err_max"] <= 1e-6, st


def test_empty_inputs(orc):
    """n_vec = 0 is a no-op that leaves the outputs untouched; channels with
    no vectors (every channel but one, and a ragged tail) give the oracle's
    results for the vectors that exist."""
    dev = torch.device("cuda:0")
    rng = W.rng_for(72, 0)
    K = M = 8
    C = 37                                   # 2 search tiles of channels plus a ragged tail
    H = W.channels(rng, C, K, M)
    x = torch.full((4, M), complex(7.0, 7.0), dtype=torch.complex64, device=dev)
    l = torch.full((4, K, 2), 99, dtype=torch.int8, device=dev)
    g = torch.full((4,), 5.0, dtype=torch.float32, device=dev)
    sym = torch.zeros((4, K), dtype=torch.uint8, device=dev)
    with vp.Plan(K, M, 64, 64) as plan:
        vp.vp_factorize(plan.handle, torch.from_numpy(H).to(dev), C)
        vp.vp_precode(plan.handle, sym, 0, torch.zeros(C + 1, dtype=torch.int32, device=dev), 0, x, l, g)
        vp.vp_precode(plan.handle, sym, 0, None, 0, x, l, g)
        with pytest.raises(vp.VPError) as e:           # S per channel must agree with n_vec
            vp.vp_precode(plan.handle, sym, 3, None, 0, x, l, g)
        assert e.value.code == 1
        torch.cuda.synchronize()
    assert torch.all(x == complex(7.0, 7.0)) and torch.all(l == 99) and torch.all(g == 5.0)
    for counts in (np.r_[np.zeros(C - 1, dtype=int), 3], np.r_[2, np.zeros(C - 2, dtype=int), 1]):
        off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        symn = W.symbols(rng, int(off[-1]), K, 64)
        gpu = run_gpu(H, symn, off, 64, 64)
        ref = oracle_run(orc, H, symn, off, 64, 64)
        st = compare(orc, H, symn, off, 64, gpu, ref)
        assert st["n_l_diff"] == 0, st
        assert_parity(st)


def test_host_buffer_slot_equals_device_path():
    b = W.make_batch(W.SLOT_16x16, subcarriers=64)
    wl = b.workload
    S = wl.symbols
    dev = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, want_factor=False, uniform_S=S)
    C, K, M = b.H.shape
    V = C * S
    Hh = torch.from_numpy(b.H).pin_memory()
    sh = torch.from_numpy(b.sym).pin_memory()
    xh = torch.empty((V, M), dtype=torch.complex64).pin_memory()
    lh = torch.empty((V, K, 2), dtype=torch.int8).pin_memory()
    gh = torch.empty((V,), dtype=torch.float32).pin_memory()
    with vp.Plan(K, M, wl.qam, wl.n_paths) as plan:
        vp.vp_run_slot_host(plan.handle, Hh, C, sh, S, xh, lh, gh)
        assert vp.vp_last_launch_count(plan.handle) == 4
    assert np.array_equal(xh.numpy(), dev["x"])
    assert np.array_equal(lh.numpy(), dev["l"])
    assert np.array_equal(gh.numpy().astype(np.float64), dev["gamma"])


@pytest.mark.parametrize("K,M,qam,n,S", [(16, 16, 16, 8, 14), (8, 8, 64, 16, 14), (4, 4, 16, 4, 7), (12, 16, 256, 1, 30),
                                         (2, 3, 64, 9, 2), (16, 16, 256, 16, 3)])
def test_small_budgets_several_vectors_per_warp(orc, K, M, qam, n, S):
    """Budgets of <= 16 paths run several data vectors per warp; against the
    oracle, and bit-equal to the same problems through the uneven-batch path
    (one vector per warp)."""
    rng = W.rng_for(130, K * 1000 + n * 10 + S)
    C = 40
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    off = W.vec_offsets_uniform(C, S)
    gpu = run_gpu(H, sym, off, qam, n, want_factor=False, uniform_S=S)
    ref = orc.precode_batch(H, sym, off, qam, n, nthreads=orc.max_threads())
    assert_parity(compare(orc, H, sym, off, qam, gpu, ref))
    dev = torch.device("cuda:0")
    probs = [W.Problem(K, M, qam, n, H[c], sym[c * S:(c + 1) * S]) for c in range(C)]
    pk = W.pack_problems(probs)
    Hd, sd = torch.from_numpy(pk.H).to(dev), torch.from_numpy(pk.sym).to(dev)
    x = torch.empty(pk.x_size, dtype=torch.complex64, device=dev)
    l = torch.empty(pk.l_size, dtype=torch.int8, device=dev)
    g = torch.empty(pk.g_size, dtype=torch.float32, device=dev)
    with vp.Batch(vp.packed_descs(pk, Hd, sd, x, l, g)) as bt:
        bt.launch()
        torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy().reshape(C * S, M), gpu["x"])
    assert np.array_equal(l.cpu().numpy().reshape(C * S, K, 2), gpu["l"])
    assert np.array_equal(g.cpu().numpy().astype(np.float64), gpu["gamma"])


def test_concurrent_plans_on_two_streams_equal_sequential():
    """Two plans launched on two streams at once give the same bits as the
    same calls one after another, and a repeated run gives the same bits."""
    dev = torch.device("cuda:0")
    runs = []
    for wl, sub in ((W.SLOT_16x16, 96), (W.RB_8x8, 12 * 20)):
        b = W.make_batch(wl, subcarriers=sub)
        C, K, M = b.H.shape
        V = b.sym.shape[0]
        runs.append((wl, b, torch.from_numpy(b.H).to(dev), torch.from_numpy(b.sym).to(dev),
                     torch.from_numpy(b.vec_off).to(dev), C, K, M, V))

    def outputs(streams):
        res = []
        plans = []
        for (wl, b, H, sym, off, C, K, M, V), st in zip(runs, streams):
            x = torch.empty((V, M), dtype=torch.complex64, device=dev)
            l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
            g = torch.empty((V,), dtype=torch.float32, device=dev)
            p = vp.Plan(K, M, wl.qam, wl.n_paths)
            plans.append(p)
            vp.vp_factorize(p.handle, H, C, stream=st)
            vp.vp_precode(p.handle, sym, 0, off, V, x, l, g, stream=st)
            res.append((x, l, g))
        torch.cuda.synchronize()
        out = [tuple(t.cpu().numpy() for t in r) for r in res]
        for p in plans:
            p.close()
        return out

    seq = outputs([None, None])
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    conc = outputs([s1, s2])
    again = outputs([s2, s1])
    for a, b, c in zip(seq, conc, again):
        for u, v, w in zip(a, b, c):
            assert np.array_equal(u, v) and np.array_equal(u, w)


@pytest.mark.parametrize("lam", [0.0, 0.3])
def test_maximum_path_budget_16x16(orc, lam):
    """n = VP_MAX_PATHS at the 16-level tile (32 chunks of 32 paths, shared
    prefixes), ragged vector counts per channel, with and without the K
    regularisation rows of P: the launch then reads the paths from global
    memory instead of staging them (four blocks per SM)."""
    K = M = 16
    n = vp.VP_MAX_PATHS
    rng = W.rng_for(73, int(lam * 10))
    C = 10
    H = W.channels(rng, C, K, M, "kron", 0.5, 0.2)
    counts = rng.integers(0, 5, C)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    sym = W.symbols(rng, int(off[-1]), K, 256)
    gpu = run_gpu(H, sym, off, 256, n, lam=lam)
    ref = orc.precode_batch(H, sym, off, 256, n, lam=lam, nthreads=orc.max_threads())
    assert np.array_equal(gpu["status"] & 3, ref["status"])
    assert_parity(compare(orc, H, sym, off, 256, gpu, ref, lam=lam))


def gpu_weights(U):
    """w_l = U_ll^2 as the FP32 factor forms it (the real diagonal squared in FP32)."""
    d = np.real(np.diagonal(U, axis1=1, axis2=2)).astype(np.float32)
    return (d * d).astype(np.float32)


@pytest.mark.parametrize("wl,sub", [(W.SMALL_4x4, None), (W.RB_8x8, 24 * 12 + 6), (W.SLOT_16x16, 200)])
def test_path_lists_bit_exact_on_gpu_weights(orc, wl, sub):
    """Path selection is integer work once the weights are fixed: on the GPU's
    own FP32 weights the oracle's MoP K-Best (Eq. mop, per-level children
    sorted by (metric, code)) must give the GPU's lists, in rank order, on
    every channel. Checked where both sides' metrics are exact sums: FP32
    channels (the FP64-flagged ones round w from FP64 and do not expose it)
    whose weights span less than 2^22, so every FP64 partial sum of
    w_l * (p_l - 1) is exact (24-bit weights, 3-bit digits, 16 terms) and the
    GPU's integer scaling keeps every weight."""
    b = W.make_batch(wl) if sub is None else W.make_batch(wl, subcarriers=sub)
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths)
    w = gpu_weights(gpu["U"])
    checked = 0
    for c in range(b.H.shape[0]):
        if gpu["status"][c] != 0:
            continue
        wc = w[c].astype(np.float64)
        if not np.all(wc > 0) or wc.max() / wc.min() >= 2.0 ** 22:
            continue
        codes, _ = orc.mop_kbest(wc, wl.n_paths)
        assert np.array_equal(gpu["codes"][c][:len(codes)], codes), c
        checked += 1
    print(wl.name, "channels checked", checked, "of", b.H.shape[0])
    assert checked >= 0.7 * b.H.shape[0]


def test_path_lists_bit_exact_full_slot(orc):
    """The same bit-exact check on 256 channels of the full 16x16 slot launch
    (the benchmark's configuration)."""
    b = W.make_batch(W.SLOT_16x16)
    wl = b.workload
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, uniform_S=wl.symbols)
    w = gpu_weights(gpu["U"])
    rng = np.random.default_rng(11)
    checked = 0
    for c in np.sort(rng.choice(b.H.shape[0], size=256, replace=False)):
        wc = w[c].astype(np.float64)
        if gpu["status"][c] != 0 or not np.all(wc > 0) or wc.max() / wc.min() >= 2.0 ** 22:
            continue
        codes, _ = orc.mop_kbest(wc, wl.n_paths)
        assert np.array_equal(gpu["codes"][c], codes), c
        checked += 1
    assert checked >= 150


def test_config1_against_the_exhaustive_minimum(orc):
    """4x4 16-QAM with 16 paths (n = 9^4 exceeds the 1024-path limit, so the
    GPU cannot search all perturbations itself): on 8 independent draws of the
    64-vector workload, the GPU's gamma is never below the brute-force minimum
    over all 9^4 bounded perturbations (oracle), equals the oracle's own
    16-path result, and reaches the minimum on most vectors (the paper's
    near-optimality claim for the most promising paths, Section III-A-2)."""
    w = W.SMALL_4x4
    tau = orc.default_tau(w.qam)
    ratios = []
    for slot in range(8):
        b = W.make_batch(w, slot=slot)
        gpu = run_gpu(b.H, b.sym, b.vec_off, w.qam, w.n_paths, want_factor=False, uniform_S=w.symbols)
        ref = oracle_run(orc, b.H, b.sym, b.vec_off, w.qam, w.n_paths)
        assert_parity(compare(orc, b.H, b.sym, b.vec_off, w.qam, gpu, ref))
        for c in range(b.H.shape[0]):
            f = orc.factor_channel(b.H[c].astype(np.complex128), 1)
            if f["status"] != 0:
                continue
            for v in range(b.vec_off[c], b.vec_off[c + 1]):
                vl = orc.qam_points(w.qam, b.sym[v])[f["user_of_level"]]
                g_bf, _ = orc.brute_min(f["Rt"], vl, tau)
                ratios.append(gpu["gamma"][v] / g_bf)
    r = np.asarray(ratios)
    print("vectors", r.size, "reach", float(np.mean(r <= 1 + 1e-5)), "mean", float(r.mean()))
    assert r.size >= 400
    assert np.all(r >= 1.0 - 1e-5)
    assert np.mean(r <= 1.0 + 1e-5) >= 0.9
