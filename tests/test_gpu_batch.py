"""Uneven batches (vp_batch_* / vp_precode_batch) through the C-ABI.

Problems of mixed K x M, QAM order, path budget and vector count run in one
grouped launch sequence; every problem is compared with the FP64 oracle
(small batch), with the plan path on the same problem (same kernels, so the
outputs must be identical), and on samples of a 20,000-problem batch. A CUDA
graph replay of vp_batch_launch on new inputs must equal a direct launch.
"""
import numpy as np
import pytest
import torch

import paper_2602_12098_gb300 as vp
from paper_2602_12098_gb300 import workloads as W
from vp_gpu_util import GAMMA_RTOL, L_MATCH_MIN, X_RTOL, compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vp.load()


class Packed:
    """Packed problems on the device with their output buffers and descriptors."""

    def __init__(self, problems, tau=0.0):
        dev = torch.device("cuda:0")
        self.problems = problems
        self.pk = W.pack_problems(problems)
        pk = self.pk
        self.H = torch.from_numpy(pk.H).to(dev)
        self.sym = torch.from_numpy(pk.sym).to(dev) if pk.sym.size else torch.zeros(16, dtype=torch.uint8, device=dev)
        self.x = torch.full((max(pk.x_size, 1),), complex(np.nan, np.nan), dtype=torch.complex64, device=dev)
        self.l = torch.full((max(pk.l_size, 1),), 99, dtype=torch.int8, device=dev)
        self.g = torch.full((max(pk.g_size, 1),), np.nan, dtype=torch.float32, device=dev)
        self.st = torch.full((len(problems),), 255, dtype=torch.uint8, device=dev)
        self.descs = vp.packed_descs(pk, self.H, self.sym, self.x, self.l, self.g, self.st, tau=tau)

    def outputs(self, i):
        pk = self.pk
        S, K, M = int(pk.S[i]), int(pk.K[i]), int(pk.M[i])
        x = self.x_np[pk.x_off[i]:pk.x_off[i] + S * M].reshape(S, M)
        l = self.l_np[pk.l_off[i]:pk.l_off[i] + S * K * 2].reshape(S, K, 2)
        g = self.g_np[pk.g_off[i]:pk.g_off[i] + S].astype(np.float64)
        return {"x": x, "l": l, "gamma": g, "status": self.st_np[i:i + 1]}

    def fetch(self):
        torch.cuda.synchronize()
        self.x_np = self.x.cpu().numpy()
        self.l_np = self.l.cpu().numpy()
        self.g_np = self.g.cpu().numpy()
        self.st_np = self.st.cpu().numpy()


def mixed_problems(n, seed, s_max=14):
    rng = W.rng_for(80, seed)
    probs = W.uneven_problems(n, seed_offset=80 + seed)
    out = []
    for p in probs:
        S = int(rng.integers(0, s_max + 1))
        out.append(W.Problem(p.K, p.M, p.qam, p.n_paths, p.H, p.sym[:S].copy()))
    # small tiles (K <= 2) and K = 1, square and wide
    for K, M, qam, n in [(1, 1, 16, 9), (2, 2, 64, 81), (2, 5, 4, 40), (6, 6, 16, 100)]:
        out.append(W.Problem(K, M, qam, n, W.channels(rng, 1, K, M)[0], W.symbols(rng, 5, K, qam)))
    return out


def aggregate(orc, pkd, idx):
    tot = {"V": 0, "n_l_diff": 0, "gamma_rel_max": 0.0, "x_err_max": 0.0, "tie_gamma_rel_max": 0.0,
           "tie_x_err_max": 0.0}
    for i in idx:
        p = pkd.problems[i]
        S = p.sym.shape[0]
        off = np.array([0, S], dtype=np.int32)
        gpu = pkd.outputs(i)
        ref = orc.precode_batch(p.H[None].astype(np.complex64), p.sym, off, p.qam, p.n_paths, nthreads=1)
        assert (gpu["status"][0] & 3) == ref["status"][0]
        st = compare(orc, p.H[None], p.sym, off, p.qam, gpu, ref)
        tot["V"] += st["V"]
        tot["n_l_diff"] += st["n_l_diff"]
        for k in ("gamma_rel_max", "x_err_max", "tie_gamma_rel_max", "tie_x_err_max"):
            tot[k] = max(tot[k], st[k])
    tot["l_match"] = 1.0 - tot["n_l_diff"] / max(tot["V"], 1)
    return tot


def assert_agg(tot):
    assert tot["l_match"] >= L_MATCH_MIN, tot
    for k, tol in (("gamma_rel_max", GAMMA_RTOL), ("x_err_max", X_RTOL), ("tie_gamma_rel_max", GAMMA_RTOL),
                   ("tie_x_err_max", X_RTOL)):
        assert tot[k] <= tol, tot


def test_mixed_batch_vs_oracle_and_plan_path(orc):
    probs = mixed_problems(60, 1)
    # a non-finite channel and a rank-deficient one
    bad = W.Problem(4, 8, 16, 16, W.channels(W.rng_for(81, 0), 1, 4, 8)[0], W.symbols(W.rng_for(81, 1), 3, 4, 16))
    bad.H[1, 2] = np.inf
    sing = W.Problem(4, 4, 16, 16, W.channels(W.rng_for(81, 2), 1, 4, 4)[0], W.symbols(W.rng_for(81, 3), 3, 4, 16))
    sing.H[3] = sing.H[0]
    probs += [bad, sing]
    pkd = Packed(probs)
    with vp.Batch(pkd.descs) as b:
        b.launch()
        pkd.fetch()
    nb, ns = len(probs) - 2, len(probs) - 1
    assert pkd.st_np[nb] == vp.VP_CH_NONFINITE and pkd.st_np[ns] & vp.VP_CH_SINGULAR
    for i in (nb, ns):
        o = pkd.outputs(i)
        assert np.all(o["x"] == 0) and np.all(o["l"] == 0) and np.all(o["gamma"] == 0)
    tot = aggregate(orc, pkd, range(nb))
    print(tot)
    assert_agg(tot)
    # the plan path on each problem gives the same bits
    for i in range(nb):
        p = probs[i]
        S = p.sym.shape[0]
        if S == 0:
            continue
        ref = run_gpu(p.H[None], p.sym, np.array([0, S], dtype=np.int32), p.qam, p.n_paths, want_factor=False,
                      uniform_S=S)
        o = pkd.outputs(i)
        assert np.array_equal(o["x"], ref["x"]) and np.array_equal(o["l"], ref["l"]), i
        assert np.array_equal(o["gamma"], ref["gamma"]) and o["status"][0] == ref["status"][0], i


def test_one_shot_entry_point_equals_handle():
    probs = mixed_problems(24, 2)
    a, c = Packed(probs), Packed(probs)
    nbytes = vp.vp_precode_batch_workspace_bytes(a.descs)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    vp.vp_precode_batch(a.descs, base, nbytes)
    a.fetch()
    with vp.Batch(c.descs) as b:
        b.launch()
        c.fetch()
    assert np.array_equal(a.x_np, c.x_np) and np.array_equal(a.l_np, c.l_np)
    assert np.array_equal(a.g_np, c.g_np) and np.array_equal(a.st_np, c.st_np)


def test_full_size_uneven_batch_sampled(orc):
    """20,000 problems x 14 vectors of mixed shape; oracle on sampled problems."""
    probs = W.uneven_problems(20000)
    pkd = Packed(probs)
    with vp.Batch(pkd.descs) as b:
        b.launch()
        pkd.fetch()
    rng = np.random.default_rng(9)
    tot = aggregate(orc, pkd, sorted(rng.choice(len(probs), 40, replace=False)))
    print(tot)
    assert_agg(tot)
    assert np.all((pkd.st_np & 3) == 0)
    assert np.all(np.abs(pkd.l_np) <= 1) and np.all(pkd.g_np > 0)
    for i in rng.choice(len(probs), 500, replace=False):
        assert np.allclose(np.linalg.norm(pkd.outputs(i)["x"], axis=1), 1.0, atol=1e-5)


def test_graph_replay_on_new_inputs_equals_direct_launch():
    probs = mixed_problems(40, 3)
    pkd = Packed(probs)
    stream = torch.cuda.Stream()
    with vp.Batch(pkd.descs, stream=stream) as b:
        with torch.cuda.stream(stream):
            b.launch(stream)                       # first launch outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            b.launch(stream)
        # new inputs in the same buffers, then replay
        probs2 = mixed_problems(40, 4)
        for p, q in zip(probs, probs2):
            q.K, q.M, q.qam, q.n_paths = p.K, p.M, p.qam, p.n_paths
            q.H = W.channels(W.rng_for(82, len(q.sym)), 1, p.K, p.M)[0]
            q.sym = W.symbols(W.rng_for(83, p.K), p.sym.shape[0], p.K, p.qam)
        pk2 = W.pack_problems(probs2)
        pkd.H.copy_(torch.from_numpy(pk2.H))
        if pk2.sym.size:
            pkd.sym[:pk2.sym.size].copy_(torch.from_numpy(pk2.sym))
        g.replay()
        pkd.fetch()
        replay = (pkd.x_np.copy(), pkd.l_np.copy(), pkd.g_np.copy())
        with torch.cuda.stream(stream):
            b.launch(stream)
        pkd.fetch()
    assert np.array_equal(replay[0], pkd.x_np) and np.array_equal(replay[1], pkd.l_np)
    assert np.array_equal(replay[2], pkd.g_np)


def test_autotuned_launch_equals_default_and_cache_roundtrip(tmp_path):
    """The tuned mapping changes no output; a second batch of the same shape
    takes its knobs from the JSON cache."""
    probs = mixed_problems(60, 5)
    a, t = Packed(probs), Packed(probs)
    with vp.Batch(a.descs) as b:
        b.launch()
        a.fetch()
    cache = str(tmp_path / "tune.json")
    with vp.Batch(t.descs) as b:
        knobs = b.autotune(reps=2, cache=cache)
        assert len(knobs) == len(vp.vp_batch_group_info(b.handle))
        b.launch()
        t.fetch()
    assert np.array_equal(a.x_np, t.x_np) and np.array_equal(a.l_np, t.l_np)
    assert np.array_equal(a.g_np, t.g_np) and np.array_equal(a.st_np, t.st_np)
    import json
    table = json.load(open(cache))
    assert list(table.values()) == [knobs]
    c = Packed(probs)
    with vp.Batch(c.descs) as b:
        assert b.autotune(reps=2, cache=cache) == knobs
        assert vp.vp_batch_get_tuning(b.handle) == knobs
        # every explicit setting gives the same outputs too
        stages = [g[0] for g in vp.vp_batch_group_info(b.handle)]
        vp.vp_batch_set_tuning(b.handle, [0 if s == 0 else (256 if s == 1 else 3) for s in stages])
        b.launch()
        c.fetch()
    assert np.array_equal(a.x_np, c.x_np) and np.array_equal(a.l_np, c.l_np) and np.array_equal(a.g_np, c.g_np)


def test_persistent_search_equals_grouped_launches():
    """The search in one persistent launch (heaviest first over all K tiles)
    gives the same outputs, bit for bit, as one launch per K tile (the
    default), under every mapping of the persistent launch: warps per block,
    resident blocks per SM, and the 16-level tile's path codes staged in
    shared memory or read in place."""
    probs = mixed_problems(120, 9)
    ref = Packed(probs)
    with vp.Batch(ref.descs) as b:
        assert vp.vp_batch_launch_count(b.handle) > 10
        b.launch()
        ref.fetch()
    for knob in (0, 7 | (1 << 3), 6 | (2 << 3) | (1 << 6), 5 | (3 << 3) | (2 << 6)):
        got = Packed(probs)
        with vp.Batch(got.descs, persistent=1) as b:
            stages = [g[0] for g in vp.vp_batch_group_info(b.handle)]
            vp.vp_batch_set_tuning(b.handle, [knob if st == 3 else 0 for st in stages])
            b.launch()
            got.fetch()
        assert np.array_equal(ref.x_np, got.x_np) and np.array_equal(ref.l_np, got.l_np)
        assert np.array_equal(ref.g_np, got.g_np) and np.array_equal(ref.st_np, got.st_np)


def test_concurrent_stages_equal_in_order_launches():
    """The launches of a stage run side by side by default (the batch's side
    streams); the outputs equal those of the in-order launches on one stream,
    directly and through a CUDA graph capture."""
    probs = mixed_problems(60, 5)
    outs = []
    for conc in (0, 1):
        pkd = Packed(probs)
        stream = torch.cuda.Stream()
        with vp.Batch(pkd.descs, stream=stream, concurrent=conc) as b:
            with torch.cuda.stream(stream):
                b.launch(stream)
            torch.cuda.synchronize()
            outs.append([t.cpu().numpy().copy() for t in (pkd.x, pkd.l, pkd.g)])
            if conc:
                for t in (pkd.x, pkd.l, pkd.g):
                    t.zero_()
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    b.launch(stream)
                g.replay()
                torch.cuda.synchronize()
                outs.append([t.cpu().numpy().copy() for t in (pkd.x, pkd.l, pkd.g)])
    for other in outs[1:]:
        for a, c in zip(outs[0], other):
            assert np.array_equal(a, c, equal_nan=a.dtype.kind in "fc")
