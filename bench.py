#!/usr/bin/env python3
"""Benchmark of the VP precoder on GB300: precoded vectors/s on one 100 MHz slot.

Workload (one "step" = one slot through the whole hot path): 3276 subcarriers
x 14 OFDM symbols = 45,864 data vectors, K = M = 16, 256-QAM, 256 candidate
paths, Kronecker-correlated Rayleigh channels (rho_ap = 0.5, rho_u = 0.2),
one channel per subcarrier. A step runs vp_factorize (sorted RQ + FP64 fix-up
+ MoP path selection for all 3276 channels) and vp_precode (search + x for
all vectors). Inputs are resident in HBM when a step starts; L2 is flushed
between steps (a 256 MiB device write outside the timed events).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU runs are independent replicas (one slot per rank, no collective on
the data path); value is the vectors of all ranks / the slowest rank's time.
The "reference" arm times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VP-precoded vectors/s (16x16 256-QAM) + p99 slot latency, batched vs plain"
UNIT = "vectors/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", default="slot_16x16")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--subcarriers", type=int, default=None,
                    help="run a reduced slot (profiling captures); the default is the full slot")
    ap.add_argument("--paths", type=int, default=None,
                    help="candidate paths per vector instead of the workload's (the default is its own)")
    ap.add_argument("--no-batched", action="store_true", help="skip the uneven batched-vs-plain measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the Poisson serving measurement")
    ap.add_argument("--serving-slots", type=int, default=2000)
    ap.add_argument("--serving-paths", type=int, nargs="+", default=[64, 256])
    ap.add_argument("--serving-lanes", type=int, default=8)
    ap.add_argument("--serving-pool-mib", type=int, default=1024)
    return ap.parse_args()


def paper_work_flops(K: int, M: int, n: int) -> float:
    """FP32 flops of one precoded vector from the paper's per-vector count of
    complex multiplications N_r N_t + N_t^2 + n N_t (1 + (N_t + 1) / 2)
    (Section III-B, with N_t -> K for the tree size), 8 flops (4 FMA) each."""
    cmul = K * M + K * K + n * K * (1 + (K + 1) / 2)
    return 8.0 * cmul


def executed_cmul(codes, K: int, M: int, n: int) -> float:
    """Complex multiplications per vector in the paper's unit (level l of K,
    1-based from the bottom, costs 1 + l), counting the top T shared levels
    once per distinct prefix as the search runs them. T per channel is path
    selection's rule: the largest T <= 3 whose distinct top-T-level prefixes
    number <= 32, when K fills its search tile (2, 4, 8, 12 or 16), K >= 8 and
    n > 32; else 0. codes: uint64 [C][n] path digits (4 bits per level)."""
    import numpy as np
    codes = np.asarray(codes, dtype=np.uint64)
    C = codes.shape[0]
    tile = 2 if K <= 2 else 4 if K <= 4 else 8 if K <= 8 else 12 if K <= 12 else 16
    lvl = lambda l: 1 + l
    total = 0.0
    for c in range(C):
        T, npf = 0, n
        if K == tile and K >= 8 and n > 32:
            for t in (3, 2, 1):
                npre = len(np.unique(codes[c] >> np.uint64(4 * (K - t))))
                if npre <= 32:
                    T, npf = t, npre
                    break
        shared = sum(lvl(l) for l in range(K - T + 1, K + 1))
        rest = sum(lvl(l) for l in range(1, K - T + 1))
        total += npf * shared + n * rest
    return K * M + K * K + total / max(C, 1)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"samples": 0, "note": "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return {"samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_batch(w, rank: int, subcarriers=None):
    """Rank r precodes its own slot (an independent seeded draw): replicas
    share nothing, so no collective touches the data path."""
    from paper_2602_12098_gb300 import workloads as W
    return W.make_batch(w, slot=rank, subcarriers=subcarriers)


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest of the ranks' values (the slowest rank's time)."""
    if dist is None or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: int, steps: int, slowest_s: float) -> float:
    """Units all ranks processed / the slowest rank's time (weak scaling)."""
    return ws * units_per_rank * steps / slowest_s


def run_reference(args):
    """FP64 CPU oracle on the host cores, bounded sample per step (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2602_12098_gb300 import workloads as W
    w = W.WORKLOADS[args.workload]
    if args.paths is not None:
        import dataclasses
        w = dataclasses.replace(w, n_paths=args.paths)
    threads = os.cpu_count() or 1
    O.build()
    # calibrate: how many channels fit a per-step budget so K + W steps take ~2 minutes
    cal = W.make_batch(w, subcarriers=8)
    t0 = time.perf_counter()
    O.precode_batch(cal.H, cal.sym, cal.vec_off, w.qam, w.n_paths, nthreads=threads)
    rate = cal.sym.shape[0] / max(time.perf_counter() - t0, 1e-6)      # vectors/s
    per_step_s = max(0.05, 120.0 / max(1, args.steps + args.warmup))
    sub = int(max(threads, min(w.subcarriers, per_step_s * rate / w.symbols)))
    b = W.make_batch(w, subcarriers=sub)
    V = b.sym.shape[0]
    for _ in range(args.warmup):
        O.precode_batch(b.H, b.sym, b.vec_off, w.qam, w.n_paths, nthreads=threads)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.precode_batch(b.H, b.sym, b.vec_off, w.qam, w.n_paths, nthreads=threads)
        ts.append(time.perf_counter() - t0)
    tot = sum(ts)
    value = V * args.steps / tot
    cores = min(threads, O.max_threads()) if O.max_threads() > 1 else 1
    sample = f"first {sub} of {w.subcarriers} subcarriers x {w.symbols} symbols ({V} vectors) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "K": w.K, "M": w.M, "qam": w.qam,
                                             "n_paths": w.n_paths, "vectors_per_step": V},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def oracle_configs(configs_sample: dict, threads: int) -> dict:
    """Oracle leg for the C1 / C2 lines: the FP64 oracle on each config's
    slot (all host cores and one core), its agreement with the GPU outputs
    on every vector, and for C1 how often the 16-path search reaches the
    exhaustive minimum over all 9^4 bounded perturbations (oracle brute
    force on every vector of every draw)."""
    import numpy as np

    from oracle import oracle as O
    out = {}
    for tag, res in configs_sample.items():
        b, x, l, g = res[0]
        w = b.workload
        t0 = time.perf_counter()
        ref = O.precode_batch(b.H, b.sym, b.vec_off, w.qam, w.n_paths, nthreads=threads)
        dt = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.precode_batch(b.H, b.sym, b.vec_off, w.qam, w.n_paths, nthreads=1)
        dt1 = time.perf_counter() - t0
        V = b.sym.shape[0]
        leq = np.all(l == ref["l"], axis=(1, 2))
        m = leq & (ref["gamma"] > 0)
        rec = {"oracle_vectors_per_s": V / dt, "oracle_one_core_vectors_per_s": V / dt1,
               "vectors_compared": int(V), "l_match": float(leq.mean()),
               "gamma_rel_max": float(np.max(np.abs(g[m] - ref["gamma"][m]) / ref["gamma"][m])),
               "x_err_max": float(np.max(np.linalg.norm(x[m] - ref["x"][m], axis=1)))}
        if tag == "C1":
            tau = O.default_tau(w.qam)
            ratios = []
            for bb, xx, ll, gg in res:
                for c in range(bb.H.shape[0]):
                    f = O.factor_channel(bb.H[c].astype(np.complex128), 1)
                    if f["status"] != 0:
                        continue
                    for v in range(bb.vec_off[c], bb.vec_off[c + 1]):
                        vl = O.qam_points(w.qam, bb.sym[v])[f["user_of_level"]]
                        g_bf, _ = O.brute_min(f["Rt"], vl, tau)
                        ratios.append(gg[v] / g_bf)
            r = np.asarray(ratios)
            rec["exhaustive"] = {"vectors": int(r.size), "draws": len(res),
                                 "reach_frac": float(np.mean(r <= 1.0 + 1e-5)),
                                 "gamma_over_min_mean": float(r.mean()), "gamma_over_min_p99": float(np.percentile(r, 99)),
                                 "gamma_over_min_max": float(r.max()),
                                 "basis": "GPU gamma (16 paths) over the oracle's brute-force minimum over all 9^4 "
                                          "perturbations with entries in {-1,0,1}+j{-1,0,1}; reached = within 1e-5"}
        out[tag] = rec
    return out


def cpu_baseline(w, budget_s: float = 10.0, gpu_sample=None, configs_sample=None, budget_gammas=None) -> dict:
    """The oracle on whole slots of the workload (independent draws) until
    about budget_s seconds of wall time have been spent, all host cores; then
    on one core, on the leading channels of one slot, doubled until one run
    takes budget_s / 8 seconds. gpu_sample = (batch, x, l,
    gamma) of the timed GPU slot: the oracle recomputes 24 of its channels and
    the line reports the agreement."""
    import numpy as np

    from oracle import oracle as O
    from paper_2602_12098_gb300 import workloads as W
    threads = os.cpu_count() or 1
    O.build()
    parity = None
    if gpu_sample is not None:
        b, x, l, g = gpu_sample
        rng = np.random.default_rng(5)
        C = b.H.shape[0]
        chans = np.sort(rng.choice(C, min(24, C), replace=False))
        vecs = np.concatenate([np.arange(b.vec_off[c], b.vec_off[c + 1]) for c in chans])
        off = np.concatenate([[0], np.cumsum(np.diff(b.vec_off)[chans])]).astype(np.int32)
        ref = O.precode_batch(b.H[chans], b.sym[vecs], off, w.qam, w.n_paths, nthreads=threads)
        leq = np.all(l[vecs] == ref["l"], axis=(1, 2))
        m = leq & (ref["gamma"] > 0)
        parity = {"channels": int(len(chans)), "vectors": int(len(vecs)), "l_match": float(leq.mean()),
                  "gamma_rel_max": float(np.max(np.abs(g[vecs][m] - ref["gamma"][m]) / ref["gamma"][m])),
                  "x_err_max": float(np.max(np.linalg.norm(x[vecs][m] - ref["x"][m], axis=1))),
                  "note": "where l matches; the GPU parity tests treat l differences (near-ties)"}
        # the exact bounded-alphabet minimum (depth-first sphere encoder) on 4 vectors of each channel
        tau = O.default_tau(w.qam)
        ratios, vs, gmins = [], [], []
        for c in chans:
            f = O.factor_channel(b.H[c].astype(np.complex128), 1)
            if f["status"] != 0:
                continue
            for v in range(b.vec_off[c], min(b.vec_off[c + 1], b.vec_off[c] + 4)):
                vl = O.qam_points(w.qam, b.sym[v])[f["user_of_level"]]
                g_min, _ = O.sphere_min(f["Rt"], vl, tau)
                ratios.append(g[v] / g_min)
                vs.append(v)
                gmins.append(g_min)
        r = np.asarray(ratios)
        if budget_gammas and vs:
            gm = np.asarray(gmins)
            parity["exact_minimum_by_paths"] = {
                str(n): {"reach_frac": float(np.mean(gg[vs] / gm <= 1.0 + 1e-5)),
                         "gamma_over_min_mean": float(np.mean(gg[vs] / gm)),
                         "gamma_over_min_max": float(np.max(gg[vs] / gm))}
                for n, gg in sorted(budget_gammas.items())}
        if r.size:
            parity["exact_minimum"] = {
                "vectors": int(r.size), "reach_frac": float(np.mean(r <= 1.0 + 1e-5)),
                "gamma_over_min_mean": float(r.mean()), "gamma_over_min_p99": float(np.percentile(r, 99)),
                "gamma_over_min_max": float(r.max()),
                "basis": f"GPU gamma ({w.n_paths} paths) over the oracle's sphere-encoder minimum over all "
                         "perturbations with entries in {-1,0,1}+j{-1,0,1}; reached = within 1e-5"}
    V = 0
    dt = 0.0
    slots = 0
    while dt < budget_s and slots < 50:
        b = W.make_batch(w, slot=100 + slots)
        t0 = time.perf_counter()
        O.precode_batch(b.H, b.sym, b.vec_off, w.qam, w.n_paths, nthreads=threads)
        dt += time.perf_counter() - t0
        V += b.sym.shape[0]
        slots += 1
    cores = min(threads, O.max_threads()) if O.max_threads() > 1 else 1
    # one core: leading channels of one slot, grown until ~budget_s / 4
    sub_c, dt1, V1 = 8, 0.0, 0
    while dt1 < budget_s / 8 and sub_c <= w.subcarriers:
        b1 = W.make_batch(w, slot=100, subcarriers=sub_c)
        t0 = time.perf_counter()
        O.precode_batch(b1.H, b1.sym, b1.vec_off, w.qam, w.n_paths, nthreads=1)
        dt1 = time.perf_counter() - t0
        V1 = b1.sym.shape[0]
        sub_c *= 2
    out = {"value": V / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{slots} whole slot(s) of {w.subcarriers} subcarriers x {w.symbols} symbols ({V} vectors), "
                     f"{dt:.1f} s wall",
           "one_core": {"value": V1 / dt1, "unit": UNIT, "sample": f"{V1} vectors, {dt1:.1f} s"}}
    if parity is not None:
        out["parity_sample"] = parity
    if configs_sample:
        out["configs"] = oracle_configs(configs_sample, threads)
    return out


def code_fingerprint(files) -> str:
    """sha256 of C/CUDA sources with comments and whitespace removed, so that
    an edit of comments or layout alone keeps a profile of the kernel valid
    (string literals in these sources hold no comment markers)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        src = open(os.path.join(ROOT, f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
        h.update(b"\0")
    return h.hexdigest()


def profiled_traffic(kernel_file: str) -> dict | None:
    """DRAM bytes per launch from a committed ncu summary, if the kernel's
    sources still have the code fingerprint that was profiled (else None:
    stale counters)."""
    path = os.path.join(ROOT, "profiles", kernel_file)
    try:
        txt = open(path).read()
    except OSError:
        return None
    fields = {}
    for ln in txt.splitlines():
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    srcs = fields.get("sources", "").split()
    try:
        fp = code_fingerprint(srcs)
    except OSError:
        return None
    if not srcs or fp != fields.get("sources_code_sha256"):
        return None
    try:
        out = {"bytes": float(fields["dram_bytes_per_launch"]), "file": "profiles/" + kernel_file}
    except (KeyError, ValueError):
        return None
    try:
        out["warp_instructions"] = float(fields["warp_instructions_per_launch"])
    except (KeyError, ValueError):
        pass
    return out


def measure_batched(dev, flush, symbols_per_problem: int = 14) -> dict:
    """Uneven batch: 20,000 problems x 14 vectors, (K x M, Q, n) uniform over
    {4x8, 8x16, 12x16, 16x16} x {16, 64, 256} x {16, 64, 256, 1024}. The
    search as one launch per K tile with each stage's launches side by side
    (the default; also captured in a CUDA graph and autotuned), the same
    launches in order on one stream, the search in one persistent launch
    (direct and autotuned), and the plain path (one vp_factorize +
    vp_precode per problem, one plan per distinct shape)."""
    import numpy as np
    import torch

    import paper_2602_12098_gb300 as vp
    from paper_2602_12098_gb300 import workloads as W
    stream = torch.cuda.Stream(device=dev)      # graph capture needs a non-default stream
    probs = W.uneven_problems(20000, symbols_per_problem=symbols_per_problem)
    pk = W.pack_problems(probs)
    V = int(pk.S.sum())
    H = torch.from_numpy(pk.H).to(dev)
    sym = torch.from_numpy(pk.sym).to(dev)
    x = torch.empty(pk.x_size, dtype=torch.complex64, device=dev)
    l = torch.empty(pk.l_size, dtype=torch.int8, device=dev)
    g = torch.empty(pk.g_size, dtype=torch.float32, device=dev)
    descs = vp.packed_descs(pk, H, sym, x, l, g)
    out = {"workload": f"20000 problems x {symbols_per_problem} vector(s), (K x M, Q, n) uniform over "
                       "{4x8, 8x16, 12x16, 16x16} x {16, 64, 256} x {16, 64, 256, 1024}, iid channels", "vectors": V}

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    torch.cuda.synchronize()
    # the search in one persistent launch, heaviest first over all K tiles
    with vp.Batch(descs, stream=stream, persistent=1) as b:
        for _ in range(3):
            b.launch(stream)
        torch.cuda.synchronize()
        ms = timed(lambda: b.launch(stream), 10)
        out["persistent_ms"] = ms
        out["persistent_vectors_per_s"] = V / (ms / 1e3)
        out["persistent_launches"] = b.launches
        out["persistent_tuned_knob"] = b.autotune(reps=3, cache="", stream=stream)[-1]
        ms = timed(lambda: b.launch(stream), 10)
        out["persistent_tuned_ms"] = ms
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            b.launch(stream)

        def replay_p():
            with torch.cuda.stream(stream):
                graph.replay()

        for _ in range(3):
            replay_p()
        out["persistent_graph_ms"] = timed(replay_p, 10)
        del graph
    # every launch in order on one stream (the stages' groups not side by side)
    with vp.Batch(descs, stream=stream, concurrent=0) as b:
        for _ in range(3):
            b.launch(stream)
        torch.cuda.synchronize()
        ms = timed(lambda: b.launch(stream), 10)
        out["in_order_ms"] = ms
        out["in_order_vectors_per_s"] = V / (ms / 1e3)
    # the search as one launch per K tile and each stage's launches side by
    # side on the batch's streams (the default); direct, in a CUDA graph, and
    # autotuned
    with vp.Batch(descs, stream=stream) as b:
        for _ in range(3):
            b.launch(stream)
        torch.cuda.synchronize()
        ms = timed(lambda: b.launch(stream), 10)
        out["batched_ms"] = ms
        out["batched_vectors_per_s"] = V / (ms / 1e3)
        out["batched_launches"] = b.launches
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            b.launch(stream)
        def replay():
            with torch.cuda.stream(stream):
                graph.replay()

        for _ in range(3):
            replay()
        ms = timed(replay, 10)
        out["graph_ms"] = ms
        out["graph_vectors_per_s"] = V / (ms / 1e3)
        del graph
        # the project's autotuner (vp_batch_autotune): per-group mapping knobs,
        # same outputs; against one generic mapping (two warps per channel's
        # path lists, four warps per search block) and the built-in choices
        stages = [gi[0] for gi in vp.vp_batch_group_info(b.handle)]
        vp.vp_batch_set_tuning(b.handle, [64 if st == 1 else (4 if st == 2 else 0) for st in stages])
        ms = timed(lambda: b.launch(stream), 10)
        out["generic_mapping_ms"] = ms
        vp.vp_batch_set_tuning(b.handle, [0] * len(stages))
        out["tuned_knobs"] = b.autotune(reps=3, cache="", stream=stream)
        for _ in range(3):
            b.launch(stream)
        ms = timed(lambda: b.launch(stream), 10)
        out["tuned_ms"] = ms
        out["tuned_vectors_per_s"] = V / (ms / 1e3)

    plans = {}
    for i in range(len(probs)):
        key = (int(pk.K[i]), int(pk.M[i]), int(pk.qam[i]), int(pk.n_paths[i]))
        if key not in plans:
            plans[key] = vp.Plan(*key)
    hb, sb, xb, lb, gb = H.data_ptr(), sym.data_ptr(), x.data_ptr(), l.data_ptr(), g.data_ptr()
    calls = []
    for i in range(len(probs)):
        key = (int(pk.K[i]), int(pk.M[i]), int(pk.qam[i]), int(pk.n_paths[i]))
        S = int(pk.S[i])
        calls.append((plans[key].handle, hb + 8 * int(pk.H_off[i]), sb + int(pk.sym_off[i]), S,
                      xb + 8 * int(pk.x_off[i]), lb + int(pk.l_off[i]), gb + 4 * int(pk.g_off[i])))
    lib = vp.load()
    sh = stream.cuda_stream

    def plain():
        for h, hp, sp, S, xp, lp, gp in calls:
            if lib.vp_factorize(h, hp, 1, None, None, None, None, sh) != 0:
                raise RuntimeError("vp_factorize failed")
            if lib.vp_precode(h, sp, S, None, S, xp, lp, gp, sh) != 0:
                raise RuntimeError("vp_precode failed")

    plain()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ms = timed(plain, 2)
    out["plain_ms"] = ms
    out["plain_vectors_per_s"] = V / (ms / 1e3)
    out["plain_launches"] = 4 * len(probs)
    out["plain_host_s"] = (time.perf_counter() - t0) / 2
    for p in plans.values():
        p.close()
    return out


def measure_lut(dev, b, w, flush, steps: int) -> dict:
    """The same slot with the region-LUT DEMAP (VP_DEMAP_LUT): vp_precode time
    and the gamma it reaches against the exact ranking (same paths)."""
    import numpy as np
    import torch

    import paper_2602_12098_gb300 as vp
    C, K, M = b.H.shape
    V, S = b.sym.shape[0], w.symbols
    stream = torch.cuda.current_stream()
    H = torch.from_numpy(b.H).to(dev)
    sym = torch.from_numpy(b.sym).to(dev)
    out = {}
    g = {}
    for name, mode in (("exact", vp.VP_DEMAP_EXACT), ("lut", vp.VP_DEMAP_LUT)):
        x = torch.empty((V, M), dtype=torch.complex64, device=dev)
        l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
        gam = torch.empty((V,), dtype=torch.float32, device=dev)
        with vp.Plan(K, M, w.qam, w.n_paths, demap=mode) as plan:
            vp.vp_factorize(plan.handle, H, C, stream=stream)
            for _ in range(3):
                vp.vp_precode(plan.handle, sym, S, None, V, x, l, gam, stream=stream)
            ts = []
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vp.vp_precode(plan.handle, sym, S, None, V, x, l, gam, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
        out[name + "_precode_ms"] = statistics.median(ts)
        g[name] = gam.cpu().numpy().astype(np.float64)
    m = g["exact"] > 0
    r = g["lut"][m] / g["exact"][m]
    out["search_speedup"] = out["exact_precode_ms"] / out["lut_precode_ms"]
    out["gamma_ratio_mean"] = float(r.mean())
    out["gamma_ratio_p99"] = float(np.percentile(r, 99))
    out["note"] = "VP_DEMAP_LUT (region lookup, Section III-A-2) vs the exact ranking on the same slot and paths"
    return out


def measure_fixed(dev, b, w, flush, steps: int, fracs=(8, 9, 10, 11, 12, 13)) -> dict:
    """The word-length study (Section IV: 16-bit words, 8..13 fractional
    bits): the same slot and factor with the fixed-point search; per F the
    vp_precode time, the gamma it reaches against the floating-point search
    and the share of vectors whose l differs from it."""
    import numpy as np
    import torch

    import paper_2602_12098_gb300 as vp
    C, K, M = b.H.shape
    V, S = b.sym.shape[0], w.symbols
    stream = torch.cuda.current_stream()
    H = torch.from_numpy(b.H).to(dev)
    sym = torch.from_numpy(b.sym).to(dev)
    x = torch.empty((V, M), dtype=torch.complex64, device=dev)
    l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
    gam = torch.empty((V,), dtype=torch.float32, device=dev)
    res = {}
    with vp.Plan(K, M, w.qam, w.n_paths) as plan:
        vp.vp_factorize(plan.handle, H, C, stream=stream)
        for f in (0,) + tuple(fracs):
            vp.vp_plan_set_fixed_point(plan.handle, f)
            for _ in range(3):
                vp.vp_precode(plan.handle, sym, S, None, V, x, l, gam, stream=stream)
            ts = []
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vp.vp_precode(plan.handle, sym, S, None, V, x, l, gam, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            res[f] = (statistics.median(ts), gam.cpu().numpy().astype(np.float64), l.cpu().numpy())
    g0, l0 = res[0][1], res[0][2]
    m = g0 > 0
    out = {"float_precode_ms": res[0][0], "by_frac_bits": {}}
    for f in fracs:
        ms, g, lf = res[f]
        r = g[m] / g0[m]
        out["by_frac_bits"][str(f)] = {
            "precode_ms": ms, "gamma_ratio_mean": float(r.mean()), "gamma_ratio_p99": float(np.percentile(r, 99)),
            "gamma_penalty_db": float(10 * np.log10(r.mean())),
            "l_differs": float(np.mean(np.any(lf != l0, axis=(1, 2))))}
    out["note"] = ("vp_plan_set_fixed_point (16-bit words, F fractional bits) vs the floating-point search "
                   "on the same slot, factor and paths")
    return out


def measure_pipelined(dev, w, steps: int, n_inputs: int = 8) -> dict:
    """Consecutive slots with overlap: two plans on two streams, so that slot
    i + 1's vp_factorize runs beside slot i's vp_precode. Inputs rotate over
    n_inputs independent slot draws (with the two plans' state the working set
    exceeds L2, so no flush runs between slots). Reported beside the plain
    per-slot line, which runs the slots one after another."""
    import torch

    import paper_2602_12098_gb300 as vp
    from paper_2602_12098_gb300 import workloads as W
    bs = [W.make_batch(w, slot=200 + i) for i in range(n_inputs)]
    C, K, M = bs[0].H.shape
    V, S = bs[0].sym.shape[0], w.symbols
    Hs = [torch.from_numpy(b.H).to(dev) for b in bs]
    Ss = [torch.from_numpy(b.sym).to(dev) for b in bs]
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    plans = [vp.Plan(K, M, w.qam, w.n_paths) for _ in range(2)]
    outs = [(torch.empty((V, M), dtype=torch.complex64, device=dev), torch.empty((V, K, 2), dtype=torch.int8, device=dev),
             torch.empty((V,), dtype=torch.float32, device=dev)) for _ in range(2)]

    def slot(i):
        k = i % 2
        vp.vp_factorize(plans[k].handle, Hs[i % n_inputs], C, stream=streams[k])
        vp.vp_precode(plans[k].handle, Ss[i % n_inputs], S, None, V, *outs[k], stream=streams[k])

    for i in range(4):
        slot(i)
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for st in streams:
        st.wait_event(e0)
    for i in range(steps):
        slot(i)
    for st in streams:
        ev = torch.cuda.Event()
        ev.record(st)
        main.wait_event(ev)
    e1.record(main)
    torch.cuda.synchronize()
    for p in plans:
        p.close()
    ms = e0.elapsed_time(e1) / steps
    return {"ms_per_slot": ms, "vectors_per_s": V / (ms / 1e3), "slots": steps,
            "note": "two plans on two streams, slot i + 1 factorised while slot i is precoded; inputs rotate over "
                    f"{n_inputs} slot draws (working set > L2), no flush"}


def measure_configs(dev, flush, steps: int, c1_draws: int = 16):
    """The two smaller configurations as their own bench lines: C1 (4x4
    16-QAM, 64 subcarriers x 1 symbol, 16 paths, i.i.d.) and C2 (8x8 64-QAM,
    1638 subcarriers x 14 symbols, one channel per 12-subcarrier RB, 64
    paths). Per config: vp_factorize + vp_precode on the device-resident
    slot, L2 flushed between steps, median slot time and vectors/s. C1 also
    runs `c1_draws` independent draws (slots) for the oracle leg's
    exhaustive-minimum comparison. Returns (lines, outputs for the oracle
    leg)."""
    import numpy as np
    import torch

    import paper_2602_12098_gb300 as vp
    from paper_2602_12098_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    lines, outs = {}, {}
    for tag, w in (("C1", W.SMALL_4x4), ("C2", W.RB_8x8)):
        draws = c1_draws if tag == "C1" else 1
        res = []
        ts = []
        with vp.Plan(w.K, w.M, w.qam, w.n_paths) as plan:
            for slot in range(draws):
                b = W.make_batch(w, slot=slot)
                C, V = b.H.shape[0], b.sym.shape[0]
                H, sym = torch.from_numpy(b.H).to(dev), torch.from_numpy(b.sym).to(dev)
                off = torch.from_numpy(b.vec_off).to(dev) if w.per_rb else None
                S = 0 if w.per_rb else w.symbols
                x = torch.empty((V, w.M), dtype=torch.complex64, device=dev)
                l = torch.empty((V, w.K, 2), dtype=torch.int8, device=dev)
                g = torch.empty((V,), dtype=torch.float32, device=dev)
                reps = steps + 3 if slot == 0 else 1
                for it in range(reps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    vp.vp_factorize(plan.handle, H, C, stream=stream)
                    vp.vp_precode(plan.handle, sym, S, off, V, x, l, g, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if slot == 0 and it >= 3:
                        ts.append(e0.elapsed_time(e1))
                res.append((b, x.cpu().numpy(), l.cpu().numpy(), g.cpu().numpy().astype(np.float64)))
        ms = statistics.median(ts)
        V0 = res[0][0].sym.shape[0]
        lines[tag] = {"workload": w.name, "slot_ms": ms, "vectors_per_s": V0 / (ms / 1e3),
                      "vectors_per_slot": V0, "channels": int(res[0][0].H.shape[0]),
                      "note": "vp_factorize + vp_precode, device-resident inputs, L2 flushed between steps"}
        outs[tag] = res
    return lines, outs


def measure_path_budgets(dev, b, w, flush, steps: int, budgets=(16, 64, 256, 1024)) -> tuple:
    """The benchmark slot at other path budgets n: vp_factorize + vp_precode
    per slot (device-resident, L2 flushed between steps) and gamma of every
    vector, for the oracle leg's comparison with the exact minimum. Returns
    (lines, {n: gamma})."""
    import numpy as np
    import torch

    import paper_2602_12098_gb300 as vp
    stream = torch.cuda.current_stream()
    C, K, M = b.H.shape
    V, S = b.sym.shape[0], w.symbols
    H, sym = torch.from_numpy(b.H).to(dev), torch.from_numpy(b.sym).to(dev)
    x = torch.empty((V, M), dtype=torch.complex64, device=dev)
    l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
    g = torch.empty((V,), dtype=torch.float32, device=dev)
    lines, gammas = [], {}
    for n in budgets:
        ts = []
        with vp.Plan(K, M, w.qam, n) as plan:
            for it in range(steps + 3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vp.vp_factorize(plan.handle, H, C, stream=stream)
                vp.vp_precode(plan.handle, sym, S, None, V, x, l, g, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if it >= 3:
                    ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        gammas[n] = g.cpu().numpy().astype(np.float64)
        lines.append({"n_paths": n, "slot_ms": ms, "vectors_per_s": V / (ms / 1e3),
                      "gamma_mean": float(gammas[n].mean())})
    return lines, gammas


def measure_paper_points(dev, flush, steps: int) -> list:
    """The shapes of the paper's FPGA throughput table (K = M = 4, 8, 12, 16,
    16-QAM) as whole slots with 8 paths: vectors/s of vp_factorize +
    vp_precode, device-resident, L2 flushed between steps. The FPGA's figures
    (one vector per clock: 424, 410, 264, 256 M vectors/s) are context."""
    import torch

    import paper_2602_12098_gb300 as vp
    from paper_2602_12098_gb300 import workloads as W
    fpga = {4: 424e6, 8: 410e6, 12: 264e6, 16: 256e6}
    stream = torch.cuda.current_stream()
    res = []
    for w in W.PAPER_POINTS:
        b = W.make_batch(w)
        C, K, M = b.H.shape
        V, S = b.sym.shape[0], w.symbols
        H, sym = torch.from_numpy(b.H).to(dev), torch.from_numpy(b.sym).to(dev)
        x = torch.empty((V, M), dtype=torch.complex64, device=dev)
        l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
        g = torch.empty((V,), dtype=torch.float32, device=dev)
        with vp.Plan(K, M, w.qam, w.n_paths) as plan:
            for _ in range(3):
                vp.vp_factorize(plan.handle, H, C, stream=stream)
                vp.vp_precode(plan.handle, sym, S, None, V, x, l, g, stream=stream)
            ts = []
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vp.vp_factorize(plan.handle, H, C, stream=stream)
                vp.vp_precode(plan.handle, sym, S, None, V, x, l, g, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        res.append({"workload": w.name, "slot_ms": ms, "vectors_per_s": V / (ms / 1e3),
                    "fpga_vectors_per_s": fpga[K], "fpga_note": "paper's FPGA (16-bit fixed point, "
                    "one vector per clock), context only"})
    return res


def serving_inputs(dev, jobs, ring: int) -> dict:
    """Device inputs of a Poisson job trace: per job type (K, M, qam), `ring`
    independent draws (those of the type's first `ring` jobs) with their own
    output buffers; the k-th job of a type reads draw k mod ring and writes
    output set k mod ring. The caller keeps the returned tensors alive while
    any descriptor that points at them is in use."""
    import torch

    from paper_2602_12098_gb300 import workloads as W
    sets = {}
    for j in jobs:
        t = (j.K, j.M, j.qam)
        sets.setdefault(t, [])
        if len(sets[t]) < ring:
            Hn, sn = W.job_inputs(j)
            V = sn.shape[0]
            sets[t].append((torch.from_numpy(Hn).to(dev), torch.from_numpy(sn).to(dev),
                            torch.empty((V, j.M), dtype=torch.complex64, device=dev),
                            torch.empty((V, j.K, 2), dtype=torch.int8, device=dev),
                            torch.empty((V,), dtype=torch.float32, device=dev)))
    torch.cuda.synchronize()
    return sets


def serving_outputs_match(dev, sets, last_of: dict, n: int) -> int:
    """Checks the outputs a trace left behind: for every (type, ring slot)
    the last job that wrote it must equal the plan path (vp_factorize +
    vp_precode) on the same inputs, bit for bit. Returns the number checked;
    raises on a mismatch."""
    import torch

    import paper_2602_12098_gb300 as vp
    checked = 0
    for (t, k), _ in sorted(last_of.items()):
        K, M, qam = t
        H, sym, x, l, g = sets[t][k]
        C, V = H.shape[0], sym.shape[0]
        x2, l2, g2 = torch.empty_like(x), torch.empty_like(l), torch.empty_like(g)
        with vp.Plan(K, M, qam, n) as plan:
            vp.vp_factorize(plan.handle, H, C)
            vp.vp_precode(plan.handle, sym, V // C, None, V, x2, l2, g2)
            torch.cuda.synchronize()
        if not (torch.equal(l, l2) and torch.equal(x, x2) and torch.equal(g, g2)):
            raise RuntimeError(f"serving: outputs of a {t} job differ from the plan path")
        checked += 1
    return checked


def measure_serving(dev, n_slots: int, lanes: int = 8, pool_mib: int = 1024, n_paths=(64, 256),
                    loads=(0.1, 0.25, 0.5, 1.0, 2.0, 4.0), ring: int = 8) -> dict:
    """Open-loop serving through the job server (vp_server_*): Poisson job
    arrivals at `loads` mean jobs per 0.5 ms slot; a job is one cell's slot,
    3276 subcarriers x 14 symbols, K in {4, 8, 12, 16}, M = 16, Q in {16, 64,
    256}, iid channels, at each path count in `n_paths`, under both admission
    policies. Each trace is replayed by vp_server_replay (a C++ loop submits
    each job when the host clock reaches its arrival time), so host dispatch
    lag (submission - arrival) is reported apart from device latency (end -
    submission); job latency = end - arrival, on the server's clock. Inputs:
    `ring` independent draws per job type (see serving_inputs); after each
    trace the outputs left in every ring slot are checked against the plan
    path. `capacity_vectors_per_s` is the same jobs submitted all at once."""
    import numpy as np

    import paper_2602_12098_gb300 as vp
    from paper_2602_12098_gb300 import workloads as W
    out = {"workload": f"Poisson arrivals over {n_slots} slots of 0.5 ms; job = 3276 subcarriers x 14 symbols, "
                       "K in {4,8,12,16}, M 16, Q in {16,64,256}, iid",
           "engine": f"vp_server: {lanes} lanes (streams), {pool_mib} MiB state pool, first come first served "
                     "admission by idle lane and pool space; traces replayed by vp_server_replay",
           "deadline_ms": 0.5, "runs": []}
    names = {vp.VP_SERVE_FCFS: "fcfs", vp.VP_SERVE_AGE_PRIORITY: "age_priority"}
    pct = lambda a, q: float(np.percentile(a, q))
    for load in loads:
        jobs = W.poisson_jobs(n_slots, mean_per_slot=load)
        sets = serving_inputs(dev, jobs, ring)
        slot_of, last_of, seen = [], {}, {}
        for i, j in enumerate(jobs):
            t = (j.K, j.M, j.qam)
            slot_of.append(seen.get(t, 0) % ring)
            seen[t] = seen.get(t, 0) + 1
            last_of[(t, slot_of[-1])] = i
        arrival = [j.arrival_us * 1e-3 for j in jobs]
        V = sum(j.subcarriers * j.symbols for j in jobs)
        for n in n_paths:
            descs = []
            for j, k in zip(jobs, slot_of):
                H, sym, x, l, g = sets[(j.K, j.M, j.qam)][k]
                descs.append(vp.job_desc(j.K, j.M, j.qam, n, j.subcarriers, j.symbols, H, sym, x, l, g))
            warm = list({(j.K, j.qam): d for j, d in zip(jobs, descs)}.values())
            cap = None
            for policy in (vp.VP_SERVE_FCFS, vp.VP_SERVE_AGE_PRIORITY):
                with vp.Server(pool_mib << 20, lanes) as srv:
                    srv.set_policy(policy)
                    srv.replay(warm, [0.0] * len(warm))                 # warm-up: every job type once
                    if cap is None:
                        recs, _ = srv.replay(descs, [0.0] * len(descs), timeout_s=600.0)
                        cap = V / (max(r[3] for r in recs) / 1e3)
                    recs, sub = srv.replay(descs, arrival, timeout_s=600.0)
                    st = srv.stats()
                if any(r[1] != 0 for r in recs):
                    raise RuntimeError("serving: a job failed")
                checked = serving_outputs_match(dev, sets, last_of, n)
                end = np.array([r[3] for r in recs])
                arr, subm = np.array(arrival), np.array(sub)
                lat, dev_lat, lag = end - arr, end - subm, subm - arr
                out["runs"].append({
                    "n_paths": n, "jobs_per_slot": load, "jobs": len(jobs), "policy": names[policy],
                    "p50_job_ms": pct(lat, 50), "p99_job_ms": pct(lat, 99), "max_job_ms": float(lat.max()),
                    "deadline_miss_frac": float(np.mean(lat > 0.5)),
                    "p50_device_ms": pct(dev_lat, 50), "p99_device_ms": pct(dev_lat, 99),
                    "p50_dispatch_lag_ms": pct(lag, 50), "p99_dispatch_lag_ms": pct(lag, 99),
                    "max_dispatch_lag_ms": float(lag.max()),
                    "vectors_per_s": V / (end.max() / 1e3), "offered_vectors_per_s": V / (arr[-1] / 1e3),
                    "capacity_vectors_per_s": cap, "outputs_checked": checked,
                    "max_in_flight": st["max_in_flight"], "pool_high_water_mib": st["pool_high_water"] / 2**20})
        if load == loads[0]:
            # each job type alone (arrivals 3 ms apart, after a warm-up): the floor of its latency
            alone = {}
            for n in n_paths:
                types = sorted(sets)
                descs = []
                for t in types:
                    H, sym, x, l, g = sets[t][0]
                    descs.append(vp.job_desc(t[0], t[1], t[2], n, H.shape[0], sym.shape[0] // H.shape[0],
                                             H, sym, x, l, g))
                with vp.Server(pool_mib << 20, lanes) as srv:
                    srv.replay(descs, [0.0] * len(descs))
                    recs, sub = srv.replay(descs * 3, [3.0 * i for i in range(3 * len(descs))], timeout_s=60.0)
                for i, t in enumerate(types):
                    ms = sorted(recs[i + k * len(types)][3] - sub[i + k * len(types)] for k in range(3))
                    alone[f"n{n}_K{t[0]}_Q{t[2]}"] = ms[1]
            out["alone_job_ms"] = alone
        out["inputs"] = (f"{ring} independent draws per job type with their own outputs "
                         f"({sum(t[0].numel() * 8 + t[1].numel() for v in sets.values() for t in v) / 2**20:.0f} MiB "
                         "of H and symbols at the last load)")
        del sets
    for n in n_paths:
        ok = [r["jobs_per_slot"] for r in out["runs"]
              if r["n_paths"] == n and r["policy"] == "fcfs" and r["p99_job_ms"] <= out["deadline_ms"]]
        out[f"max_load_p99_within_deadline_n{n}"] = max(ok) if ok else None
    return out


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2602_12098_gb300 as vp
    from paper_2602_12098_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = W.WORKLOADS[args.workload]
    if args.paths is not None:
        import dataclasses
        w = dataclasses.replace(w, n_paths=args.paths)
    b = replica_batch(w, rank, args.subcarriers)
    C, K, M = b.H.shape
    V = b.sym.shape[0]
    S = w.symbols
    uniform = not w.per_rb
    vp.load()
    stream = torch.cuda.current_stream()
    H = torch.from_numpy(b.H).to(dev)
    sym = torch.from_numpy(b.sym).to(dev)
    off = None if uniform else torch.from_numpy(b.vec_off).to(dev)
    x = torch.empty((V, M), dtype=torch.complex64, device=dev)
    l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
    g = torch.empty((V,), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    plan = vp.Plan(K, M, w.qam, w.n_paths)
    h = plan.handle
    launches = [0]

    def step():
        vp.vp_factorize(h, H, C, stream=stream)
        n = vp.vp_last_launch_count(h)
        vp.vp_precode(h, sym, S if uniform else 0, off, V, x, l, g, stream=stream)
        launches[0] += n + vp.vp_last_launch_count(h)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(dev)
    gid = None
    if hasattr(props, "uuid"):
        u = str(props.uuid)
        gid = u if u.startswith("GPU-") else "GPU-" + u
    sampler = ClockSampler(gid)
    sampler.start()
    time.sleep(0.3)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    launches[0] = 0
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        vp.vp_factorize(h, H, C, stream=stream)
        n = vp.vp_last_launch_count(h)
        ev[i][1].record(stream)
        vp.vp_precode(h, sym, S if uniform else 0, off, V, x, l, g, stream=stream)
        launches[0] += n + vp.vp_last_launch_count(h)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    fac_ms = [e[0].elapsed_time(e[1]) for e in ev]
    srch_ms = [e[1].elapsed_time(e[2]) for e in ev]
    tot_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = whole_job_rate(ws, V, args.steps, tot_ms / 1e3)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        Hh = torch.from_numpy(b.H).pin_memory()
        sh = torch.from_numpy(b.sym).pin_memory()
        xh = torch.empty((V, M), dtype=torch.complex64).pin_memory()
        lh = torch.empty((V, K, 2), dtype=torch.int8).pin_memory()
        gh = torch.empty((V,), dtype=torch.float32).pin_memory()
        n_e2e = max(3, min(args.steps, 200))
        for _ in range(3):
            vp.vp_run_slot_host(h, Hh, C, sh, S, xh, lh, gh, stream=stream)
        ts = []
        for _ in range(n_e2e):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            vp.vp_run_slot_host(h, Hh, C, sh, S, xh, lh, gh, stream=stream)
            ts.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(sum(ts), dist, dev)
        e2e = {"value": whole_job_rate(ws, V, n_e2e, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(b.H.nbytes + b.sym.nbytes),
               "d2h_bytes_per_step": int(V * M * 8 + V * K * 2 + V * 4),
               "p50_slot_ms": 1e3 * statistics.median(ts),
               "api": "vp_run_slot_host (H2D copies of H and symbols, vp_factorize, vp_precode writing x, l, gamma "
                      "into the pinned host buffers over the C2C link, stream sync)"}

    # roofline of the dominant kernel (the search), ALU-bound FP32
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = props.multi_processor_count
    peak_tflops = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    flops_launch = paper_work_flops(K, M, w.n_paths) * V
    search_avg = statistics.mean(srch_ms)
    achieved = flops_launch / (search_avg / 1e3) / 1e12
    # the state of the timed slot: FP64 channels and the paths (outside the timed region)
    stt = torch.empty((C,), dtype=torch.uint8, device=dev)
    vp.vp_factorize(h, H, C, None, None, None, stt, stream=stream)
    codes = torch.empty((C, w.n_paths), dtype=torch.int64, device=dev)
    vp.vp_get_paths(h, codes, stream=stream)
    torch.cuda.synchronize()
    fp64_frac = float((stt.cpu().numpy() & vp.VP_CH_FP64).astype(bool).mean())
    exec_flops = 8.0 * executed_cmul(codes.cpu().numpy().view(np.uint64), K, M, w.n_paths) * V
    executed = exec_flops / (search_avg / 1e3) / 1e12
    tr = (profiled_traffic("search_kernel_slot16x16.md")
          if args.subcarriers is None and args.paths is None and args.workload == "slot_16x16" else None)
    roofline = {"bound": "alu", "kernel": "search_kernel<16> (vp_precode)", "achieved": achieved,
                "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                "traffic": tr["bytes"] if tr else None,
                "traffic_basis": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, {tr['file']}"
                                  if tr else "no ncu capture of the current search kernel sources"),
                "peak_basis": f"FP32 FMA: {sms} SMs x 128 lanes x 2 flops x {sm_mhz:.0f} MHz "
                              "(max SM clock, MEASURED_PEAKS.json)",
                "work_basis": "paper's per-vector complex-multiplication count x 8 flops (effective: every "
                              "path's full descent)",
                "executed": executed, "executed_frac": executed / peak_tflops,
                "executed_basis": "the same count with the shared top levels once per distinct prefix, as run"}
    if tr and "warp_instructions" in tr:
        # the bound that binds: instruction issue (4 schedulers per SM, one warp instruction each per clock)
        issue_peak = sms * 4 * sm_mhz * 1e6
        issue_ach = tr["warp_instructions"] / (search_avg / 1e3)
        roofline["issue"] = {"achieved": issue_ach / 1e12, "peak": issue_peak / 1e12, "unit": "T warp instr/s",
                             "frac": issue_ach / issue_peak,
                             "basis": f"ncu smsp__inst_executed.sum per launch ({tr['file']}) / the live search time; "
                                      f"peak {sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "K": K, "M": M, "qam": w.qam, "n_paths": w.n_paths,
                       "channels": C, "vectors_per_step": V, "parallelism": f"replicas x{ws}",
                       "fp64_channels_frac": fp64_frac,
                       "l2": "flushed between steps (256 MiB device write outside the timed events)"},
            "p50_slot_ms": statistics.median(step_ms),
            "p99_slot_ms": sorted(step_ms)[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)],
            "kernel_ms": {"vp_factorize": statistics.mean(fac_ms), "vp_precode": search_avg},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches[0], "clocks": clocks}
    plan.close()
    configs_out = None
    budget_gammas = None
    if ws == 1 and not args.no_batched:
        line["demap_lut"] = measure_lut(dev, b, w, flush, min(args.steps, 100))
        line["fixed_point"] = measure_fixed(dev, b, w, flush, min(args.steps, 20))
        line["batched"] = measure_batched(dev, flush)
        line["batched_one_vector"] = measure_batched(dev, flush, symbols_per_problem=1)
        line["paper_points"] = measure_paper_points(dev, flush, min(args.steps, 50))
        line["configs"], configs_out = measure_configs(dev, flush, min(args.steps, 50))
        line["path_budgets"], budget_gammas = measure_path_budgets(dev, b, w, flush, min(args.steps, 20))
        line["pipelined"] = measure_pipelined(dev, w, min(args.steps, 200))
    if ws == 1 and not args.no_serving:
        line["serving"] = measure_serving(dev, args.serving_slots, args.serving_lanes, args.serving_pool_mib,
                                          args.serving_paths)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, gpu_sample=(b, x.cpu().numpy(), l.cpu().numpy(),
                                                           g.cpu().numpy().astype(np.float64)),
                                            configs_sample=configs_out, budget_gammas=budget_gammas)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
