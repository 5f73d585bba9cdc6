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
    return ap.parse_args()


def paper_work_flops(K: int, M: int, n: int) -> float:
    """FP32 flops of one precoded vector from the paper's per-vector count of
    complex multiplications N_r N_t + N_t^2 + n N_t (1 + (N_t + 1) / 2)
    (Section III-B, with N_t -> K for the tree size), 8 flops (4 FMA) each."""
    cmul = K * M + K * K + n * K * (1 + (K + 1) / 2)
    return 8.0 * cmul


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


def run_reference(args):
    """FP64 CPU oracle on the host cores, bounded sample per step (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2602_12098_gb300 import workloads as W
    w = W.WORKLOADS[args.workload]
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


def cpu_baseline(w, sub_channels: int = 1024) -> dict:
    from oracle import oracle as O
    from paper_2602_12098_gb300 import workloads as W
    threads = os.cpu_count() or 1
    b = W.make_batch(w, subcarriers=min(sub_channels, w.subcarriers))
    t0 = time.perf_counter()
    O.precode_batch(b.H, b.sym, b.vec_off, w.qam, w.n_paths, nthreads=threads)
    dt = time.perf_counter() - t0
    V = b.sym.shape[0]
    cores = min(threads, O.max_threads()) if O.max_threads() > 1 else 1
    return {"value": V / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{b.H.shape[0]} of {w.subcarriers} subcarriers x {w.symbols} symbols ({V} vectors), "
                      f"{dt:.1f} s wall"}


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
    b = W.make_batch(w, slot=rank, subcarriers=args.subcarriers)
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
    tot_ms = sum(step_ms)
    if dist:
        t = torch.tensor([tot_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = ws * V * args.steps / (tot_ms / 1e3)

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
        e2e_s = sum(ts)
        if dist:
            t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": ws * V * n_e2e / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(b.H.nbytes + b.sym.nbytes),
               "d2h_bytes_per_step": int(V * M * 8 + V * K * 2 + V * 4),
               "p50_slot_ms": 1e3 * statistics.median(ts),
               "api": "vp_run_slot_host (H2D copies, vp_factorize, vp_precode, D2H copies, stream sync)"}

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
    roofline = {"bound": "alu", "kernel": "search_kernel<16> (vp_precode)", "achieved": achieved,
                "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": None,
                "peak_basis": f"FP32 FMA: {sms} SMs x 128 lanes x 2 flops x {sm_mhz:.0f} MHz "
                              "(max SM clock, MEASURED_PEAKS.json)",
                "work_basis": "paper's per-vector complex-multiplication count x 8 flops"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "K": K, "M": M, "qam": w.qam, "n_paths": w.n_paths,
                       "channels": C, "vectors_per_step": V, "parallelism": f"replicas x{ws}",
                       "l2": "flushed between steps (256 MiB device write outside the timed events)"},
            "p50_slot_ms": statistics.median(step_ms),
            "p99_slot_ms": sorted(step_ms)[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)],
            "kernel_ms": {"vp_factorize": statistics.mean(fac_ms), "vp_precode": search_avg},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches[0], "clocks": clocks}
    plan.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
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
