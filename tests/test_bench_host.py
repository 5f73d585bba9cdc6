"""Host-side arithmetic of bench.py (no GPU): the per-vector work counts
behind roofline.achieved and roofline.executed."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _codes(rows):
    """uint64 path codes from digit lists (level 0 first)."""
    out = []
    for digs in rows:
        c = 0
        for l, d in enumerate(digs):
            c |= d << (4 * l)
        out.append(c)
    return np.array(out, dtype=np.uint64)


def test_paper_count_closed_form():
    # N_r N_t + N_t^2 + n N_t (1 + (N_t + 1) / 2) complex multiplications, 8 flops each
    assert bench.paper_work_flops(16, 16, 256) == 8.0 * (256 + 256 + 256 * 16 * 9.5) == 8.0 * 39424
    assert bench.paper_work_flops(4, 4, 16) == 8.0 * (16 + 16 + 16 * 4 * 3.5)


def test_executed_equals_paper_without_shared_levels():
    # K = 4 (< 8) never shares levels: every path runs all levels
    rng = np.random.default_rng(0)
    codes = _codes(rng.integers(0, 9, size=(16, 4)).tolist())[None]
    K, M, n = 4, 4, 16
    assert bench.executed_cmul(codes, K, M, n) == bench.paper_work_flops(K, M, n) / 8.0


def test_executed_counts_shared_prefixes_once():
    # K = 8, n = 64 paths over 2 distinct top-3-level prefixes: the top three
    # levels (8, 7, 6 from the bottom; costs 9, 8, 7) run twice, the rest 64 times
    K, M, n = 8, 8, 64
    rows = []
    for i in range(n):
        low = [(i >> b) & 1 for b in range(5)]          # levels 0-4
        top = [0, 0, i & 1]                             # levels 5, 6, 7: two prefixes
        rows.append(low + top)
    codes = _codes(rows)[None]
    want = K * M + K * K + 2 * (9 + 8 + 7) + n * sum(1 + l for l in range(1, 6))
    assert bench.executed_cmul(codes, K, M, n) == want


def test_whole_job_rate_and_slowest_rank():
    assert bench.whole_job_rate(2, 1000, 10, 0.5) == 2 * 1000 * 10 / 0.5
    assert bench.max_over_ranks(3.0) == 3.0


def test_code_fingerprint_ignores_comments_and_layout(tmp_path, monkeypatch):
    """A profile stays valid across comment and whitespace edits of the
    kernel sources, and not across code edits."""
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "k.cu").write_text("int f(int a) {  // add one\n    return a + 1; /* one */\n}\n")
    base = bench.code_fingerprint(["k.cu"])
    (tmp_path / "k.cu").write_text("// header\nint f(int a)\n{\n  return a + 1;\n}\n")
    assert bench.code_fingerprint(["k.cu"]) == base
    (tmp_path / "k.cu").write_text("int f(int a) { return a + 2; }\n")
    assert bench.code_fingerprint(["k.cu"]) != base


def test_profiled_counters_valid_only_for_the_profiled_code(tmp_path, monkeypatch):
    """DRAM bytes and warp instructions from a profile summary are used only
    while the listed sources keep the profiled code fingerprint."""
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("__global__ void k() {}\n")
    fp = bench.code_fingerprint(["k.cu"])
    (tmp_path / "profiles" / "p.md").write_text(
        f"# k\n\n- sources: `k.cu`\n- sources_code_sha256: `{fp}`\n- dram_bytes_per_launch: `1000`\n"
        "- warp_instructions_per_launch: `5000`\n")
    got = bench.profiled_traffic("p.md")
    assert got["bytes"] == 1000.0 and got["warp_instructions"] == 5000.0
    (tmp_path / "k.cu").write_text("__global__ void k() { int a = 1; }\n")
    assert bench.profiled_traffic("p.md") is None
