"""The C-ABI library builds, loads and exports every declared entry point.

These run without a GPU: only argument validation paths are exercised (they
return before any CUDA call).
"""
import os
import re

import pytest

import paper_2602_12098_gb300 as vp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(vp_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_header_declares_the_binding_names():
    decl = declared_entry_points()
    assert set(vp.EXPORTED_SYMBOLS) <= set(decl)
    assert "vp_precode" in decl and "vp_factorize" in decl and "vp_plan_create" in decl


def test_library_exports_every_declared_symbol():
    lib = vp.load()
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_plan_argument_validation():
    bad = [(0, 4, 16, 16), (17, 17, 16, 16), (4, 0, 16, 16), (4, 4, 32, 16), (4, 4, 16, 0),
           (2, 2, 16, 82), (4, 4, 16, 2000), (4, 17, 16, 16)]
    for K, M, q, n in bad:
        with pytest.raises(vp.VPError) as e:
            vp.vp_plan_create(K, M, q, n)
        assert e.value.code == 1
    with pytest.raises(vp.VPError):
        vp.vp_plan_create(4, 4, 16, 16, tau=-1.0)
    h = vp.vp_plan_create(4, 4, 16, 16)
    try:
        with pytest.raises(vp.VPError):
            vp.vp_plan_set_fp64_threshold(h, -1.0)
        vp.vp_plan_set_fp64_threshold(h, 100.0)
        with pytest.raises(vp.VPError) as e:         # nothing factorised yet
            vp.vp_precode(h, 1, 1, None, 1, 1, 1, 1, stream=0)
        assert e.value.code == 5
        with pytest.raises(vp.VPError) as e:
            vp.vp_factorize(h, 1, 0, stream=0)
        assert e.value.code == 1
        assert vp.vp_last_launch_count(h) == 0
    finally:
        lib = vp.load()
        lib.vp_plan_destroy(h)


def test_status_strings():
    assert vp.vp_status_string(0) == "ok"
    assert "invalid" in vp.vp_status_string(1)
    assert vp.vp_status_string(99) == "unknown status"


def _desc(K=4, M=8, qam=16, n=16, S=14, tau=0.0, ptr=256):
    return vp.vp_problem_desc(K, M, qam, n, tau, S, ptr, ptr, ptr, ptr, ptr, 0)


def test_batch_validation_and_grouping():
    """Batch planning is host-only: descriptors are validated and grouped
    into one factor launch per (K, M), one path launch per n class and one
    search launch per K tile (+ the FP64 launch)."""
    good = [_desc(4, 8, 16, 16), _desc(8, 16, 64, 64), _desc(12, 16, 256, 256), _desc(16, 16, 256, 1024),
            _desc(4, 8, 256, 1024), _desc(8, 16, 16, 20, S=0)]
    assert vp.vp_precode_batch_workspace_bytes(good) > 0
    for bad in [_desc(K=17), _desc(K=4, M=3), _desc(qam=32), _desc(n=0), _desc(K=2, M=2, n=82),
                _desc(n=2000), _desc(S=-1), _desc(tau=-1.0), _desc(ptr=0)]:
        assert vp.vp_precode_batch_workspace_bytes(good + [bad]) == 0
        with pytest.raises(vp.VPError) as e:
            vp.vp_batch_create(good + [bad])
        assert e.value.code == 1
    b = vp.vp_batch_create(good)
    try:
        # factor: (4,8), (8,16), (12,16), (16,16); paths: n classes 16, 64, 256, 1024;
        # search: K tiles 4, 8, 12, 16 (the default) or one persistent launch;
        # plus the FP64 fix-up
        assert vp.vp_batch_launch_count(b) == 4 + 4 + 4 + 1
        vp.vp_batch_set_persistent(b, 1)
        assert vp.vp_batch_launch_count(b) == 4 + 4 + 1 + 1
        vp.vp_batch_set_persistent(b, 0)
        with pytest.raises(vp.VPError):
            vp.vp_batch_set_persistent(b, 2)
        for bad in (2, -1):
            with pytest.raises(vp.VPError) as e:
                vp.vp_batch_set_concurrent(b, bad)
            assert e.value.code == 1
        vp.vp_batch_set_concurrent(b, 0)                 # unbound: no streams needed either way
        vp.vp_batch_set_concurrent(b, 1)
        assert vp.vp_batch_launch_count(b) == 4 + 4 + 4 + 1
        info = vp.vp_batch_group_info(b)
        assert [g[0] for g in info] == [0] * 4 + [1] * 4 + [2] * 4 + [3]
        assert info[-1][1] == len(good) and info[-1][4] == 1024 and info[-1][5] == 14
        knobs = vp.vp_batch_get_tuning(b)
        assert len(knobs) == 13
        for bad in (5 << 3, 3 << 6, 256, -1):             # no such blocks / staging value
            with pytest.raises(vp.VPError):
                vp.vp_batch_set_tuning(b, knobs[:-1] + [bad])
        vp.vp_batch_set_tuning(b, knobs[:-1] + [7 | (2 << 3) | (1 << 6)])
        ws = vp.vp_batch_workspace_bytes(b)
        assert ws == vp.vp_precode_batch_workspace_bytes(good)
        with pytest.raises(vp.VPError) as e:          # never bound to a workspace
            vp.vp_batch_launch(b, stream=0)
        assert e.value.code == 5
        with pytest.raises(vp.VPError) as e:          # workspace too small / misaligned
            vp.vp_batch_bind(b, 4096, ws - 1, stream=0)
        assert e.value.code == 1
        with pytest.raises(vp.VPError) as e:
            vp.vp_batch_bind(b, 4100, ws, stream=0)
        assert e.value.code == 1
    finally:
        vp.vp_batch_destroy(b)
    with pytest.raises(vp.VPError):
        vp.vp_batch_create(good, fp64_threshold=float("nan"))


def test_overloaded_plan_needs_lambda():
    """K > M is a valid plan, but factorising it needs lambda > 0 (checked on
    the host before any device work)."""
    h = vp.vp_plan_create(8, 4, 4, 64)
    try:
        with pytest.raises(vp.VPError) as e:
            vp.vp_factorize(h, 256, 2, stream=0)
        assert e.value.code == 1
        for bad in (-0.5, float("nan"), float("inf")):
            with pytest.raises(vp.VPError):
                vp.vp_plan_set_lambda(h, bad)
        vp.vp_plan_set_lambda(h, 0.5)
        vp.vp_plan_set_lambda(h, 0.0)
    finally:
        vp.vp_plan_destroy(h)


def test_demap_option_validation():
    h = vp.vp_plan_create(4, 4, 16, 16)
    try:
        vp.vp_plan_set_demap(h, vp.VP_DEMAP_LUT)
        vp.vp_plan_set_demap(h, vp.VP_DEMAP_EXACT)
        for bad in (-1, 2, 7):
            with pytest.raises(vp.VPError) as e:
                vp.vp_plan_set_demap(h, bad)
            assert e.value.code == 1
    finally:
        vp.vp_plan_destroy(h)


def test_fixed_point_option_validation():
    h = vp.vp_plan_create(4, 4, 16, 16)
    try:
        for f in (1, 8, 13, 15, 0):
            vp.vp_plan_set_fixed_point(h, f)
        for bad in (-1, 16, 40):
            with pytest.raises(vp.VPError) as e:
                vp.vp_plan_set_fixed_point(h, bad)
            assert e.value.code == 1
        # only with the exact DEMAP, whichever is set first
        vp.vp_plan_set_fixed_point(h, 11)
        with pytest.raises(vp.VPError):
            vp.vp_plan_set_demap(h, vp.VP_DEMAP_LUT)
        vp.vp_plan_set_fixed_point(h, 0)
        vp.vp_plan_set_demap(h, vp.VP_DEMAP_LUT)
        with pytest.raises(vp.VPError):
            vp.vp_plan_set_fixed_point(h, 11)
    finally:
        vp.vp_plan_destroy(h)


def test_server_argument_validation():
    """Argument errors of the job server come back before any CUDA call."""
    for pool, lanes in ((1 << 19, 4), (1 << 20, 0), (1 << 20, 33), (1 << 30, -1)):
        with pytest.raises(vp.VPError) as e:
            vp.vp_server_create(pool, lanes)
        assert e.value.code == 1
    lib = vp.load()
    job = vp.job_desc(4, 4, 16, 16, 8, 14, 1, 1, 1, 1, 1)
    import ctypes
    i = ctypes.c_int64()
    n = ctypes.c_int()
    assert lib.vp_server_submit(None, ctypes.byref(job), ctypes.byref(i)) == 1
    assert lib.vp_server_poll(None, None, 0, ctypes.byref(n)) == 1
    assert lib.vp_server_drain(None, 1.0) == 1
    assert lib.vp_server_reset_clock(None) == 1
    assert lib.vp_server_get_stats(None, None) == 1
    assert lib.vp_server_destroy(None) == 0


def test_batch_tuning_knobs_host_side():
    """Tuning knobs per launch group: group shapes, validation of set values,
    and the autotuner's refusal on an unbound batch (all before any CUDA call)."""
    good = [_desc(4, 8, 16, 16), _desc(8, 16, 64, 64), _desc(16, 16, 256, 1024)]
    b = vp.vp_batch_create(good)
    try:
        info = vp.vp_batch_group_info(b)
        stages = [g[0] for g in info]
        assert stages == sorted(stages) and set(stages) == {0, 1, 2, 3}
        # every group is one launch except the form of the search not in use
        assert len(info) == vp.vp_batch_launch_count(b) - 1 + stages.count(3)
        assert vp.vp_batch_get_tuning(b) == [0] * len(info)
        knob = {0: 0, 1: 128, 2: 5, 3: 6 | (2 << 3) | (2 << 6)}
        knobs = [knob[st] for st in stages]
        vp.vp_batch_set_tuning(b, knobs)
        assert vp.vp_batch_get_tuning(b) == knobs
        for bad in (knobs[:-1], [48 if st == 1 else knob[st] for st in stages],
                    [8 if st == 2 else knob[st] for st in stages],
                    [7 if st == 0 else knob[st] for st in stages],
                    [(3 << 6) if st == 3 else knob[st] for st in stages]):
            with pytest.raises(vp.VPError) as e:
                vp.vp_batch_set_tuning(b, bad)
            assert e.value.code == 1
        assert vp.vp_batch_get_tuning(b) == knobs           # unchanged by the refused calls
        with pytest.raises(vp.VPError) as e:
            vp.vp_batch_autotune(b, 3, stream=0)
        assert e.value.code == 5
    finally:
        vp.vp_batch_destroy(b)


def test_noalloc_capacity_checked_before_any_device_work():
    """vp_precode_noalloc refuses C > vp_noalloc_max_channels(plan) with
    VP_ERR_CAPACITY before touching a device, for the plain layout, the
    lambda > 0 layout (K extra rows of P) and a status-only call (S = 0);
    C = C_max passes the capacity check (it then needs a device: without
    one the call fails with VP_ERR_CUDA, never with VP_ERR_CAPACITY)."""
    import torch
    lib = vp.load()
    caps = {}
    for name, (K, M, q, n, lam) in {"plain": (16, 16, 256, 256, 0.0), "lambda": (16, 16, 256, 256, 0.5),
                                     "overloaded": (8, 4, 4, 64, 0.5), "small": (4, 4, 16, 16, 0.0)}.items():
        with vp.Plan(K, M, q, n, lam=lam) as plan:
            cmax = vp.vp_noalloc_max_channels(plan.handle)
            caps[name] = cmax
            assert cmax > 0
            for S in (14, 0):
                rc = lib.vp_precode_noalloc(plan.handle, 256, cmax + 1, 256, S, 256, 256, 256, None, None)
                assert rc == 6, (name, S, rc)
                if not torch.cuda.is_available():
                    rc = lib.vp_precode_noalloc(plan.handle, 256, cmax, 256, S, 256, 256, 256, None, None)
                    assert rc != 6, (name, S, rc)
    assert caps["lambda"] < caps["plain"] < caps["small"]
