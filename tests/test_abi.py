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
    bad = [(0, 4, 16, 16), (17, 17, 16, 16), (4, 3, 16, 16), (4, 4, 32, 16), (4, 4, 16, 0),
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
