"""vp_precode_noalloc (state in the library's static device array) against the
plan path vp_factorize + vp_precode, through the C-ABI.

Two calls in a row on different slots and channel counts, so that the second
call runs on storage the first one left behind. Outputs must agree within the
parity tolerances of the other GPU tests (the kernels are the same, so they
are expected to agree exactly). Kept in a file of its own, collected last.
"""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2602_12098_gb300 as vp
from paper_2602_12098_gb300 import workloads as W
from vp_gpu_util import GAMMA_RTOL, L_MATCH_MIN, X_RTOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vp.load()


def _plan_path(b, S):
    dev = torch.device("cuda:0")
    w = b.workload
    C, K, M = b.H.shape
    V = C * S
    H = torch.from_numpy(b.H).to(dev)
    sym = torch.from_numpy(b.sym).to(dev)
    x = torch.empty((V, M), dtype=torch.complex64, device=dev)
    l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
    g = torch.empty((V,), dtype=torch.float32, device=dev)
    st = torch.empty((C,), dtype=torch.uint8, device=dev)
    with vp.Plan(K, M, w.qam, w.n_paths) as plan:
        vp.vp_factorize(plan.handle, H, C, None, None, None, st)
        vp.vp_precode(plan.handle, sym, S, None, V, x, l, g)
        torch.cuda.synchronize()
    return {"x": x.cpu().numpy(), "l": l.cpu().numpy(), "gamma": g.cpu().numpy(), "status": st.cpu().numpy()}


def _noalloc(plan, b, S):
    dev = torch.device("cuda:0")
    C, K, M = b.H.shape
    V = C * S
    H = torch.from_numpy(b.H).to(dev)
    sym = torch.from_numpy(b.sym).to(dev)
    # poisoned outputs: every element must be written
    x = torch.full((V, M), float("nan"), dtype=torch.complex64, device=dev)
    l = torch.full((V, K, 2), 99, dtype=torch.int8, device=dev)
    g = torch.full((V,), float("nan"), dtype=torch.float32, device=dev)
    st = torch.full((C,), 255, dtype=torch.uint8, device=dev)
    vp.vp_precode_noalloc(plan.handle, H, C, sym, S, x, l, g, st)
    torch.cuda.synchronize()
    return {"x": x.cpu().numpy(), "l": l.cpu().numpy(), "gamma": g.cpu().numpy(), "status": st.cpu().numpy()}


def _assert_close(a, b):
    assert np.array_equal(a["status"], b["status"])
    l_eq = np.all(a["l"] == b["l"], axis=(1, 2))
    assert l_eq.mean() >= L_MATCH_MIN, l_eq.mean()
    m = l_eq & (b["gamma"] > 0)
    assert np.all(np.abs(a["gamma"][m] - b["gamma"][m]) <= GAMMA_RTOL * b["gamma"][m])
    assert np.all(np.linalg.norm(a["x"][m] - b["x"][m], axis=1) <= X_RTOL)
    z = b["gamma"] == 0
    assert np.all(a["gamma"][z] == 0) and np.all(a["x"][z] == 0)


def test_noalloc_matches_plan_path_two_calls():
    wl = W.SLOT_16x16
    S = wl.symbols
    # larger slot first, then a smaller one with other channels (FP64 channels in both)
    batches = [W.make_batch(wl, slot=3, subcarriers=96), W.make_batch(wl, slot=4, subcarriers=40)]
    with vp.Plan(wl.K, wl.M, wl.qam, wl.n_paths) as plan:
        outs = [_noalloc(plan, b, S) for b in batches]
    for b, out in zip(batches, outs):
        ref = _plan_path(b, S)
        assert np.any(ref["status"] == vp.VP_CH_FP64)
        _assert_close(out, ref)


def test_noalloc_capacity_boundary():
    """The largest channel count the library reports is accepted and matches the
    plan path; one more channel is refused with VP_ERR_CAPACITY."""
    wl = W.SLOT_16x16
    K, M = wl.K, wl.M
    S = 2
    with vp.Plan(K, M, wl.qam, wl.n_paths) as plan:
        cmax = vp.vp_noalloc_max_channels(plan.handle)
        assert 0 < cmax < 100000
        b = W.make_batch(dataclasses.replace(wl, symbols=S), slot=5, subcarriers=cmax)
        out = _noalloc(plan, b, S)
        dev = torch.device("cuda:0")
        C = cmax + 1
        H = torch.zeros((C, K, M), dtype=torch.complex64, device=dev)
        sym = torch.zeros((C, K), dtype=torch.uint8, device=dev)
        x = torch.zeros((C, M), dtype=torch.complex64, device=dev)
        l = torch.zeros((C, K, 2), dtype=torch.int8, device=dev)
        g = torch.zeros((C,), dtype=torch.float32, device=dev)
        with pytest.raises(vp.VPError) as e:
            vp.vp_precode_noalloc(plan.handle, H, C, sym, 1, x, l, g)
        assert e.value.code == 6
        torch.cuda.synchronize()
    _assert_close(out, _plan_path(b, S))
