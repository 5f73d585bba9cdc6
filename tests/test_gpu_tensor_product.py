"""w = P u on the tensor cores (vp_plan_set_tensor_product, the PV block of
Section IV-B, Eqs. 24-25): element by element against the FP64 oracle, and
against the CUDA-core product on the same search (l identical, gamma and x
to FP32 rounding), through the C-ABI. Cases cover one round of 16 vectors
per channel, channels with more vectors than a round (per-RB channels),
FP64-refined channels (P as a hi/lo pair), the K regularisation rows of
lambda > 0, and path budgets that would otherwise take the one-pass kernel."""
import numpy as np
import pytest
import torch

import paper_2602_12098_gb300 as vp
from paper_2602_12098_gb300 import workloads as W
from vp_gpu_util import assert_parity, compare, run_gpu

pytestmark = pytest.mark.gpu

# the tensor-core and CUDA-core products of the same perturbation agree to
# FP32 rounding of w (both are exact up to the rounding of P and of the sums)
AGREE = 2e-6


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vp.load()


def _agree(a, b):
    assert np.array_equal(a["l"], b["l"])
    assert np.array_equal(a["status"], b["status"])
    m = b["gamma"] > 0
    assert np.all(np.abs(a["gamma"][m] - b["gamma"][m]) <= AGREE * b["gamma"][m])
    assert np.max(np.linalg.norm(a["x"] - b["x"], axis=1)) <= AGREE


CASES = [
    # K, M, qam, n, channels, vectors per channel, lambda, every channel in FP64
    (16, 16, 256, 256, 48, 14, 0.0, False),
    (16, 16, 256, 256, 24, 14, 0.0, True),
    (8, 8, 64, 64, 12, 40, 0.0, False),
    (4, 8, 16, 16, 64, 5, 0.0, False),
    (12, 16, 64, 1024, 16, 14, 0.0, False),
    (12, 8, 16, 64, 20, 14, 0.4, False),
    (2, 2, 4, 9, 30, 3, 0.0, False),
]


@pytest.mark.parametrize("K,M,qam,n,C,S,lam,fp64", CASES)
def test_tensor_product_vs_oracle(orc, K, M, qam, n, C, S, lam, fp64):
    rng = W.rng_for(97, K * 1000 + M * 10 + S)
    H = W.channels(rng, C, K, M, "kron" if K == 16 else "iid", 0.5, 0.2)
    sym = W.symbols(rng, C * S, K, qam)
    off = W.vec_offsets_uniform(C, S)
    thr = 0.0 if fp64 else None
    tcp = run_gpu(H, sym, off, qam, n, lam=lam, fp64_threshold=thr, want_factor=False, uniform_S=S, tensor_product=1)
    cuda = run_gpu(H, sym, off, qam, n, lam=lam, fp64_threshold=thr, want_factor=False, uniform_S=S)
    _agree(tcp, cuda)
    ref = orc.precode_batch(H, sym, off, qam, n, lam=lam, nthreads=orc.max_threads())
    st = compare(orc, H, sym, off, qam, tcp, ref, lam=lam)
    print(K, M, n, S, lam, fp64, st)
    assert_parity(st)


def test_tensor_product_full_slot_agrees():
    """The whole 16x16 slot (3276 channels x 14 symbols): the tensor-core
    product equals the CUDA-core one on every vector to FP32 rounding."""
    b = W.make_batch(W.SLOT_16x16, slot=7)
    w = b.workload
    kw = dict(want_factor=False, uniform_S=w.symbols)
    tcp = run_gpu(b.H, b.sym, b.vec_off, w.qam, w.n_paths, tensor_product=1, **kw)
    cuda = run_gpu(b.H, b.sym, b.vec_off, w.qam, w.n_paths, **kw)
    _agree(tcp, cuda)
    assert np.allclose(np.linalg.norm(tcp["x"], axis=1), 1.0, atol=1e-6)


def test_tensor_product_setting_is_checked():
    with vp.Plan(4, 4, 16, 16) as plan:
        with pytest.raises(vp.VPError):
            vp.vp_plan_set_tensor_product(plan.handle, 2)
        vp.vp_plan_set_tensor_product(plan.handle, 1)
        vp.vp_plan_set_tensor_product(plan.handle, 0)
