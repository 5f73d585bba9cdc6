"""Regularised and overloaded VP on the GPU (lambda > 0, Alg. 2 "Regularize &
factorize", Section III-A-1), element by element against the FP64 oracle's
regularised path, through the C-ABI."""
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


CASES = [(4, 4, 16, 16, 0.3), (6, 6, 64, 40, 1.2), (8, 4, 4, 64, 0.5), (12, 8, 16, 64, 0.4),
         (16, 16, 256, 256, 0.2), (16, 8, 4, 128, 0.6)]


@pytest.mark.parametrize("K,M,qam,n,lam", CASES)
@pytest.mark.parametrize("fp64", [False, True])
def test_regularised_vs_oracle(orc, K, M, qam, n, lam, fp64):
    rng = W.rng_for(95, K * 100 + M * 10 + int(fp64))
    C, S = 40, 3
    H = W.channels(rng, C, K, M)
    sym = W.symbols(rng, C * S, K, qam)
    off = W.vec_offsets_uniform(C, S)
    gpu = run_gpu(H, sym, off, qam, n, lam=lam, fp64_threshold=0.0 if fp64 else None)
    ref = orc.precode_batch(H, sym, off, qam, n, lam=lam, nthreads=orc.max_threads())
    assert np.all(ref["status"] == 0)
    assert np.all((gpu["status"] & 3) == 0)
    if fp64:
        assert np.all(gpu["status"] == vp.VP_CH_FP64)
    # P = H^H (H H^H + lambda^2 I)^-1 (RZF)
    for c in range(C):
        Hc = H[c].astype(np.complex128)
        Pn = Hc.conj().T @ np.linalg.inv(Hc @ Hc.conj().T + lam * lam * np.eye(K))
        assert np.linalg.norm(gpu["P"][c] - Pn) <= 2e-5 * np.linalg.norm(Pn), c
    st = compare(orc, H, sym, off, qam, gpu, ref, lam=lam)
    print(K, M, lam, fp64, st)
    assert_parity(st)
    assert np.all(np.linalg.norm(gpu["x"], axis=1) < 1.0)


def test_lambda_change_refactorises(orc):
    """Setting lambda on a plan drops its channels; the next factorisation uses it."""
    K = M = 4
    rng = W.rng_for(96, 0)
    H = W.channels(rng, 8, K, M)
    sym = W.symbols(rng, 8, K, 16)
    dev = torch.device("cuda:0")
    Hd, sd = torch.from_numpy(H).to(dev), torch.from_numpy(sym).to(dev)
    x = torch.empty((8, M), dtype=torch.complex64, device=dev)
    l = torch.empty((8, K, 2), dtype=torch.int8, device=dev)
    g = torch.empty((8,), dtype=torch.float32, device=dev)
    with vp.Plan(K, M, 16, 16) as plan:
        vp.vp_factorize(plan.handle, Hd, 8)
        vp.vp_plan_set_lambda(plan.handle, 0.7)
        with pytest.raises(vp.VPError) as e:
            vp.vp_precode(plan.handle, sd, 1, None, 8, x, l, g)
        assert e.value.code == 5
        vp.vp_factorize(plan.handle, Hd, 8)
        vp.vp_precode(plan.handle, sd, 1, None, 8, x, l, g)
        torch.cuda.synchronize()
    ref = orc.precode_batch(H, sym, W.vec_offsets_uniform(8, 1), 16, 16, lam=0.7)
    gpu = {"x": x.cpu().numpy(), "l": l.cpu().numpy(), "gamma": g.cpu().numpy().astype(np.float64)}
    assert_parity(compare(orc, H, sym, W.vec_offsets_uniform(8, 1), 16, gpu, ref, lam=0.7))
