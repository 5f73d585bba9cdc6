"""The region-LUT DEMAP variant (VP_DEMAP_LUT, Section III-A-2) on the GPU,
element by element against the oracle's LUT DEMAP, through the C-ABI."""
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


@pytest.mark.parametrize("wl,sub", [(W.SMALL_4x4, None), (W.RB_8x8, 24 * 12 + 6), (W.SLOT_16x16, 40)])
def test_lut_demap_vs_oracle(orc, wl, sub):
    b = W.make_batch(wl, subcarriers=sub)
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, demap=vp.VP_DEMAP_LUT, want_factor=False)
    ref = orc.precode_batch(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, nthreads=orc.max_threads(), demap="lut")
    st = compare(orc, b.H, b.sym, b.vec_off, wl.qam, gpu, ref)
    print(wl.name, st)
    assert_parity(st)


def test_lut_demap_full_slot_sampled(orc):
    wl = W.SLOT_16x16
    b = W.make_batch(wl)
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, demap=vp.VP_DEMAP_LUT, want_factor=False,
                  uniform_S=wl.symbols)
    rng = np.random.default_rng(11)
    chans = np.sort(rng.choice(b.H.shape[0], 40, replace=False))
    vecs = np.concatenate([np.arange(b.vec_off[c], b.vec_off[c + 1])[:4] for c in chans])
    off = np.arange(len(chans) + 1, dtype=np.int32) * 4
    ref = orc.precode_batch(b.H[chans], b.sym[vecs], off, wl.qam, wl.n_paths, nthreads=orc.max_threads(), demap="lut")
    sub = {k: gpu[k][vecs] for k in ("x", "l", "gamma")}
    assert_parity(compare(orc, b.H[chans], b.sym[vecs], off, wl.qam, sub, ref))
    # the exact DEMAP on the same slot: the LUT's gamma is never far above it
    ex = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, want_factor=False, uniform_S=wl.symbols)
    m = ex["gamma"] > 0
    ratio = gpu["gamma"][m] / ex["gamma"][m]
    print("gamma lut / exact: mean %.5f max %.4f" % (ratio.mean(), ratio.max()))
    assert ratio.mean() < 1.01
