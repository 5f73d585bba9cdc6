"""The fixed-point search (vp_plan_set_fixed_point: Section IV's 16-bit words
with F fractional bits) on the GPU, element by element against the oracle's
fixed-point search, through the C-ABI.

With every channel on the FP64 factor (threshold 0) both sides round the same
U~ entries to words (up to the FP32 storage of the factor), and from there
the word arithmetic and DEMAP are exact on both; what remains are FP32 PED
sums against FP64 ones, and entries within an FP32 rounding of a half-word.
Where l differs the GPU's gamma and x must still be the exact ones of its own
l, and the oracle's gamma there is within a relative 2^(4-F) of its optimum
(a near-tie of the word-quantised metric, whose rounding is ~2^-F relative).
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


def assert_fixed_parity(st, F):
    assert st["l_match"] >= L_MATCH_MIN, st
    assert st["gamma_rel_max"] <= GAMMA_RTOL, st
    assert st["x_err_max"] <= X_RTOL, st
    assert st["tie_x_err_max"] <= X_RTOL, st
    assert st["tie_gamma_rel_max"] <= 2.0 ** (4 - F), st


@pytest.mark.parametrize("wl,sub,F", [(W.SMALL_4x4, None, 8), (W.SMALL_4x4, None, 13), (W.RB_8x8, 24 * 12 + 6, 11),
                                      (W.RB_8x8, 24 * 12 + 6, 13), (W.SLOT_16x16, 40, 8), (W.SLOT_16x16, 40, 11)])
def test_fixed_point_vs_oracle(orc, wl, sub, F):
    b = W.make_batch(wl, subcarriers=sub)
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, fp64_threshold=0.0, frac_bits=F, want_factor=False)
    ref = orc.precode_batch(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, nthreads=orc.max_threads(), frac_bits=F,
                            word_bits=16)
    assert np.all(gpu["status"] == vp.VP_CH_FP64)
    st = compare(orc, b.H, b.sym, b.vec_off, wl.qam, gpu, ref)
    print(wl.name, F, st)
    assert_fixed_parity(st, F)


def test_fixed_point_full_slot_sampled(orc):
    """The 16 x 16 slot at full size, F = 9 (the word length that comes closest
    to the floating-point search on this slot: with more fractional bits the
    +-2^(15-F) range saturates); sampled vectors against the oracle, and the
    whole slot against the floating-point search."""
    wl, F = W.SLOT_16x16, 9
    b = W.make_batch(wl)
    gpu = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, fp64_threshold=0.0, frac_bits=F, want_factor=False,
                  uniform_S=wl.symbols)
    rng = np.random.default_rng(12)
    chans = np.sort(rng.choice(b.H.shape[0], 40, replace=False))
    vecs = np.concatenate([np.arange(b.vec_off[c], b.vec_off[c + 1])[:4] for c in chans])
    off = np.arange(len(chans) + 1, dtype=np.int32) * 4
    ref = orc.precode_batch(b.H[chans], b.sym[vecs], off, wl.qam, wl.n_paths, nthreads=orc.max_threads(),
                            frac_bits=F, word_bits=16)
    sub = {k: gpu[k][vecs] for k in ("x", "l", "gamma")}
    assert_fixed_parity(compare(orc, b.H[chans], b.sym[vecs], off, wl.qam, sub, ref), F)
    fl = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, fp64_threshold=0.0, want_factor=False,
                 uniform_S=wl.symbols)
    m = fl["gamma"] > 0
    ratio = gpu["gamma"][m] / fl["gamma"][m]
    print("gamma fixed(F=9) / float: mean %.6f max %.4f, l differs on %.4f" %
          (ratio.mean(), ratio.max(), np.mean(np.any(gpu["l"] != fl["l"], axis=(1, 2)))))
    assert ratio.mean() < 1.01
    assert np.allclose(np.linalg.norm(gpu["x"], axis=1), 1.0, atol=1e-5)


def test_fixed_point_plan_switches_back():
    """frac_bits = 0 restores the floating-point search on the same plan."""
    wl = W.RB_8x8
    b = W.make_batch(wl, subcarriers=48)
    a = run_gpu(b.H, b.sym, b.vec_off, wl.qam, wl.n_paths, want_factor=False)
    dev = torch.device("cuda:0")
    C, K, M = b.H.shape
    V = b.sym.shape[0]
    H = torch.from_numpy(b.H).to(dev)
    sym = torch.from_numpy(b.sym).to(dev)
    off = torch.from_numpy(b.vec_off).to(dev)
    outs = []
    with vp.Plan(K, M, wl.qam, wl.n_paths) as plan:
        vp.vp_factorize(plan.handle, H, C)
        for f in (9, 0):
            vp.vp_plan_set_fixed_point(plan.handle, f)
            x = torch.empty((V, M), dtype=torch.complex64, device=dev)
            l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
            g = torch.empty((V,), dtype=torch.float32, device=dev)
            vp.vp_precode(plan.handle, sym, 0, off, V, x, l, g)
            outs.append((x.cpu().numpy(), l.cpu().numpy(), g.cpu().numpy()))
    assert np.array_equal(outs[1][1], a["l"]) and np.array_equal(outs[1][0], a["x"])
    assert not np.array_equal(outs[0][1], outs[1][1])
