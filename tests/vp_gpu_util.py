"""Helpers shared by the GPU parity tests: run the CUDA path through the C-ABI
and compare it element by element with the FP64 oracle.

Tolerances (from the problem statement for this precoder): the integer
perturbation l must be identical on >= 99.9% of vectors; gamma within 1e-5
relative and x within 1e-5 relative (2-norm, ||x|| = 1). Where l differs the
two candidates must be a near-tie: the oracle's own gamma at the GPU's l is
within 1e-5 of its optimum, and the GPU's x matches the oracle's x at the
GPU's l.
"""
import numpy as np
import torch

import paper_2602_12098_gb300 as vp

L_MATCH_MIN = 0.999
GAMMA_RTOL = 1e-5
X_RTOL = 1e-5


def run_gpu(H, sym, vec_off, qam, n, tau=0.0, fp64_threshold=None, want_factor=True, uniform_S=None, lam=0.0,
            demap=0, frac_bits=0, tensor_product=0):
    """Whole path on cuda:0 through the C-ABI. Returns numpy outputs."""
    dev = torch.device("cuda:0")
    C, K, M = H.shape
    V = sym.shape[0]
    Hd = torch.from_numpy(np.ascontiguousarray(H)).to(dev)
    symd = torch.from_numpy(np.ascontiguousarray(sym)).to(dev)
    offd = None if uniform_S is not None else torch.from_numpy(np.ascontiguousarray(vec_off, dtype=np.int32)).to(dev)
    x = torch.empty((V, M), dtype=torch.complex64, device=dev)
    l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
    g = torch.empty((V,), dtype=torch.float32, device=dev)
    U = torch.zeros((C, K, K), dtype=torch.complex64, device=dev) if want_factor else None
    P = torch.zeros((C, M, K), dtype=torch.complex64, device=dev) if want_factor else None
    ul = torch.zeros((C, K), dtype=torch.uint8, device=dev) if want_factor else None
    st = torch.zeros((C,), dtype=torch.uint8, device=dev)
    codes = torch.zeros((C, n), dtype=torch.int64, device=dev)
    with vp.Plan(K, M, qam, n, tau, fp64_threshold, lam=lam, demap=demap, frac_bits=frac_bits,
                 tensor_product=tensor_product) as plan:
        vp.vp_factorize(plan.handle, Hd, C, U, P, ul, st)
        if uniform_S is not None:
            vp.vp_precode(plan.handle, symd, uniform_S, None, V, x, l, g)
        else:
            vp.vp_precode(plan.handle, symd, 0, offd, V, x, l, g)
        vp.vp_get_paths(plan.handle, codes)
        torch.cuda.synchronize()
    out = {"x": x.cpu().numpy(), "l": l.cpu().numpy(), "gamma": g.cpu().numpy().astype(np.float64),
           "status": st.cpu().numpy(), "codes": codes.cpu().numpy().view(np.uint64)}
    if want_factor:
        out.update(U=U.cpu().numpy(), P=P.cpu().numpy(), ul=ul.cpu().numpy())
    return out


def oracle_x_at(orc, H, qam, tau, l_user, sym_user, lam=0.0):
    """Oracle x and gamma for a GIVEN perturbation (user order), from its factor."""
    f = orc.factor_channel(H.astype(np.complex128), 1, lam)
    ul = f["user_of_level"]
    s = orc.qam_points(qam, sym_user)
    u = s + tau * (l_user[:, 0] + 1j * l_user[:, 1])
    z = f["Rt"] @ u[ul]
    gam = float(np.real(np.vdot(z, z)))
    w = f["Qbar"][:, :H.shape[1]].conj().T @ z
    return w / np.sqrt(gam), gam


def compare(orc, H, sym, vec_off, qam, gpu, ref, tau=None, lam=0.0):
    """Element-wise comparison; returns a stats dict (asserts nothing)."""
    tau = orc.default_tau(qam) if tau is None else tau
    V = sym.shape[0]
    ch_of = np.repeat(np.arange(len(vec_off) - 1), np.diff(vec_off))
    l_eq = np.all(gpu["l"] == ref["l"], axis=(1, 2))
    st = {"V": V, "l_match": float(l_eq.mean()) if V else 1.0, "n_l_diff": int((~l_eq).sum()),
          "gamma_rel_max": 0.0, "x_err_max": 0.0, "tie_gamma_rel_max": 0.0, "tie_x_err_max": 0.0}
    good = ref["gamma"] > 0
    if np.any(l_eq & good):
        m = l_eq & good
        st["gamma_rel_max"] = float(np.max(np.abs(gpu["gamma"][m] - ref["gamma"][m]) / ref["gamma"][m]))
        st["x_err_max"] = float(np.max(np.linalg.norm(gpu["x"][m] - ref["x"][m], axis=1)))
    for v in np.nonzero(~l_eq & good)[0]:
        c = ch_of[v]
        xg, gg = oracle_x_at(orc, H[c], qam, tau, gpu["l"][v].astype(np.int64), sym[v], lam)
        st["tie_gamma_rel_max"] = max(st["tie_gamma_rel_max"], (gg - ref["gamma"][v]) / ref["gamma"][v])
        st["tie_x_err_max"] = max(st["tie_x_err_max"], float(np.linalg.norm(gpu["x"][v] - xg)))
        st["gamma_rel_max"] = max(st["gamma_rel_max"], abs(gpu["gamma"][v] - gg) / gg)
    return st


def assert_parity(st, l_match_min=L_MATCH_MIN):
    assert st["l_match"] >= l_match_min, st
    assert st["gamma_rel_max"] <= GAMMA_RTOL, st
    assert st["x_err_max"] <= X_RTOL, st
    assert st["tie_gamma_rel_max"] <= GAMMA_RTOL, st
    assert st["tie_x_err_max"] <= X_RTOL, st
