"""GB300-native vector-perturbation precoding (ViPer NL-COMM hot path).

Thin ctypes binding of libvp (``include/vp.h``): the functions below have the
C-ABI's names and only marshal arguments (tensor -> device pointer, stream ->
handle, status code -> exception). Every step of the precoder runs in the
CUDA kernels of ``csrc/``; there is no CPU fallback, and a missing or
unloadable library raises.

Arguments that the C-ABI takes as device pointers accept torch CUDA tensors
(or raw integer addresses); host pointers accept numpy arrays or pinned torch
CPU tensors; ``stream`` accepts a torch.cuda.Stream, a raw handle, or None
(torch's current stream when torch is importable, else the default stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = [
    "VPError", "load", "build", "library_path",
    "vp_plan_create", "vp_plan_set_fp64_threshold", "vp_plan_destroy", "vp_factorize", "vp_precode",
    "vp_get_paths", "vp_run_slot_host", "vp_last_launch_count", "vp_status_string",
    "vp_precode_noalloc", "vp_noalloc_capacity_bytes", "VP_CH_NONFINITE", "VP_CH_SINGULAR", "VP_CH_FP64", "VP_MAX_K", "VP_MAX_M", "VP_MAX_PATHS",
    "EXPORTED_SYMBOLS", "Plan",
]

VP_CH_NONFINITE = 1
VP_CH_SINGULAR = 2
VP_CH_FP64 = 4
VP_MAX_K = 16
VP_MAX_M = 16
VP_MAX_PATHS = 1024

EXPORTED_SYMBOLS = (
    "vp_plan_create", "vp_plan_set_fp64_threshold", "vp_plan_destroy", "vp_factorize", "vp_precode",
    "vp_get_paths", "vp_run_slot_host", "vp_last_launch_count", "vp_status_string",
    "vp_precode_noalloc", "vp_noalloc_capacity_bytes",
)

_lock = threading.Lock()
_lib = None


class VPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        super().__init__(f"{where}: {vp_status_string(code)} (status {code})")


def library_path() -> str:
    return _build.LIB


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load():
    """Load libvp.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise ImportError(f"libvp.so not found at {path}")
            L = ctypes.CDLL(path)
            vpp = ctypes.c_void_p
            L.vp_plan_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                         ctypes.POINTER(vpp)]
            L.vp_plan_set_fp64_threshold.argtypes = [vpp, ctypes.c_float]
            L.vp_plan_destroy.argtypes = [vpp]
            L.vp_factorize.argtypes = [vpp, vpp, ctypes.c_int, vpp, vpp, vpp, vpp, vpp]
            L.vp_precode.argtypes = [vpp, vpp, ctypes.c_int, vpp, ctypes.c_int, vpp, vpp, vpp, vpp]
            L.vp_get_paths.argtypes = [vpp, vpp, vpp]
            L.vp_run_slot_host.argtypes = [vpp, vpp, ctypes.c_int, vpp, ctypes.c_int, vpp, vpp, vpp, vpp]
            L.vp_last_launch_count.argtypes = [vpp]
            L.vp_last_launch_count.restype = ctypes.c_int
            L.vp_precode_noalloc.argtypes = [vpp, vpp, ctypes.c_int, vpp, ctypes.c_int, vpp, vpp, vpp, vpp, vpp]
            L.vp_noalloc_capacity_bytes.argtypes = []
            L.vp_noalloc_capacity_bytes.restype = ctypes.c_size_t
            L.vp_status_string.argtypes = [ctypes.c_int]
            L.vp_status_string.restype = ctypes.c_char_p
            for name in ("vp_plan_create", "vp_plan_set_fp64_threshold", "vp_plan_destroy", "vp_factorize",
                         "vp_precode", "vp_get_paths", "vp_run_slot_host", "vp_precode_noalloc"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _addr(a):
    """Pointer of a tensor / numpy array / integer address / None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a).__name__}")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(code: int, where: str):
    if code != 0:
        raise VPError(code, where)


def vp_status_string(code: int) -> str:
    return load().vp_status_string(int(code)).decode()


def vp_plan_create(K: int, M: int, qam: int, n_paths: int, tau: float = 0.0) -> int:
    out = ctypes.c_void_p()
    _check(load().vp_plan_create(K, M, qam, n_paths, float(tau), ctypes.byref(out)), "vp_plan_create")
    return out.value


def vp_plan_set_fp64_threshold(plan: int, kappa_hat: float) -> None:
    _check(load().vp_plan_set_fp64_threshold(plan, float(kappa_hat)), "vp_plan_set_fp64_threshold")


def vp_plan_destroy(plan: int) -> None:
    _check(load().vp_plan_destroy(plan), "vp_plan_destroy")


def vp_factorize(plan: int, H, C: int, U=None, P=None, user_of_level=None, status=None, stream=None) -> None:
    _check(load().vp_factorize(plan, _addr(H), int(C), _addr(U), _addr(P), _addr(user_of_level), _addr(status),
                               _stream(stream)), "vp_factorize")


def vp_precode(plan: int, sym_idx, S: int, vec_offsets, n_vec: int, x, l, gamma, stream=None) -> None:
    _check(load().vp_precode(plan, _addr(sym_idx), int(S), _addr(vec_offsets), int(n_vec), _addr(x), _addr(l),
                             _addr(gamma), _stream(stream)), "vp_precode")


def vp_get_paths(plan: int, codes, stream=None) -> None:
    _check(load().vp_get_paths(plan, _addr(codes), _stream(stream)), "vp_get_paths")


def vp_run_slot_host(plan: int, H_host, C: int, sym_host, S: int, x_host, l_host=None, gamma_host=None,
                     stream=None) -> None:
    _check(load().vp_run_slot_host(plan, _addr(H_host), int(C), _addr(sym_host), int(S), _addr(x_host),
                                   _addr(l_host), _addr(gamma_host), _stream(stream)), "vp_run_slot_host")


def vp_precode_noalloc(plan: int, H, C: int, sym_idx, S: int, x, l, gamma, status=None, stream=None) -> None:
    """One slot without any allocation (state in the library's static device array)."""
    _check(load().vp_precode_noalloc(plan, _addr(H), int(C), _addr(sym_idx), int(S), _addr(x), _addr(l),
                                     _addr(gamma), _addr(status), _stream(stream)), "vp_precode_noalloc")


def vp_noalloc_capacity_bytes() -> int:
    return int(load().vp_noalloc_capacity_bytes())


def vp_last_launch_count(plan: int) -> int:
    return int(load().vp_last_launch_count(plan))


class Plan:
    """Owning handle of a vp_plan (destroys it on close / exit of a with-block)."""

    def __init__(self, K: int, M: int, qam: int, n_paths: int, tau: float = 0.0,
                 fp64_threshold: float | None = None):
        self.K, self.M, self.qam, self.n_paths = K, M, qam, n_paths
        self.handle = vp_plan_create(K, M, qam, n_paths, tau)
        if fp64_threshold is not None:
            vp_plan_set_fp64_threshold(self.handle, fp64_threshold)

    def close(self):
        if self.handle:
            vp_plan_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
