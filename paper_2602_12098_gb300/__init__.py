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
    "vp_plan_create", "vp_plan_set_fp64_threshold", "vp_plan_set_lambda", "vp_plan_set_demap",
    "vp_plan_set_fixed_point", "vp_plan_destroy", "vp_factorize", "vp_precode", "vp_get_paths", "vp_run_slot_host",
    "vp_last_launch_count", "vp_status_string",
    "vp_precode_noalloc", "vp_noalloc_capacity_bytes", "vp_noalloc_max_channels", "vp_problem_desc",
    "vp_plan_set_tensor_product", "vp_batch_create", "VP_DEMAP_EXACT", "VP_DEMAP_LUT",
    "vp_batch_workspace_bytes", "vp_batch_bind", "vp_batch_launch", "vp_batch_launch_count", "vp_batch_destroy",
    "vp_precode_batch", "vp_precode_batch_workspace_bytes", "problem_desc", "packed_descs", "Batch", "VP_CH_NONFINITE", "VP_CH_SINGULAR", "VP_CH_FP64", "VP_MAX_K", "VP_MAX_M", "VP_MAX_PATHS",
    "vp_job_desc", "vp_job_done", "vp_server_stats", "vp_server_create", "vp_server_submit", "vp_server_poll",
    "vp_server_drain", "vp_server_reset_clock", "vp_server_get_stats", "vp_server_destroy", "Server",
    "vp_batch_autotune", "vp_batch_get_tuning", "vp_batch_set_tuning", "vp_batch_group_info",
    "vp_server_create_fake", "vp_batch_set_persistent", "EXPORTED_SYMBOLS", "Plan",
    "vp_server_set_policy", "vp_server_replay", "VP_SERVE_FCFS", "VP_SERVE_AGE_PRIORITY", "vp_batch_set_concurrent",
]

VP_CH_NONFINITE = 1
VP_CH_SINGULAR = 2
VP_CH_FP64 = 4
VP_MAX_K = 16
VP_MAX_M = 16
VP_MAX_PATHS = 1024

VP_DEMAP_EXACT = 0
VP_DEMAP_LUT = 1

VP_SERVE_FCFS = 0
VP_SERVE_AGE_PRIORITY = 1

EXPORTED_SYMBOLS = (
    "vp_plan_create", "vp_plan_set_fp64_threshold", "vp_plan_set_lambda", "vp_plan_set_demap",
    "vp_plan_set_fixed_point", "vp_plan_destroy",
    "vp_factorize",
    "vp_precode",
    "vp_get_paths", "vp_run_slot_host", "vp_last_launch_count", "vp_status_string",
    "vp_precode_noalloc", "vp_noalloc_capacity_bytes", "vp_noalloc_max_channels", "vp_plan_set_tensor_product",
    "vp_batch_create",
    "vp_batch_workspace_bytes",
    "vp_batch_bind", "vp_batch_launch", "vp_batch_launch_count", "vp_batch_destroy", "vp_precode_batch",
    "vp_precode_batch_workspace_bytes", "vp_server_create", "vp_server_submit", "vp_server_poll", "vp_server_drain",
    "vp_server_reset_clock", "vp_server_get_stats", "vp_server_destroy", "vp_batch_autotune", "vp_batch_get_tuning",
    "vp_batch_set_tuning", "vp_batch_group_info", "vp_server_create_fake", "vp_batch_set_persistent",
    "vp_server_set_policy", "vp_server_replay", "vp_batch_set_concurrent",
)


class vp_problem_desc(ctypes.Structure):
    """One problem of an uneven batch (layout of the C struct)."""
    _fields_ = [("K", ctypes.c_int), ("M", ctypes.c_int), ("qam", ctypes.c_int), ("n_paths", ctypes.c_int),
                ("tau", ctypes.c_float), ("S", ctypes.c_int), ("H", ctypes.c_void_p), ("sym_idx", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("l", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


class vp_job_desc(ctypes.Structure):
    """One job of the server: a slot of one plan shape (layout of the C struct)."""
    _fields_ = [("K", ctypes.c_int), ("M", ctypes.c_int), ("qam", ctypes.c_int), ("n_paths", ctypes.c_int),
                ("tau", ctypes.c_float), ("lam", ctypes.c_float), ("fp64_threshold", ctypes.c_float),
                ("demap", ctypes.c_int), ("frac_bits", ctypes.c_int), ("C", ctypes.c_int), ("S", ctypes.c_int),
                ("H", ctypes.c_void_p), ("sym_idx", ctypes.c_void_p), ("x", ctypes.c_void_p), ("l", ctypes.c_void_p),
                ("gamma", ctypes.c_void_p), ("status", ctypes.c_void_p), ("ready_event", ctypes.c_void_p)]


class vp_job_done(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("admit_ms", ctypes.c_float),
                ("end_ms", ctypes.c_float), ("rank", ctypes.c_int)]


class vp_server_stats(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int), ("queued", ctypes.c_int), ("in_flight", ctypes.c_int),
                ("max_in_flight", ctypes.c_int), ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("pool_bytes", ctypes.c_size_t), ("pool_used", ctypes.c_size_t), ("pool_high_water", ctypes.c_size_t)]


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
            L.vp_plan_set_lambda.argtypes = [vpp, ctypes.c_float]
            L.vp_plan_set_demap.argtypes = [vpp, ctypes.c_int]
            L.vp_plan_set_fixed_point.argtypes = [vpp, ctypes.c_int]
            L.vp_plan_set_tensor_product.argtypes = [vpp, ctypes.c_int]
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
            L.vp_noalloc_max_channels.argtypes = [vpp]
            L.vp_noalloc_max_channels.restype = ctypes.c_int
            descp = ctypes.POINTER(vp_problem_desc)
            L.vp_batch_create.argtypes = [descp, ctypes.c_int, ctypes.c_float, ctypes.POINTER(vpp)]
            L.vp_batch_workspace_bytes.argtypes = [vpp]
            L.vp_batch_workspace_bytes.restype = ctypes.c_size_t
            L.vp_batch_bind.argtypes = [vpp, vpp, ctypes.c_size_t, vpp]
            L.vp_batch_launch.argtypes = [vpp, vpp]
            L.vp_batch_set_persistent.argtypes = [vpp, ctypes.c_int]
            L.vp_batch_set_persistent.restype = ctypes.c_int
            L.vp_batch_set_concurrent.argtypes = [vpp, ctypes.c_int]
            L.vp_batch_set_concurrent.restype = ctypes.c_int
            L.vp_batch_launch_count.argtypes = [vpp]
            L.vp_batch_launch_count.restype = ctypes.c_int
            L.vp_batch_destroy.argtypes = [vpp]
            L.vp_precode_batch.argtypes = [descp, ctypes.c_int, ctypes.c_size_t, vpp, vpp]
            L.vp_precode_batch_workspace_bytes.argtypes = [descp, ctypes.c_int]
            L.vp_precode_batch_workspace_bytes.restype = ctypes.c_size_t
            sp = ctypes.c_void_p
            L.vp_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(sp)]
            L.vp_server_create_fake.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(sp)]
            L.vp_server_create_fake.restype = ctypes.c_int
            L.vp_server_submit.argtypes = [sp, ctypes.POINTER(vp_job_desc), ctypes.POINTER(ctypes.c_int64)]
            L.vp_server_poll.argtypes = [sp, ctypes.POINTER(vp_job_done), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            L.vp_server_drain.argtypes = [sp, ctypes.c_double]
            L.vp_server_reset_clock.argtypes = [sp]
            L.vp_server_get_stats.argtypes = [sp, ctypes.POINTER(vp_server_stats)]
            L.vp_server_destroy.argtypes = [sp]
            L.vp_server_set_policy.argtypes = [sp, ctypes.c_int]
            L.vp_server_replay.argtypes = [sp, ctypes.POINTER(vp_job_desc), ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_int, ctypes.c_double, ctypes.POINTER(vp_job_done),
                                           ctypes.POINTER(ctypes.c_double)]
            for name in ("vp_server_create", "vp_server_submit", "vp_server_poll", "vp_server_drain",
                         "vp_server_reset_clock", "vp_server_get_stats", "vp_server_destroy",
                         "vp_server_set_policy", "vp_server_replay"):
                getattr(L, name).restype = ctypes.c_int
            L.vp_batch_autotune.argtypes = [vpp, ctypes.c_int, vpp]
            L.vp_batch_autotune.restype = ctypes.c_int
            ip = ctypes.POINTER(ctypes.c_int)
            L.vp_batch_get_tuning.argtypes = [vpp, ip, ctypes.c_int]
            L.vp_batch_get_tuning.restype = ctypes.c_int
            L.vp_batch_set_tuning.argtypes = [vpp, ip, ctypes.c_int]
            L.vp_batch_set_tuning.restype = ctypes.c_int
            L.vp_batch_group_info.argtypes = [vpp, ip, ctypes.c_int]
            L.vp_batch_group_info.restype = ctypes.c_int
            L.vp_status_string.argtypes = [ctypes.c_int]
            L.vp_status_string.restype = ctypes.c_char_p
            for name in ("vp_plan_create", "vp_plan_set_fp64_threshold", "vp_plan_set_lambda", "vp_plan_set_demap",
                         "vp_plan_set_fixed_point", "vp_plan_set_tensor_product", "vp_plan_destroy",
                         "vp_factorize",
                         "vp_precode", "vp_get_paths", "vp_run_slot_host", "vp_precode_noalloc", "vp_batch_create",
                         "vp_batch_bind", "vp_batch_launch", "vp_batch_destroy", "vp_precode_batch"):
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


def vp_plan_set_lambda(plan: int, lam: float) -> None:
    _check(load().vp_plan_set_lambda(plan, float(lam)), "vp_plan_set_lambda")


def vp_plan_set_demap(plan: int, demap: int) -> None:
    _check(load().vp_plan_set_demap(plan, int(demap)), "vp_plan_set_demap")


def vp_plan_set_fixed_point(plan: int, frac_bits: int) -> None:
    _check(load().vp_plan_set_fixed_point(plan, int(frac_bits)), "vp_plan_set_fixed_point")


def vp_plan_set_tensor_product(plan: int, enable: int) -> None:
    _check(load().vp_plan_set_tensor_product(plan, int(enable)), "vp_plan_set_tensor_product")


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


def vp_noalloc_max_channels(plan: int) -> int:
    """Largest channel count vp_precode_noalloc accepts for the plan's shape."""
    return int(load().vp_noalloc_max_channels(plan))


def vp_last_launch_count(plan: int) -> int:
    return int(load().vp_last_launch_count(plan))


def _desc_array(descs):
    if isinstance(descs, ctypes.Array):
        return descs
    arr = (vp_problem_desc * len(descs))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def vp_batch_create(descs, fp64_threshold: float = 1e4) -> int:
    arr = _desc_array(descs)
    out = ctypes.c_void_p()
    _check(load().vp_batch_create(arr, len(arr), float(fp64_threshold), ctypes.byref(out)), "vp_batch_create")
    return out.value


def vp_batch_workspace_bytes(batch: int) -> int:
    return int(load().vp_batch_workspace_bytes(batch))


def vp_batch_bind(batch: int, workspace, workspace_bytes: int, stream=None) -> None:
    _check(load().vp_batch_bind(batch, _addr(workspace), int(workspace_bytes), _stream(stream)), "vp_batch_bind")


def vp_batch_launch(batch: int, stream=None) -> None:
    _check(load().vp_batch_launch(batch, _stream(stream)), "vp_batch_launch")


def vp_batch_launch_count(batch: int) -> int:
    return int(load().vp_batch_launch_count(batch))


def vp_batch_destroy(batch: int) -> None:
    _check(load().vp_batch_destroy(batch), "vp_batch_destroy")


def vp_precode_batch(descs, workspace, workspace_bytes: int, stream=None) -> None:
    arr = _desc_array(descs)
    _check(load().vp_precode_batch(arr, len(arr), int(workspace_bytes), _addr(workspace), _stream(stream)),
           "vp_precode_batch")


def vp_precode_batch_workspace_bytes(descs) -> int:
    arr = _desc_array(descs)
    return int(load().vp_precode_batch_workspace_bytes(arr, len(arr)))


def problem_desc(K, M, qam, n_paths, H, sym_idx, x, l, gamma, status=None, tau=0.0, S=None) -> vp_problem_desc:
    """Descriptor of one problem from tensors (S defaults to sym_idx's row count)."""
    S = int(sym_idx.shape[0]) if S is None else int(S)
    return vp_problem_desc(int(K), int(M), int(qam), int(n_paths), float(tau), S, _addr(H), _addr(sym_idx),
                           _addr(x), _addr(l), _addr(gamma), _addr(status))


def packed_descs(pk, H, sym, x, l, gamma, status=None, tau=0.0):
    """Descriptors of packed problems (workloads.PackedProblems) whose flat
    arrays live in the given device tensors (H, x complex64; sym uint8; l int8;
    gamma float32; status uint8 [N] or None)."""
    n = len(pk.K)
    arr = (vp_problem_desc * n)()
    hb, sb, xb, lb, gb = _addr(H), _addr(sym), _addr(x), _addr(l), _addr(gamma)
    stb = _addr(status)
    for i in range(n):
        S = int(pk.S[i])
        arr[i] = vp_problem_desc(int(pk.K[i]), int(pk.M[i]), int(pk.qam[i]), int(pk.n_paths[i]), float(tau), S,
                                 hb + 8 * int(pk.H_off[i]), sb + int(pk.sym_off[i]) if S else None,
                                 xb + 8 * int(pk.x_off[i]) if S else None, lb + int(pk.l_off[i]) if S else None,
                                 gb + 4 * int(pk.g_off[i]) if S else None, stb + i if stb else None)
    return arr


class Batch:
    """Owning handle of a vp_batch and its device workspace (a torch uint8 tensor)."""

    def __init__(self, descs, fp64_threshold: float = 1e4, stream=None, persistent: int = 0, concurrent: int = 1):
        import torch
        self.descs = _desc_array(descs)
        self.handle = vp_batch_create(self.descs, fp64_threshold)
        if persistent:
            vp_batch_set_persistent(self.handle, persistent)
        if not concurrent:
            vp_batch_set_concurrent(self.handle, 0)
        nbytes = vp_batch_workspace_bytes(self.handle)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        self.ws_addr = (base + 255) // 256 * 256
        vp_batch_bind(self.handle, self.ws_addr, nbytes, stream)
        self.launches = vp_batch_launch_count(self.handle)

    def launch(self, stream=None):
        vp_batch_launch(self.handle, stream)

    def autotune(self, reps: int = 3, cache: str | None = None, stream=None) -> list:
        """Tune the launch mapping (vp_batch_autotune) or take it from a JSON
        cache keyed by device name and group shapes; cache = None uses
        $VP_TUNE_CACHE when set. Returns the knobs in force."""
        import json
        import torch
        cache = cache if cache is not None else os.environ.get("VP_TUNE_CACHE")
        key = tuning_key(self.handle, torch.cuda.get_device_name())
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                vp_batch_set_tuning(self.handle, table[key])
                return table[key]
        vp_batch_autotune(self.handle, reps, stream)
        knobs = vp_batch_get_tuning(self.handle)
        if cache:
            table[key] = knobs
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1)
            os.replace(tmp, cache)
        return knobs

    def close(self):
        if self.handle:
            vp_batch_destroy(self.handle)
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


def vp_batch_set_persistent(batch: int, persistent: int) -> None:
    _check(load().vp_batch_set_persistent(batch, int(persistent)), "vp_batch_set_persistent")


def vp_batch_set_concurrent(batch: int, concurrent: int) -> None:
    _check(load().vp_batch_set_concurrent(batch, int(concurrent)), "vp_batch_set_concurrent")


def vp_batch_autotune(batch: int, reps: int = 3, stream=None) -> None:
    _check(load().vp_batch_autotune(batch, int(reps), _stream(stream)), "vp_batch_autotune")


def vp_batch_get_tuning(batch: int) -> list:
    n = load().vp_batch_get_tuning(batch, None, 0)
    if n < 0:
        raise VPError(1, "vp_batch_get_tuning")
    buf = (ctypes.c_int * max(n, 1))()
    load().vp_batch_get_tuning(batch, buf, n)
    return [int(buf[i]) for i in range(n)]


def vp_batch_set_tuning(batch: int, knobs) -> None:
    knobs = [int(k) for k in knobs]
    buf = (ctypes.c_int * max(len(knobs), 1))(*knobs)
    _check(load().vp_batch_set_tuning(batch, buf, len(knobs)), "vp_batch_set_tuning")


def vp_batch_group_info(batch: int) -> list:
    """Per group: (stage, problems, K or K tile, M, largest n_paths, largest S)."""
    n = load().vp_batch_group_info(batch, None, 0)
    if n < 0:
        raise VPError(1, "vp_batch_group_info")
    buf = (ctypes.c_int * max(6 * n, 1))()
    load().vp_batch_group_info(batch, buf, n)
    return [tuple(int(buf[6 * i + k]) for k in range(6)) for i in range(n)]


def tuning_key(batch: int, device_name: str) -> str:
    """Cache key of a batch's tuning: the device and the groups' shapes."""
    import hashlib
    shape = ";".join(",".join(str(v) for v in g) for g in vp_batch_group_info(batch))
    return device_name + "|" + hashlib.sha256(shape.encode()).hexdigest()[:16]


def vp_server_create(pool_bytes: int, lanes: int) -> int:
    h = ctypes.c_void_p()
    _check(load().vp_server_create(int(pool_bytes), int(lanes), ctypes.byref(h)), "vp_server_create")
    return h.value


def vp_server_create_fake(pool_bytes: int, lanes: int) -> int:
    h = ctypes.c_void_p()
    _check(load().vp_server_create_fake(int(pool_bytes), int(lanes), ctypes.byref(h)), "vp_server_create_fake")
    return h.value


def vp_server_submit(server: int, job: vp_job_desc) -> int:
    i = ctypes.c_int64()
    _check(load().vp_server_submit(server, ctypes.byref(job), ctypes.byref(i)), "vp_server_submit")
    return i.value


def vp_server_poll(server: int, max_done: int = 256) -> list:
    """Finished jobs since the last poll: list of (id, status, admit_ms, end_ms, rank)."""
    buf = (vp_job_done * max(int(max_done), 1))()
    n = ctypes.c_int()
    out = []
    while True:
        _check(load().vp_server_poll(server, buf, len(buf), ctypes.byref(n)), "vp_server_poll")
        out += [(buf[i].id, buf[i].status, buf[i].admit_ms, buf[i].end_ms, buf[i].rank) for i in range(n.value)]
        if n.value < len(buf):
            return out


def vp_server_set_policy(server: int, policy: int) -> None:
    _check(load().vp_server_set_policy(server, int(policy)), "vp_server_set_policy")


def vp_server_replay(server: int, jobs: list, arrival_ms, timeout_s: float = 60.0):
    """Replay `jobs` (vp_job_desc list) at `arrival_ms` (host-clock ms from the
    clock zero). Returns (records, submit_ms): records[i] = (id, status,
    admit_ms, end_ms, rank) of job i, submit_ms[i] its submission time."""
    n = len(jobs)
    if len(arrival_ms) != n:
        raise ValueError("one arrival time per job")
    descs = (vp_job_desc * max(n, 1))(*jobs)
    arr = (ctypes.c_double * max(n, 1))(*[float(a) for a in arrival_ms])
    done = (vp_job_done * max(n, 1))()
    sub = (ctypes.c_double * max(n, 1))()
    _check(load().vp_server_replay(server, descs, arr, n, float(timeout_s), done, sub), "vp_server_replay")
    recs = [(done[i].id, done[i].status, done[i].admit_ms, done[i].end_ms, done[i].rank) for i in range(n)]
    return recs, [sub[i] for i in range(n)]


def vp_server_drain(server: int, timeout_s: float = 60.0) -> None:
    _check(load().vp_server_drain(server, float(timeout_s)), "vp_server_drain")


def vp_server_reset_clock(server: int) -> None:
    _check(load().vp_server_reset_clock(server), "vp_server_reset_clock")


def vp_server_get_stats(server: int) -> dict:
    st = vp_server_stats()
    _check(load().vp_server_get_stats(server, ctypes.byref(st)), "vp_server_get_stats")
    return {k: getattr(st, k) for k, _ in vp_server_stats._fields_}


def vp_server_destroy(server: int) -> None:
    _check(load().vp_server_destroy(server), "vp_server_destroy")


def job_desc(K, M, qam, n_paths, C, S, H, sym, x, l, gamma, status=None, tau=0.0, lam=0.0, fp64_threshold=0.0,
             demap=0, frac_bits=0, ready_event=None) -> vp_job_desc:
    """A vp_job_desc from torch device tensors (or raw addresses)."""
    return vp_job_desc(int(K), int(M), int(qam), int(n_paths), float(tau), float(lam), float(fp64_threshold),
                       int(demap), int(frac_bits), int(C), int(S), _addr(H), _addr(sym), _addr(x), _addr(l),
                       _addr(gamma), _addr(status),
                       _addr(getattr(ready_event, "cuda_event", ready_event)))


class Server:
    """Owning handle of a vp_server (destroys it on close / exit of a with-block)."""

    def __init__(self, pool_bytes: int, lanes: int = 4, fake: bool = False):
        self.handle = (vp_server_create_fake if fake else vp_server_create)(pool_bytes, lanes)

    def submit(self, job: vp_job_desc) -> int:
        return vp_server_submit(self.handle, job)

    def poll(self) -> list:
        return vp_server_poll(self.handle)

    def drain(self, timeout_s: float = 60.0) -> None:
        vp_server_drain(self.handle, timeout_s)

    def reset_clock(self) -> None:
        vp_server_reset_clock(self.handle)

    def set_policy(self, policy: int) -> None:
        vp_server_set_policy(self.handle, policy)

    def replay(self, jobs: list, arrival_ms, timeout_s: float = 60.0):
        return vp_server_replay(self.handle, jobs, arrival_ms, timeout_s)

    def stats(self) -> dict:
        return vp_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            vp_server_destroy(self.handle)
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


class Plan:
    """Owning handle of a vp_plan (destroys it on close / exit of a with-block)."""

    def __init__(self, K: int, M: int, qam: int, n_paths: int, tau: float = 0.0,
                 fp64_threshold: float | None = None, lam: float = 0.0, demap: int = 0, frac_bits: int = 0,
                 tensor_product: int = 0):
        self.K, self.M, self.qam, self.n_paths = K, M, qam, n_paths
        self.handle = vp_plan_create(K, M, qam, n_paths, tau)
        if fp64_threshold is not None:
            vp_plan_set_fp64_threshold(self.handle, fp64_threshold)
        if lam:
            vp_plan_set_lambda(self.handle, lam)
        if demap:
            vp_plan_set_demap(self.handle, demap)
        if frac_bits:
            vp_plan_set_fixed_point(self.handle, frac_bits)
        if tensor_product:
            vp_plan_set_tensor_product(self.handle, tensor_product)

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
